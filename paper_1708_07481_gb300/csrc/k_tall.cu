// Tall-skinny block updates of LOBPCG (Sec. IV: the O(n l) multi-vector work): projections
// R - X F, Cholesky-QR transforms V Tm, the Rayleigh-Ritz update [X R P] Y, the residual
// R = LX - X diag(theta) with its column norms, column gathers and the row normalization
// of the embedding (Sec. II.A).
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace sc {
namespace {


// out (n x b) = beta * Cin + A (n x a) * W (a x b).
// A CTA owns RT = 128 rows and a column slice of CB = 64 outputs; W streams through shared
// memory in chunks of KC rows, the A rows of the chunk are staged once per CTA (transposed,
// k-major, so a thread's 4 rows are one 16-byte read).  256 threads = 32 row groups x 8
// column groups; a thread keeps a 4-row x 8-column register tile (rows 4 rg .. 4 rg + 3,
// columns 8 cg .. 8 cg + 7) and reads 3 vectors of shared memory per k for 32 FMAs.
constexpr int RT = 128, CB = 64;

template <typename T> struct V4T;
template <> struct V4T<float> { using type = float4; };
template <> struct V4T<double> { using type = double4; };

template <typename T>
__global__ void __launch_bounds__(256)
    k_tall_gemm(long long n, Cat3<T> A, int a, const T* __restrict__ W, int ldw, int b,
                T* __restrict__ out, long long ldo, const T* Cin, long long ldc, T beta) {
  constexpr int KC = sizeof(T) == 4 ? 32 : 16;
  using V4 = typename V4T<T>::type;
  __shared__ __align__(16) T As[KC][RT + 4];  // +4: staging writes 4-way at worst, rows 16 B aligned
  __shared__ __align__(16) T Ws[KC][CB];
  __shared__ int mblk[KC], mlc[KC];
  const long long r0 = (long long)blockIdx.x * RT;
  const int c0 = blockIdx.y * CB;
  const int rg = threadIdx.x / 8;  // rows 4 rg .. 4 rg + 3
  const int cg = threadIdx.x % 8;  // cols 8 cg .. 8 cg + 7
  T acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0;
  for (int k0 = 0; k0 < a; k0 += KC) {
    if (threadIdx.x < KC) {
      int c = k0 + threadIdx.x, blk = -1, lc = 0, s = 0;
      for (int q = 0; q < A.nblk; ++q) {
        if (c >= s && c < s + A.c[q]) {
          blk = q;
          lc = c - s;
        }
        s += A.c[q];
      }
      mblk[threadIdx.x] = blk;
      mlc[threadIdx.x] = lc;
    }
    __syncthreads();
    {
      int kk = threadIdx.x % KC;
      int blk = mblk[kk];
      const T* p = blk >= 0 ? A.p[blk] : nullptr;
      long long ld = blk >= 0 ? A.ld[blk] : 0;
      int lc = mlc[kk];
#pragma unroll 4
      for (int rr = threadIdx.x / KC; rr < RT; rr += 256 / KC) {
        long long row = r0 + rr;
        As[kk][rr] = (blk >= 0 && row < n) ? p[row * ld + lc] : (T)0;
      }
    }
    for (int q = threadIdx.x; q < KC * CB; q += 256) {
      int kk = q / CB, cc = q % CB;
      int gk = k0 + kk, gc = c0 + cc;
      Ws[kk][cc] = (gk < a && gc < b) ? W[(long long)gk * ldw + gc] : (T)0;
    }
    __syncthreads();
    const int kmax = min(KC, a - k0);
#pragma unroll 4
    for (int k = 0; k < kmax; ++k) {
      const V4 av = *reinterpret_cast<const V4*>(&As[k][4 * rg]);
      const V4 w0 = *reinterpret_cast<const V4*>(&Ws[k][8 * cg]);
      const V4 w1 = *reinterpret_cast<const V4*>(&Ws[k][8 * cg + 4]);
      const T ar[4] = {av.x, av.y, av.z, av.w};
      const T wr[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(ar[i], wr[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long row = r0 + 4 * rg + i;
    if (row >= n) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int cc = c0 + 8 * cg + j;
      if (cc >= b) continue;
      T v = acc[i][j];
      if (Cin) v = fma(beta, Cin[row * ldc + cc], v);
      out[row * ldo + cc] = v;
    }
  }
}

// FP32 out (n x b) = beta * Cin + A (n x a) * W (a x b), for operand blocks whose segments
// start on 16-byte boundaries.  A CTA owns 128 rows and NB = 4 NCG output columns; the
// padded K dimension (each segment of A rounded up to 4 columns, zero-filled) streams through
// shared memory in stages of 32 with cp.async double buffering.  16 NCG threads: thread
// (tr, tc) keeps rows tr + 16 i (i < 8) x columns 4 tc .. 4 tc + 3 in registers and per
// 4 k reads 8 + 4 float4 of shared memory for 128 FMAs; rows interleaved by 16 keep the
// A reads of a warp on distinct banks.  Cin may alias out (each element is read, then
// written, by the same thread).
constexpr int TBM = 128, TKC = 32;

struct TallA {
  const float* p[3];
  long long ld[3];
  int c[3];     // logical columns of each segment
  int kpos[3];  // first padded-K position of each segment
  int wrow[3];  // first row of W for each segment
  int nseg;
  int kp;       // padded K
};

// Output columns [0, b0) go to segment 0, [b0, b) to segment 1.  Each segment has its own
// destination, accumulate input (Cin, may alias the destination), W block and number of
// leading rows of the concatenated A that it does not use (their W rows are zero).
struct TallOut {
  float* out[2];
  long long ldo[2];
  const float* cin[2];
  long long ldc[2];
  const float* w[2];
  int ldw[2];
  int wskip[2];
  int vec[2];  // float4 stores allowed in the segment
  int b0, b;
  float beta;
};

// W entry for logical row lr of the concatenated A and output column col.
__device__ __forceinline__ float tall_w(const TallOut& o, int lr, int col) {
  if (col >= o.b) return 0.f;
  const bool s1 = col >= o.b0;
  const int skip = s1 ? o.wskip[1] : o.wskip[0];
  if (lr < skip) return 0.f;
  const float* w = s1 ? o.w[1] : o.w[0];
  const int ldw = s1 ? o.ldw[1] : o.ldw[0];
  return w[(long long)(lr - skip) * ldw + (s1 ? col - o.b0 : col)];
}

// out[row][col .. col + 3] = v + beta * Cin for the columns below b.
__device__ __forceinline__ void tall_store(const TallOut& o, long long row, int col,
                                           const float (&v)[4]) {
  const bool s1 = col >= o.b0;
  const int cs = s1 ? col - o.b0 : col;
  const int bs = s1 ? o.b - o.b0 : o.b0;
  if ((s1 ? o.vec[1] : o.vec[0]) && cs + 3 < bs) {
    float* out = s1 ? o.out[1] : o.out[0];
    const long long ldo = s1 ? o.ldo[1] : o.ldo[0];
    const float* cin = s1 ? o.cin[1] : o.cin[0];
    const long long ldc = s1 ? o.ldc[1] : o.ldc[0];
    float r[4] = {v[0], v[1], v[2], v[3]};
    if (cin) {
      const float4 c = *reinterpret_cast<const float4*>(cin + row * ldc + cs);
      r[0] = fmaf(o.beta, c.x, r[0]);
      r[1] = fmaf(o.beta, c.y, r[1]);
      r[2] = fmaf(o.beta, c.z, r[2]);
      r[3] = fmaf(o.beta, c.w, r[3]);
    }
    *reinterpret_cast<float4*>(out + row * ldo + cs) = make_float4(r[0], r[1], r[2], r[3]);
    return;
  }
  for (int j = 0; j < 4; ++j) {
    const int c = col + j;
    if (c >= o.b) break;
    const bool t1 = c >= o.b0;
    const int ct = t1 ? c - o.b0 : c;
    float* out = t1 ? o.out[1] : o.out[0];
    const long long ldo = t1 ? o.ldo[1] : o.ldo[0];
    const float* cin = t1 ? o.cin[1] : o.cin[0];
    const long long ldc = t1 ? o.ldc[1] : o.ldc[0];
    float x = v[j];
    if (cin) x = fmaf(o.beta, cin[row * ldc + ct], x);
    out[row * ldo + ct] = x;
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int NCG>
__global__ void __launch_bounds__(16 * NCG)
    k_tall_f32(long long n, TallA A, TallOut o) {
  constexpr int NB = 4 * NCG, NTH = 16 * NCG;
  extern __shared__ __align__(16) float tsm[];
  float(*As)[TBM][TKC + 4] = reinterpret_cast<float(*)[TBM][TKC + 4]>(tsm);
  float(*Ws)[TKC][NB] = reinterpret_cast<float(*)[TKC][NB]>(tsm + 2 * TBM * (TKC + 4));
  const long long r0 = (long long)blockIdx.x * TBM;
  const int c0 = blockIdx.y * NB;
  const int tc = threadIdx.x % NCG, tr = threadIdx.x / NCG;
  const int nst = (A.kp + TKC - 1) / TKC;

  auto load_stage = [&](int s, int buf) {
    for (int q = threadIdx.x; q < TBM * (TKC / 4); q += NTH) {
      const int r = q / (TKC / 4), c4 = q % (TKC / 4);
      const int kk = s * TKC + 4 * c4;
      const bool g1 = A.nseg > 1 && kk >= A.kpos[1], g2 = A.nseg > 2 && kk >= A.kpos[2];
      const float* pg = g2 ? A.p[2] : (g1 ? A.p[1] : A.p[0]);
      const long long ldg = g2 ? A.ld[2] : (g1 ? A.ld[1] : A.ld[0]);
      const int lc = kk - (g2 ? A.kpos[2] : (g1 ? A.kpos[1] : 0));
      const int cg = g2 ? A.c[2] : (g1 ? A.c[1] : A.c[0]);
      int valid = kk < A.kp ? min(4, cg - lc) : 0;
      const long long row = r0 + r;
      if (row >= n || valid < 0) valid = 0;
      const float* src = valid > 0 ? pg + row * ldg + lc : A.p[0];
      cp_async16(&As[buf][r][4 * c4], src, 4 * valid);
    }
    for (int q = threadIdx.x; q < TKC * NB; q += NTH) {
      const int kl = q / NB, cc = q % NB;
      const int kk = s * TKC + kl;
      const bool g1 = A.nseg > 1 && kk >= A.kpos[1], g2 = A.nseg > 2 && kk >= A.kpos[2];
      const int lc = kk - (g2 ? A.kpos[2] : (g1 ? A.kpos[1] : 0));
      const int cg = g2 ? A.c[2] : (g1 ? A.c[1] : A.c[0]);
      const int wr = g2 ? A.wrow[2] : (g1 ? A.wrow[1] : 0);
      const int col = c0 + cc;
      Ws[buf][kl][cc] = (kk < A.kp && lc < cg) ? tall_w(o, wr + lc, col) : 0.f;
    }
  };

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  load_stage(0, 0);
  cp_async_commit();
  for (int s = 0; s < nst; ++s) {
    const int buf = s & 1;
    if (s + 1 < nst) load_stage(s + 1, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const int kend = min(TKC, A.kp - s * TKC);  // a multiple of 4
    for (int k = 0; k < kend; k += 4) {
      float4 a[8], w[4];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = *reinterpret_cast<const float4*>(&As[buf][tr + 16 * i][k]);
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = *reinterpret_cast<const float4*>(&Ws[buf][k + q][4 * tc]);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float av[4] = {a[i].x, a[i].y, a[i].z, a[i].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[i][0] = fmaf(av[q], w[q].x, acc[i][0]);
          acc[i][1] = fmaf(av[q], w[q].y, acc[i][1]);
          acc[i][2] = fmaf(av[q], w[q].z, acc[i][2]);
          acc[i][3] = fmaf(av[q], w[q].w, acc[i][3]);
        }
      }
    }
    __syncthreads();
  }
  const int col = c0 + 4 * tc;
  if (col >= o.b) return;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long row = r0 + tr + 16 * i;
    if (row >= n) break;
    const float v[4] = {acc[i][0], acc[i][1], acc[i][2], acc[i][3]};
    tall_store(o, row, col, v);
  }
}

// FP32 tall update for padded K <= KMAX (every LOBPCG update at K <= 48): each CTA keeps
// its slice of W (Kp x NB, zero-padded) in shared memory for all its row tiles and walks row
// tiles of 64 rows, prefetching the next tile's whole K extent with cp.async while it
// computes the current one.  16 NCG threads: thread (tr, tc) owns rows tr + 16 i (i < 4)
// and columns 4 tc .. 4 tc + 3; per 4 k it reads 4 + 4 float4 for 64 FMAs.
constexpr int RBM = 64, KMAX = 96;

template <int NCG>
__global__ void __launch_bounds__(16 * NCG)
    k_tall_rt(long long n, TallA A, TallOut o, int ntiles) {
  constexpr int NB = 4 * NCG, NTH = 16 * NCG;
  extern __shared__ __align__(16) float rsm[];
  const int kp = A.kp;
  const int lda_s = kp + 4;  // shared row stride of the A tiles
  float* Ws = rsm;                         // kp x NB
  float* As0 = rsm + kp * NB;              // 2 x RBM x lda_s
  const int c0 = blockIdx.y * NB;
  const int tc = threadIdx.x % NCG, tr = threadIdx.x / NCG;
  auto load_tile = [&](int t, float* dst) {
    const long long r0 = (long long)t * RBM;
    const int nc4 = kp / 4;
    for (int q = threadIdx.x; q < RBM * nc4; q += NTH) {
      const int r = q / nc4, c4 = q % nc4;
      const int kk = 4 * c4;
      const bool g1 = A.nseg > 1 && kk >= A.kpos[1], g2 = A.nseg > 2 && kk >= A.kpos[2];
      const float* pg = g2 ? A.p[2] : (g1 ? A.p[1] : A.p[0]);
      const long long ldg = g2 ? A.ld[2] : (g1 ? A.ld[1] : A.ld[0]);
      const int lc = kk - (g2 ? A.kpos[2] : (g1 ? A.kpos[1] : 0));
      const int cg = g2 ? A.c[2] : (g1 ? A.c[1] : A.c[0]);
      int valid = min(4, cg - lc);
      const long long row = r0 + r;
      if (row >= n || valid < 0) valid = 0;
      const float* src = valid > 0 ? pg + row * ldg + lc : A.p[0];
      cp_async16(dst + r * lda_s + kk, src, 4 * valid);
    }
  };
  int t = blockIdx.x;
  if (t < ntiles) load_tile(t, As0);
  cp_async_commit();
  // W slice, zero-padded (rows of padding columns, columns past b), while the tile lands
  for (int q = threadIdx.x; q < kp * NB; q += NTH) {
    const int kk = q / NB, cc = q % NB;
    const bool g1 = A.nseg > 1 && kk >= A.kpos[1], g2 = A.nseg > 2 && kk >= A.kpos[2];
    const int lc = kk - (g2 ? A.kpos[2] : (g1 ? A.kpos[1] : 0));
    const int cg = g2 ? A.c[2] : (g1 ? A.c[1] : A.c[0]);
    const int wr = g2 ? A.wrow[2] : (g1 ? A.wrow[1] : 0);
    Ws[q] = lc < cg ? tall_w(o, wr + lc, c0 + cc) : 0.f;
  }
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    float* As = As0 + (it & 1) * RBM * lda_s;
    const int tn = t + gridDim.x;
    if (tn < ntiles) load_tile(tn, As0 + ((it + 1) & 1) * RBM * lda_s);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k = 0; k < kp; k += 4) {
      float4 a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(As + (tr + 16 * i) * lda_s + k);
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = *reinterpret_cast<const float4*>(Ws + (k + q) * NB + 4 * tc);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float av[4] = {a[i].x, a[i].y, a[i].z, a[i].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[i][0] = fmaf(av[q], w[q].x, acc[i][0]);
          acc[i][1] = fmaf(av[q], w[q].y, acc[i][1]);
          acc[i][2] = fmaf(av[q], w[q].z, acc[i][2]);
          acc[i][3] = fmaf(av[q], w[q].w, acc[i][3]);
        }
      }
    }
    const int col = c0 + 4 * tc;
    if (col < o.b) {
      const long long r0 = (long long)t * RBM;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const long long row = r0 + tr + 16 * i;
        if (row >= n) break;
        const float v[4] = {acc[i][0], acc[i][1], acc[i][2], acc[i][3]};
        tall_store(o, row, col, v);
      }
    }
    __syncthreads();  // this buffer is refilled two tiles later
  }
}

// R = LX - X diag(theta) over columns [0, K) and the squared column norms.  A thread sums the
// squares of its rows in the arithmetic of T (FP32 rows: relative error ~ rows x eps32, far
// below the rounding of R itself), the row groups of a CTA and the CTA partials are added in
// FP64 in fixed orders; the last CTA to finish (ticket) sums the partials with 8 warps
// (warp w takes partials w, w + 8, ...) and adds the 8 warp sums in warp order.
// Jacobi preconditioner entry: r / d, or r itself for an isolated vertex (d = 0).
template <typename T>
__device__ __forceinline__ T jacobi(T r, T d) {
  return d > (T)0 ? r / d : r;
}

template <typename T, bool PRE>
__global__ void __launch_bounds__(256)
    k_residual(long long n, int K, const T* __restrict__ X, const T* __restrict__ LX,
               long long ld, const double* __restrict__ theta, T* __restrict__ R,
               long long rows_per_cta, double* part, int* ticket, double* rho2,
               const T* __restrict__ deg) {
  extern __shared__ double sred[];  // [rp][kc], reused as [8][K] by the last CTA
  __shared__ int last;
  const int kc = K < 256 ? K : 256;
  const int rp = 256 / kc;                 // rows in parallel
  const int col0 = threadIdx.x % kc;
  const int rl = threadIdx.x / kc;
  long long r0 = blockIdx.x * rows_per_cta, r1 = r0 + rows_per_cta;
  if (r1 > n) r1 = n;
  for (int cb = 0; cb < K; cb += kc) {
    int j = cb + col0;
    T s0 = 0, s1 = 0;
    if (rl < rp && j < K) {
      const T th = (T)theta[j];
      long long r = r0 + rl;
      for (; r + rp < r1; r += 2 * rp) {
        const T v0 = LX[r * ld + j] - X[r * ld + j] * th;
        const T v1 = LX[(r + rp) * ld + j] - X[(r + rp) * ld + j] * th;
        R[r * ld + j] = PRE ? jacobi(v0, deg[r]) : v0;
        R[(r + rp) * ld + j] = PRE ? jacobi(v1, deg[r + rp]) : v1;
        s0 = fma(v0, v0, s0);
        s1 = fma(v1, v1, s1);
      }
      if (r < r1) {
        const T v0 = LX[r * ld + j] - X[r * ld + j] * th;
        R[r * ld + j] = PRE ? jacobi(v0, deg[r]) : v0;
        s0 = fma(v0, v0, s0);
      }
    }
    if (rl < rp) sred[rl * kc + col0] = (double)s0 + (double)s1;
    __syncthreads();
    if (threadIdx.x < kc && cb + threadIdx.x < K) {
      double t = 0.0;
      for (int q = 0; q < rp; ++q) t += sred[q * kc + threadIdx.x];
      part[(long long)blockIdx.x * K + cb + threadIdx.x] = t;
    }
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j0 = 0; j0 < K; j0 += 32) {
    const int j = j0 + lane;
    double t0 = 0.0, t1 = 0.0;
    if (j < K) {
      unsigned c = w;
      for (; c + 8 < gridDim.x; c += 16) {
        t0 += __ldcg(part + (long long)c * K + j);
        t1 += __ldcg(part + (long long)(c + 8) * K + j);
      }
      if (c < gridDim.x) t0 += __ldcg(part + (long long)c * K + j);
    }
    sred[w * 32 + lane] = t0 + t1;
    __syncthreads();
    if (w == 0 && j < K) {
      double v = sred[lane];
#pragma unroll
      for (int q = 1; q < 8; ++q) v += sred[q * 32 + lane];
      rho2[j] = v;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0;
}

template <typename T>
__global__ void k_gather_cols(long long n, const T* __restrict__ src, long long lds,
                              T* __restrict__ dst, long long ldd, const int* __restrict__ cols,
                              int kc) {
  long long tot = n * kc;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    long long r = idx / kc;
    int j = (int)(idx % kc);
    dst[r * ldd + j] = src[r * lds + cols[j]];
  }
}

// Warp per row: E_i = X_i / ||X_i||_2 (FP64 norm); rows with norm < 1e-30 become zero.
template <typename T>
__global__ void k_rownorm(long long n, int K, const T* __restrict__ X, long long ldx,
                          float* __restrict__ E, long long lde) {
  int lane = threadIdx.x & 31;
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = w; r < n; r += nw) {
    double s = 0.0;
    for (int j = lane; j < K; j += 32) {
      double v = (double)X[r * ldx + j];
      s += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    double nr = sqrt(s);
    double inv = nr >= 1e-30 ? 1.0 / nr : 0.0;
    for (int j = lane; j < K; j += 32) E[r * lde + j] = (float)((double)X[r * ldx + j] * inv);
  }
}

template <typename T>
__global__ void k_cast(int rows, int cols, const double* __restrict__ src, int lds,
                       T* __restrict__ dst, int ldd, double scale) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rows * cols;
       idx += gridDim.x * blockDim.x) {
    int i = idx / cols, j = idx % cols;
    dst[(long long)i * ldd + j] = (T)(scale * src[(long long)i * lds + j]);
  }
}

// dst (rows x cols, To, row stride ldd) = src (rows x cols, Ti, row stride lds), converted.
template <typename Ti, typename To>
__global__ void k_convert(long long rows, int cols, const Ti* __restrict__ src, long long lds,
                          To* __restrict__ dst, long long ldd) {
  const long long total = rows * cols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx / cols;
    const int j = (int)(idx - i * cols);
    dst[i * ldd + j] = (To)src[i * lds + j];
  }
}

__device__ inline unsigned long long d_sm64(unsigned long long key, unsigned long long i) {
  unsigned long long z = key + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_gauss(long long count, int K, unsigned long long key, T* X, long long ldx) {
  const double two_pi = 6.283185307179586;
  long long npair = (count + 1) / 2;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npair;
       p += (long long)gridDim.x * blockDim.x) {
    double u1 = (double)(d_sm64(key, 2 * p) >> 11) * (1.0 / 9007199254740992.0);
    double u2 = (double)(d_sm64(key, 2 * p + 1) >> 11) * (1.0 / 9007199254740992.0);
    double r = sqrt(-2.0 * log1p(-u1));
    double sn, cs;
    sincos(two_pi * u2, &sn, &cs);
    long long e0 = 2 * p, e1 = 2 * p + 1;
    X[(e0 / K) * ldx + e0 % K] = (T)(float)(r * cs);
    if (e1 < count) X[(e1 / K) * ldx + e1 % K] = (T)(float)(r * sn);
  }
}

inline unsigned cap_grid(long long g, long long cap) {
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

template <typename T>
cudaError_t tall_gemm2(cudaStream_t st, long long n, const Cat3<T>& A, const TallSeg<T>& s0,
                       const TallSeg<T>& s1, T beta, int* d_status, bool use_tc) {
  const int b = s0.b + s1.b;
  if (n == 0 || b == 0) return cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    if (use_tc) {
      const cudaError_t e = tall_gemm_tc(st, n, A, s0, s1, beta, d_status);
      if (e != cudaErrorNotSupported) return e;
    }
    // cp.async kernels: A segments 16-byte aligned.  Each segment is read up to its column
    // count rounded up to 4 (inside its row); the extra columns are zero-filled in shared
    // memory and meet zero rows of W.
    bool ok = true;
    TallA ta{};
    ta.nseg = A.nblk;
    int kp = 0, wr = 0;
    for (int q = 0; q < A.nblk; ++q) {
      ok = ok && ((uintptr_t)A.p[q] & 15) == 0 && (A.ld[q] & 3) == 0;
      ta.p[q] = A.p[q];
      ta.ld[q] = A.ld[q];
      ta.c[q] = A.c[q];
      ta.kpos[q] = kp;
      ta.wrow[q] = wr;
      kp += (A.c[q] + 3) & ~3;
      wr += A.c[q];
    }
    ta.kp = kp;
    TallOut to{};
    const TallSeg<T>* sg[2] = {&s0, &s1};
    for (int q = 0; q < 2; ++q) {
      const TallSeg<T>& g = *sg[q];
      to.out[q] = (float*)g.out;
      to.ldo[q] = g.ldo;
      to.cin[q] = (const float*)g.Cin;
      to.ldc[q] = g.ldc;
      to.w[q] = (const float*)g.W;
      to.ldw[q] = g.ldw;
      to.wskip[q] = g.wskip;
      to.vec[q] = g.b > 0 && ((uintptr_t)g.out & 15) == 0 && (g.ldo & 3) == 0 &&
                  (!g.Cin || (((uintptr_t)g.Cin & 15) == 0 && (g.ldc & 3) == 0)) &&
                  (q == 0 || (s0.b & 3) == 0);
    }
    to.b0 = s0.b;
    to.b = b;
    to.beta = (float)beta;
    if (ok && kp > 0 && kp <= KMAX) {
      ProfScope ps(st, "tall_gemm");
      const int b4 = (b + 3) & ~3;
      const int ntiles = (int)((n + RBM - 1) / RBM);
      auto smem = [&](int nb) { return sizeof(float) * ((size_t)kp * nb + 2 * RBM * (kp + 4)); };
      constexpr size_t max12 = sizeof(float) * ((size_t)KMAX * 48 + 2 * RBM * (KMAX + 4));
      constexpr size_t max24 = sizeof(float) * ((size_t)KMAX * 96 + 2 * RBM * (KMAX + 4));
      static std::once_flag rt_once;
      std::call_once(rt_once, [] {
        cudaFuncSetAttribute(k_tall_rt<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max12);
        cudaFuncSetAttribute(k_tall_rt<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max24);
      });
      // resident CTAs per SM for this shared-memory size (registers and shared memory)
      auto fit = [&](auto kern, size_t sm, int threads) {
        int nb = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, sm) != cudaSuccess)
          nb = 1;
        return std::max(1, nb);
      };
      if (b4 <= 48) {
        const int per_sm = fit(k_tall_rt<12>, smem(48), 16 * 12);
        dim3 grid((unsigned)std::min(ntiles, 152 * per_sm), 1);
        k_tall_rt<12><<<grid, 16 * 12, smem(48), st>>>(n, ta, to, ntiles);
      } else {
        const int ncol = (b4 + 95) / 96;
        const int per_sm = fit(k_tall_rt<24>, smem(96), 16 * 24);
        dim3 grid((unsigned)std::max(1, std::min(ntiles, 152 * per_sm / ncol)), (unsigned)ncol);
        k_tall_rt<24><<<grid, 16 * 24, smem(96), st>>>(n, ta, to, ntiles);
      }
      note_launch();
      return cudaGetLastError();
    }
    if (ok && kp > 0) {
      ProfScope ps(st, "tall_gemm");
      const int b4 = (b + 3) & ~3;
      constexpr size_t sm12 = sizeof(float) * (2 * TBM * (TKC + 4) + 2 * TKC * 48);
      constexpr size_t sm24 = sizeof(float) * (2 * TBM * (TKC + 4) + 2 * TKC * 96);
      static std::once_flag attr_once;
      std::call_once(attr_once, [] {
        cudaFuncSetAttribute(k_tall_f32<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm12);
        cudaFuncSetAttribute(k_tall_f32<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm24);
      });
      if (b4 <= 48) {
        dim3 grid((unsigned)((n + TBM - 1) / TBM), 1);
        k_tall_f32<12><<<grid, 16 * 12, sm12, st>>>(n, ta, to);
      } else {
        dim3 grid((unsigned)((n + TBM - 1) / TBM), (unsigned)((b4 + 95) / 96));
        k_tall_f32<24><<<grid, 16 * 24, sm24, st>>>(n, ta, to);
      }
      note_launch();
      return cudaGetLastError();
    }
  }
  // generic kernel, one launch per output segment; a segment that skips the leading rows of
  // W uses A without the leading segments those rows belong to
  const TallSeg<T>* sg[2] = {&s0, &s1};
  for (int q = 0; q < 2; ++q) {
    const TallSeg<T>& g = *sg[q];
    if (g.b == 0) continue;
    Cat3<T> Aq{};
    int skip = g.wskip, first = 0;
    while (skip > 0 && first < A.nblk && A.c[first] <= skip) skip -= A.c[first++];
    if (skip != 0) return cudaErrorInvalidValue;
    for (int i = first; i < A.nblk; ++i) {
      Aq.p[Aq.nblk] = A.p[i];
      Aq.ld[Aq.nblk] = A.ld[i];
      Aq.c[Aq.nblk] = A.c[i];
      ++Aq.nblk;
    }
    const int a = Aq.cols();
    dim3 grid((unsigned)((n + RT - 1) / RT), (unsigned)((g.b + CB - 1) / CB));
    ProfScope ps(st, "tall_gemm");
    k_tall_gemm<T><<<grid, 256, 0, st>>>(n, Aq, a, g.W, g.ldw, g.b, g.out, g.ldo, g.Cin, g.ldc,
                                         beta);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t tall_gemm(cudaStream_t st, long long n, const Cat3<T>& A, const T* W, int ldw,
                      int b, T* out, long long ldo, const T* Cin, long long ldc, T beta,
                      int* d_status, bool use_tc) {
  TallSeg<T> s0{out, ldo, Cin, ldc, W, ldw, 0, b};
  TallSeg<T> s1{};
  return tall_gemm2<T>(st, n, A, s0, s1, beta, d_status, use_tc);
}

template <typename T>
cudaError_t residual(cudaStream_t st, Alloc& al, long long n, int K, const T* X, const T* LX,
                     long long ld, const double* theta, T* R, double* rho2, const T* deg) {
  long long nct = cap_grid((n + 255) / 256, 152 * 2);
  long long rpc = (n + nct - 1) / nct;
  if (rpc < 1) rpc = 1;
  nct = (n + rpc - 1) / rpc;
  if (nct < 1) nct = 1;
  double* part = al.get<double>((size_t)nct * K);
  int* ticket = al.get<int>(1);
  if (!part || !ticket) {
    al.put(part);
    al.put(ticket);
    return cudaErrorMemoryAllocation;
  }
  cudaMemsetAsync(ticket, 0, sizeof(int), st);
  int kc = K < 256 ? K : 256;
  int rp = 256 / kc;
  size_t sm = sizeof(double) * std::max<size_t>((size_t)rp * kc, 8 * 32);
  ProfScope ps(st, "residual");
  if (deg)
    k_residual<T, true><<<(unsigned)nct, 256, sm, st>>>(n, K, X, LX, ld, theta, R, rpc, part,
                                                        ticket, rho2, deg);
  else
    k_residual<T, false><<<(unsigned)nct, 256, sm, st>>>(n, K, X, LX, ld, theta, R, rpc, part,
                                                         ticket, rho2, deg);
  note_launch();
  cudaError_t e = cudaGetLastError();
  al.put(part);
  al.put(ticket);
  return e;
}

template <typename T>
cudaError_t gather_cols(cudaStream_t st, long long n, const T* src, long long lds, T* dst,
                        long long ldd, const int* cols, int kc) {
  long long tot = n * kc;
  if (tot == 0) return cudaSuccess;
  k_gather_cols<T><<<cap_grid((tot + 255) / 256, 152 * 16), 256, 0, st>>>(n, src, lds, dst, ldd,
                                                                          cols, kc);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t rownorm(cudaStream_t st, long long n, int K, const T* X, long long ldx, float* E,
                    long long lde) {
  if (n == 0) return cudaSuccess;
  k_rownorm<T><<<cap_grid((n * 32 + 255) / 256, 152 * 16), 256, 0, st>>>(n, K, X, ldx, E, lde);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t gauss_block(cudaStream_t st, long long n, int K, unsigned long long key, T* X,
                        long long ldx) {
  long long count = n * K;
  if (count == 0) return cudaSuccess;
  ProfScope ps(st, "gauss");
  k_gauss<T><<<cap_grid((count / 2 + 255) / 256, 152 * 8), 256, 0, st>>>(count, K, key, X, ldx);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t cast_mat(cudaStream_t st, int rows, int cols, const double* src, int lds, T* dst,
                     int ldd, double scale) {
  if (rows * cols == 0) return cudaSuccess;
  k_cast<T><<<cap_grid((rows * cols + 255) / 256, 152), 256, 0, st>>>(rows, cols, src, lds, dst,
                                                                     ldd, scale);
  note_launch();
  return cudaGetLastError();
}

template <typename Ti, typename To>
cudaError_t convert_mat(cudaStream_t st, long long rows, int cols, const Ti* src, long long lds,
                        To* dst, long long ldd) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const long long blocks = (rows * cols + 255) / 256;
  k_convert<Ti, To><<<cap_grid(blocks, 4 * 152), 256, 0, st>>>(rows, cols, src, lds, dst, ldd);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t convert_mat<float, double>(cudaStream_t, long long, int, const float*,
                                                long long, double*, long long);
template cudaError_t convert_mat<double, float>(cudaStream_t, long long, int, const double*,
                                                long long, float*, long long);

#define SC_INST(T)                                                                          \
  template cudaError_t gauss_block<T>(cudaStream_t, long long, int, unsigned long long, T*,  \
                                      long long);                                            \
  template cudaError_t cast_mat<T>(cudaStream_t, int, int, const double*, int, T*, int,      \
                                   double);                                                  \
  template cudaError_t tall_gemm<T>(cudaStream_t, long long, const Cat3<T>&, const T*, int,  \
                                    int, T*, long long, const T*, long long, T, int*, bool); \
  template cudaError_t tall_gemm2<T>(cudaStream_t, long long, const Cat3<T>&,                \
                                     const TallSeg<T>&, const TallSeg<T>&, T, int*, bool);   \
  template cudaError_t residual<T>(cudaStream_t, Alloc&, long long, int, const T*, const T*, \
                                   long long, const double*, T*, double*, const T*);         \
  template cudaError_t gather_cols<T>(cudaStream_t, long long, const T*, long long, T*,      \
                                      long long, const int*, int);                           \
  template cudaError_t rownorm<T>(cudaStream_t, long long, int, const T*, long long, float*, \
                                  long long);
SC_INST(float)
SC_INST(double)
#undef SC_INST

}  // namespace sc
