// Tall-skinny block updates of LOBPCG (Sec. IV: the O(n l) multi-vector work): projections
// R - X F, Cholesky-QR transforms V Tm, the Rayleigh-Ritz update [X R P] Y, the residual
// R = LX - X diag(theta) with its column norms, column gathers and the row normalization
// of the embedding (Sec. II.A).
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

// R = LX - X diag(theta) over columns [0, K); per-CTA FP64 column sums of R^2, reduced in
// fixed CTA order by the last CTA (ticket counter).
template <typename T>
__global__ void __launch_bounds__(256)
    k_residual(long long n, int K, const T* __restrict__ X, const T* __restrict__ LX,
               long long ld, const double* __restrict__ theta, T* __restrict__ R,
               long long rows_per_cta, double* part, int* ticket, double* rho2) {
  extern __shared__ double sred[];  // [rp][K]
  __shared__ int last;
  const int kc = K < 256 ? K : 256;
  const int rp = 256 / kc;                 // rows in parallel
  const int col0 = threadIdx.x % kc;
  const int rl = threadIdx.x / kc;
  long long r0 = blockIdx.x * rows_per_cta, r1 = r0 + rows_per_cta;
  if (r1 > n) r1 = n;
  for (int cb = 0; cb < K; cb += kc) {
    int j = cb + col0;
    double s = 0.0;
    if (rl < rp && j < K) {
      T th = (T)theta[j];
      for (long long r = r0 + rl; r < r1; r += rp) {
        T v = LX[r * ld + j] - X[r * ld + j] * th;
        R[r * ld + j] = v;
        s += (double)v * (double)v;
      }
    }
    if (rl < rp) sred[rl * kc + col0] = s;
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
  // fixed-order sum over the CTA partials: 8 independent loads in flight per step
  for (int j = threadIdx.x; j < K; j += blockDim.x) {
    double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned c = 0;
    for (; c + 8 <= gridDim.x; c += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] += __ldcg(part + (long long)(c + u) * K + j);
    }
    for (; c < gridDim.x; ++c) t[0] += __ldcg(part + (long long)c * K + j);
    rho2[j] = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
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
cudaError_t tall_gemm(cudaStream_t st, long long n, const Cat3<T>& A, const T* W, int ldw,
                      int b, T* out, long long ldo, const T* Cin, long long ldc, T beta) {
  int a = A.cols();
  if (n == 0 || b == 0) return cudaSuccess;
  dim3 grid((unsigned)((n + RT - 1) / RT), (unsigned)((b + CB - 1) / CB));
  ProfScope ps(st, "tall_gemm");
  k_tall_gemm<T><<<grid, 256, 0, st>>>(n, A, a, W, ldw, b, out, ldo, Cin, ldc, beta);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t residual(cudaStream_t st, Alloc& al, long long n, int K, const T* X, const T* LX,
                     long long ld, const double* theta, T* R, double* rho2) {
  long long nct = cap_grid((n + 63) / 64, 152 * 4);
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
  size_t sm = sizeof(double) * (size_t)rp * kc;
  ProfScope ps(st, "residual");
  k_residual<T><<<(unsigned)nct, 256, sm, st>>>(n, K, X, LX, ld, theta, R, rpc, part, ticket,
                                                 rho2);
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

#define SC_INST(T)                                                                          \
  template cudaError_t gauss_block<T>(cudaStream_t, long long, int, unsigned long long, T*,  \
                                      long long);                                            \
  template cudaError_t cast_mat<T>(cudaStream_t, int, int, const double*, int, T*, int,      \
                                   double);                                                  \
  template cudaError_t tall_gemm<T>(cudaStream_t, long long, const Cat3<T>&, const T*, int,  \
                                    int, T*, long long, const T*, long long, T);             \
  template cudaError_t residual<T>(cudaStream_t, Alloc&, long long, int, const T*, const T*, \
                                   long long, const double*, T*, double*);                   \
  template cudaError_t gather_cols<T>(cudaStream_t, long long, const T*, long long, T*,      \
                                      long long, const int*, int);                           \
  template cudaError_t rownorm<T>(cudaStream_t, long long, int, const T*, long long, float*, \
                                  long long);
SC_INST(float)
SC_INST(double)
#undef SC_INST

}  // namespace sc
