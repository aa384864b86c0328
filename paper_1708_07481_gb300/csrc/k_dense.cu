// Small dense solves of one LOBPCG pass, one CTA each.
//
// chol_inv: Cholesky-QR transform of a block V (Sec. II.B: the multi-vector blocks are kept
//   orthonormal, as SciPy's lobpcg does).  From the FP64 Gram G = V'V: scale s = diag(G)^-1/2,
//   Cholesky s G s = C C' in FP64, Tm = diag(s) C^-T so that V Tm has orthonormal columns.
//
// rr_eig: Rayleigh-Ritz in an orthonormal trial basis [X R P] (Knyazev 2001): the K smallest
//   eigenpairs of the symmetric m x m matrix G = S' L S, in the arithmetic of T:
//     1. Householder reduction to tridiagonal form Q' G Q = T (Golub & Van Loan, Alg. 8.3.1),
//     2. the K smallest eigenvalues of T by multisection on Sturm counts (32 points per warp
//        step, Barth, Martin & Wilkinson 1967 bisection generalised),
//     3. eigenvectors of T by inverse iteration with tridiagonal LU and partial pivoting,
//        re-orthogonalised in order by two passes of classical Gram-Schmidt each sweep,
//     4. back-transformation Y = Q Z with the stored reflectors.
//   In an orthonormal basis the problem is perfectly conditioned, so FP32 arithmetic gives
//   Ritz values to ~eps32 * ||G||; the FP64 instantiation is the plain/check form.
#include <cfloat>

#include "common.cuh"

namespace sc {
namespace {

// Copies the rows x cols FP64 matrix G (row stride ldg) into shared memory Gs (stride cols)
// with nth threads: each thread's loads of a batch of 8 are issued before any of them is stored,
// so eight reads per thread are in flight instead of one.
__device__ __forceinline__ void stage_f64(const double* __restrict__ G, long long ldg, int rows,
                                          int cols, double* Gs, int tid, int nth) {
  const int tot = rows * cols;
  for (int base = tid; base < tot; base += 8 * nth) {
    double t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * nth;
      t[u] = idx < tot ? G[(long long)(idx / cols) * ldg + idx % cols] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int idx = base + u * nth;
      if (idx < tot) Gs[idx] = t[u];
    }
  }
}

template <typename T> struct Lim;
template <> struct Lim<float> {
  __device__ static float eps() { return FLT_EPSILON; }
  __device__ static float tiny() { return FLT_MIN; }
};
template <> struct Lim<double> {
  __device__ static double eps() { return DBL_EPSILON; }
  __device__ static double tiny() { return DBL_MIN; }
};

// Block-wide sum; every thread gets the result.  red: >= 33 slots of shared scratch.
template <typename T>
__device__ T block_sum(T v, T* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? red[lane] : (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  T r = red[32];
  __syncthreads();
  return r;
}

template <typename T>
__device__ T block_max(T v, T* red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? red[lane] : (T)(-1e300 < -3e38 ? -3e38 : -1e300);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = max(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  T r = red[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------------------
// ---- block-wide small dense kernels (all threads of the CTA take part) -------------------

// In-place lower Cholesky of the ka x ka matrix W (stride ldw) in the arithmetic of T.
// rdiag[k] = 1 / L_kk.  Returns the first column whose pivot is <= tol (or -1).
template <typename T>
__device__ int blk_chol(int ka, T* W, int ldw, T* rdiag, T tol, int* sflag) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  if (tid == 0) *sflag = -1;
  __syncthreads();
  for (int k = 0; k < ka; ++k) {
    if (tid == 0) {
      T piv = W[k * ldw + k];
      if (!(piv > tol)) {
        *sflag = k;
      } else {
        T r = rsqrt(piv);
        rdiag[k] = r;
        W[k * ldw + k] = piv * r;
      }
    }
    __syncthreads();
    if (*sflag >= 0) return *sflag;
    const T r = rdiag[k];
    for (int i = k + 1 + tid; i < ka; i += nt) W[i * ldw + k] *= r;
    __syncthreads();
    for (int i = k + 1 + warp; i < ka; i += nw) {
      const T lik = W[i * ldw + k];
      T* wi = W + i * ldw;
#pragma unroll 4
      for (int j = k + 1 + lane; j <= i; j += 32) wi[j] = fma(-lik, W[j * ldw + k], wi[j]);
    }
    __syncthreads();
  }
  return -1;
}

// Linv = L^-1 (lower, ka x ka, stride ldi) from the factor in W and rdiag, row by row:
// Linv[i][j] = -rdiag[i] * sum_{q=j}^{i-1} L[i][q] Linv[q][j]; one warp per (i, j), lanes
// split q.
template <typename T>
__device__ void blk_tri_inv(int ka, const T* W, int ldw, const T* rdiag, T* Li, int ldi) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int idx = tid; idx < ka * ka; idx += nt) {
    int i = idx / ka, j = idx % ka;
    Li[i * ldi + j] = (i == j) ? rdiag[i] : (T)0;
  }
  __syncthreads();
  for (int i = 1; i < ka; ++i) {
    const T* li = W + i * ldw;
    for (int j = warp; j < i; j += nw) {
      T a0 = 0, a1 = 0;
      int q = j + lane;
      for (; q + 32 < i; q += 64) {
        a0 = fma(li[q], Li[q * ldi + j], a0);
        a1 = fma(li[q + 32], Li[(q + 32) * ldi + j], a1);
      }
      if (q < i) a0 = fma(li[q], Li[q * ldi + j], a0);
      T acc = a0 + a1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) Li[i * ldi + j] = -acc * rdiag[i];
    }
    __syncthreads();
  }
}

// In-place LDL' factorization of the symmetric n x n matrix held in the lower triangle of M
// (row stride ldm), with the unit lower factor L replaced by L^-1 column by column as the
// elimination proceeds (Gauss-Jordan style: at step k every row i > k is reduced by
// l_ik = W_ik / d_k, which updates its trailing part W_ij (j > k) with the pivot column and
// its leading part (L^-1)_ic (c < k) with row k of L^-1).  On return M[i][c] (c < i) holds
// (L^-1)_ic and dd[k] the pivot d_k.  One barrier per column: the pivot column is passed on
// through the double buffer cb (2 n entries) by the rows that finish it.  A pivot d_k <= tol
// at k < ndrop, or an exactly zero pivot anywhere when zdrop is set (a zeroed column), drops
// column k (it lies in the span of the columns before it, to working accuracy): dd[k] = 0,
// column k of L^-1 below the diagonal is zero and the column takes no part in eliminating
// the rows below.  Returns the first other k with d_k <= tol (rows and pivots before it are
// final), else -1.
template <typename T>
__device__ int blk_ldl_inv(int n, T* M, int ldm, T* dd, T* cb, T tol, int ndrop = 0,
                           bool zdrop = false) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int i = tid; i < n; i += nt) cb[i] = M[(long long)i * ldm];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const T* cur = cb + (k & 1) * n;
    T* nxt = cb + ((k + 1) & 1) * n;
    const T dk = cur[k];
    if (!(dk > tol)) {  // every thread read the same value
      if (k >= ndrop && !(zdrop && dk == (T)0)) return k;
      if (tid == 0) dd[k] = 0;
      for (int i = k + 1 + tid; i < n; i += nt) {
        M[(long long)i * ldm + k] = 0;
        nxt[i] = M[(long long)i * ldm + k + 1];
      }
      __syncthreads();
      continue;
    }
    if (tid == 0) dd[k] = dk;
    const T invd = (T)1 / dk;
    const T* rowk = M + (long long)k * ldm;
    for (int i = k + 1 + warp; i < n; i += nw) {
      T* mi = M + (long long)i * ldm;
      const T l = cur[i] * invd;
      for (int c = lane; c <= i; c += 32) {
        // c < k: row k of L^-1; c == k: the new entry -l; c > k: the pivot column
        const T y = (c < k ? rowk : cur)[c];
        const T v = (c == k) ? -l : fma(-l, y, mi[c]);
        mi[c] = v;
        if (c == k + 1) nxt[i] = v;
      }
    }
    __syncthreads();
  }
  return -1;
}


// Register form of blk_ldl_inv run by the first NW warps of the block (named barrier 1): the
// same elimination, pivots and drops (L^-1 left in the strictly lower part of M, the pivots in
// dd, the first failing column returned, else -1), with the lower triangle of the n x n
// matrix held in registers: half-warp g (0 .. 2 NW - 1) owns rows g + 2 NW r (r < RS), lane
// cl = lane % 16 owns columns cl + 16 c (c < CS); n <= min(2 NW RS, 16 CS).  Few warps with many
// entries each keep the per-column overhead (pivot, reciprocal, buffer hand-over) small next
// to the one FMA per owned entry.  Step k reads a shared buffer (2 x 16 CS floats, double-
// buffered by the parity of k) that holds row k of L^-1 in its entries c < k and the current
// pivot column in its entries i >= k; the owners of column k + 1 and row k + 1 write the next
// one right after their update, so one barrier per column suffices.  Entries above the
// diagonal and past n take updates that are never read.  Only threads < 32 NW may call it.
template <int NW, int RS, int CS>
__device__ int ldl_inv_reg(int n, float* M, int ldm, float* dd, float* buf, float tol,
                           int ndrop, bool zdrop) {
  using T = float;
  constexpr int NHW = 2 * NW;
  constexpr int NTH = 32 * NW;
  constexpr int BL = 16 * CS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = 2 * warp + (lane >> 4), cl = lane & 15;
  auto sync = [] { asm volatile("bar.sync 1, %0;" ::"r"(NTH) : "memory"); };
  T R[RS][CS];
#pragma unroll
  for (int r = 0; r < RS; ++r)
#pragma unroll
    for (int c = 0; c < CS; ++c) {
      const int i = g + NHW * r, j = cl + 16 * c;
      R[r][c] = (i < n && j <= i) ? M[(long long)i * ldm + j] : (T)0;
    }
  for (int i = tid; i < 2 * BL; i += NTH) buf[i] = (T)0;
  sync();
  if (cl == 0) {
#pragma unroll
    for (int r = 0; r < RS; ++r)
      if (g + NHW * r < BL) buf[g + NHW * r] = R[r][0];
  }
  sync();
  int fc = -1;
  bool stop = false;
#pragma unroll
  for (int q = 0; q < CS; ++q) {
    if (stop) break;
    const int r0 = (16 * q) / NHW;  // slots below hold rows < 16 q only
    for (int kw = 0; kw < 16; ++kw) {
      const int k = 16 * q + kw;
      if (k >= n) {
        stop = true;
        break;
      }
      const T* __restrict__ cur = buf + (k & 1) * BL;
      T* __restrict__ nxt = buf + ((k + 1) & 1) * BL;
      const T dk = cur[k];
      const bool drop = !(dk > tol);
      if (drop && k >= ndrop && !(zdrop && dk == (T)0)) {  // uniform: every thread read dk
        fc = k;
        stop = true;
        break;
      }
      if (tid == 0) dd[k] = drop ? (T)0 : dk;
      const T invd = drop ? (T)0 : __frcp_rn(dk);
      T l[RS];
#pragma unroll
      for (int r = r0; r < RS; ++r) {
        const T wik = __shfl_sync(0xffffffffu, R[r][q], (lane & 16) | kw);
        l[r] = g + NHW * r > k ? wik * invd : (T)0;
      }
      // R -= l y' on the owned entries, two columns per packed FMA (each half rounds as fmaf)
      static_assert(CS % 2 == 0, "column slots come in pairs");
#pragma unroll
      for (int c = 0; c < CS; c += 2) {
        const float2 y2 = make_float2(cur[cl + 16 * c], cur[cl + 16 * (c + 1)]);
#pragma unroll
        for (int r = r0; r < RS; ++r) {
          const float2 a = __ffma2_rn(make_float2(-l[r], -l[r]), y2, make_float2(R[r][c], R[r][c + 1]));
          R[r][c] = a.x;
          R[r][c + 1] = a.y;
        }
      }
      if (cl == kw) {
#pragma unroll
        for (int r = r0; r < RS; ++r)
          if (g + NHW * r > k) R[r][q] = -l[r];
      }
      const int k1 = k + 1;
      if (cl == (k1 & 15)) {
#pragma unroll
        for (int r = r0; r < RS; ++r) {
          const int i = g + NHW * r;
          if (i >= k1 && i < BL) nxt[i] = kw < 15 ? R[r][q] : R[r][q + 1 < CS ? q + 1 : q];
        }
      }
      if (g == k1 % NHW) {
        // row k + 1 = 16 q + kw + 1 lies in slot (16 q + kw + 1) / NHW: at most 16 / NHW slots
        // past r0 = 16 q / NHW, so only those are tested
        const int rk = k1 / NHW;
#pragma unroll
        for (int r = r0; r < RS && r <= r0 + 16 / NHW; ++r)
          if (r == rk) {
#pragma unroll
            for (int c = 0; c < CS; ++c)
              if (cl + 16 * c < k1) nxt[cl + 16 * c] = R[r][c];
          }
      }
      sync();
    }
  }
#pragma unroll
  for (int r = 0; r < RS; ++r)
#pragma unroll
    for (int c = 0; c < CS; ++c) {
      const int i = g + NHW * r, j = cl + 16 * c;
      if (i < n && j <= i) M[(long long)i * ldm + j] = R[r][c];
    }
  sync();
  return fc;
}

// Cholesky-QR transform in the arithmetic of T: from the FP64 Gram G (accumulated in FP64
// across CTAs), scale s = diag(G)^-1/2 in FP64, factor s G s = L D L' in T (with L^-1 formed
// alongside), and write Tm = diag(s) L^-T D^-1/2 (ka x ka upper triangular) so that V Tm has
// orthonormal columns.  A zero column has a zero pivot, and so has a column whose norm is at
// or below its floor (rfloor for columns < keep, pfloor for the rest): it is zeroed.  With ndrop > 0, a pivot <= pivot_tol in the leading ndrop
// columns, and a zero pivot anywhere, drops that column (its column of Tm is zero; the count
// goes to *ndropped).  Any other pivot <= pivot_tol: ST_CHOL_FAIL in *status and the failing
// column in *fail_col, unless the failure lies in the trailing columns >= keep (the
// direction block), in which case the leading keep columns are returned, the rest zeroed,
// and *pflag cleared.
// SM = the matrix lives in shared memory.
template <typename T, bool SM>
__device__ __forceinline__ void k_chol_inv_body(int ka, const double* __restrict__ G, int ldg,
                                                T* __restrict__ Tm, T* Wg, int* status,
                                                int* fail_col, double pivot_tol, int keep,
                                                int* pflag, int ndrop, int* ndropped,
                                                double rfloor, double pfloor) {
  extern __shared__ __align__(16) unsigned char craw[];
  T* s = (T*)craw;    // ka scale factors
  T* dd = s + ka;     // ka pivots
  T* cb = dd + ka;    // 2 ka pivot-column buffer
  T* W = SM ? cb + 2 * ka : Wg;  // ka x ka
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < ka; i += nt) {
    double dgi = G[(long long)i * ldg + i];
    const double fl = i < keep ? rfloor * rfloor : pfloor * pfloor;
    s[i] = dgi > fl ? (T)rsqrt(dgi) : (T)0;
  }
  __syncthreads();
  for (int idx = tid; idx < ka * ka; idx += nt) {
    int i = idx / ka, j = idx % ka;
    if (j > i) continue;
    double g = 0.5 * (G[(long long)i * ldg + j] + G[(long long)j * ldg + i]);
    W[i * ka + j] = (T)g * s[i] * s[j];
  }
  __syncthreads();
  const int fc = blk_ldl_inv<T>(ka, W, ka, dd, cb, (T)pivot_tol, ndrop, ndrop > 0);
  __syncthreads();
  if (ndropped && tid == 0) {
    const int lim = fc >= 0 ? fc : ka;
    int cnt = 0;
    for (int k = 0; k < lim; ++k) cnt += dd[k] == (T)0;
    if (cnt) atomicAdd(ndropped, cnt);
  }
  int kk = ka;  // size of the leading block whose transform is returned
  if (fc >= 0) {
    if (pflag && keep > 0 && fc >= keep) {
      kk = keep;
      if (tid == 0) *pflag = 0;
    } else {
      if (tid == 0) {
        atomicOr(status, ST_CHOL_FAIL);
        if (fail_col) *fail_col = fc;
      }
      return;
    }
  }
  for (int i = tid; i < kk; i += nt) cb[i] = dd[i] > (T)0 ? rsqrt(dd[i]) : (T)0;
  __syncthreads();
  // Tm[r][c] = s_r (L^-1)_cr d_c^-1/2 for r <= c < kk
  for (int idx = tid; idx < ka * ka; idx += nt) {
    int r = idx / ka, c = idx % ka;
    T v = 0;
    if (r <= c && c < kk) v = s[r] * (r == c ? (T)1 : W[c * ka + r]) * cb[c];
    Tm[(long long)r * ka + c] = v;
  }
}

template <typename T, bool SM>
__global__ void __launch_bounds__(1024)
    k_chol_inv(int ka, const double* __restrict__ G, int ldg, T* __restrict__ Tm, T* Wg,
               int* status, int* fail_col, double pivot_tol, int keep, int* pflag, int ndrop,
               int* ndropped, double rfloor, double pfloor) {
  k_chol_inv_body<T, SM>(ka, G, ldg, Tm, Wg, status, fail_col, pivot_tol, keep, pflag, ndrop,
                         ndropped, rfloor, pfloor);
}
// One CTA per descriptor of a lockstep batch (FP32).
template <bool SM>
__global__ void __launch_bounds__(1024) k_chol_inv_b(const CholDesc* __restrict__ tab) {
  const CholDesc a = tab[blockIdx.x];
  k_chol_inv_body<float, SM>(a.ka, a.G, a.ldg, a.Tm, a.Wg, a.status, a.fail_col, a.pivot_tol,
                             a.keep, a.pflag, a.ndrop, a.ndropped, a.rfloor, a.pfloor);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rayleigh-Ritz input guard: basis columns i >= K whose FP64 Gram diagonal is exactly zero
// were dropped by the Cholesky-QR (their columns of S and LS are zero, so is their row of G).
// Their diagonal is lifted above the Gershgorin bound (the largest of the nw per-warp row-sum
// maxima in red), which puts their spurious eigenvalues above every genuine Ritz value.
template <typename T>
__device__ void lift_dropped(int m, int K, const double* __restrict__ G, int ldg, T* A,
                             int lda, const T* red, int nw) {
  T big = 0;
  for (int w = 0; w < nw; ++w) big = fmax(big, red[w]);
  big = big * (T)1.25 + (T)1;
  for (int i = K + (int)threadIdx.x; i < m; i += blockDim.x)
    if (G[(long long)i * ldg + i] == 0.0) A[(long long)i * lda + i] = big;
}

// ---------------------------------------------------------------------------------------
__device__ inline float sdiv(float a, float b) { return __fdividef(a, b); }
// 1 / b in FP64 from the hardware's reciprocal estimate (rcp.approx.ftz.f64) refined by two
// steps of Newton's iteration for the reciprocal, r <- r + r (1 - b r), each of which about
// doubles the correct bits: a few FP64 FMAs instead of an IEEE division, which matters at
// GB300's FP64 rate.  Not correctly rounded (within a few ulps); b must be normal.
__device__ __forceinline__ double rcp_newton(double b) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
  r = fma(r, fma(-b, r, 1.0), r);
  r = fma(r, fma(-b, r, 1.0), r);
  return r;
}

// FP64 a / b as a * (1 / b) by rcp_newton where b is a normal number (a few ulps; inverse
// iteration and Sturm counts need no correctly rounded quotient), else an IEEE division.
__device__ inline double sdiv(double a, double b) {
  const double ab = fabs(b);
  return (ab >= 2.2250738585072014e-308 && ab <= 1e300) ? a * rcp_newton(b) : a / b;
}

template <typename T>
__device__ int sturm_count(int m, const T* __restrict__ d, const T* __restrict__ e2, T x,
                           T pivmin) {
  int c = 0;
  T q = d[0] - x;
  if (fabs(q) <= pivmin) q = -pivmin;
  if (q <= 0) ++c;
#pragma unroll 4
  for (int i = 1; i < m; ++i) {
    // |q| > pivmin >= the smallest normal number: FP64 takes the Newton reciprocal unguarded
    if constexpr (sizeof(T) == 8) q = d[i] - x - e2[i - 1] * rcp_newton(q);
    else q = d[i] - x - sdiv(e2[i - 1], q);
    if (fabs(q) <= pivmin) q = -pivmin;
    if (q <= 0) ++c;
  }
  return c;
}

// Pseudo-random start entries in (-1, 1) for inverse iteration (SplitMix64 output mix).
__device__ inline float start_entry(int i, int j) {
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i * 7919 + j * 104729 + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * (2.0f / 16777216.0f) - 1.0f;
}

#ifdef SC_RR_PHASES
__device__ long long g_rr_phase[8];
__device__ long long g_rr_sub[4];
__device__ long long g_rr_inv[4];
#define RR_INV(i, t0)                                                  \
  do {                                                                 \
    __syncthreads();                                                   \
    if (threadIdx.x == 0) {                                            \
      long long t1 = clock64();                                        \
      g_rr_inv[i] += t1 - t0;                                          \
      t0 = t1;                                                         \
    }                                                                  \
  } while (0)
#define RR_SUB(i, t0)                                                  \
  do {                                                                 \
    if (threadIdx.x == 0) {                                            \
      long long t1 = clock64();                                        \
      g_rr_sub[i] += t1 - t0;                                          \
      t0 = t1;                                                         \
    }                                                                  \
  } while (0)
#else
#define RR_INV(i, t0) \
  do {                \
  } while (0)
#define RR_SUB(i, t0) \
  do {                \
  } while (0)
#endif
#ifdef SC_RR_PHASES
#define RR_MARK(i)                                   \
  do {                                               \
    __syncthreads();                                 \
    if (threadIdx.x == 0) g_rr_phase[i] = clock64(); \
  } while (0)
#else
#define RR_MARK(i) \
  do {             \
  } while (0)
#endif

constexpr int RR_NT = 1024;
#ifndef RR_SWEEPS
#define RR_SWEEPS 2  // inverse-iteration sweeps of the Rayleigh-Ritz eigenvector phase (FP64)
#endif
#ifndef RR_SWEEPS_F32
#define RR_SWEEPS_F32 2  // the same in FP32
#endif

// Rayleigh-Ritz in an orthonormal trial basis: the K smallest eigenpairs of the symmetric
// m x m matrix G (FP64 in, arithmetic in T), one CTA of 1024 threads.
//  1. Householder tridiagonalization (Golub & Van Loan Alg. 8.3.1), three barriers per step:
//     warp 0 forms the reflector; p = beta A' v with 8 lanes per row and four accumulators,
//     per-warp partial sums of p'v (summed in fixed order); the rank-2 update.
//  2. The K smallest eigenvalues of T by 17-point multisection on Sturm counts (16 lanes
//     per eigenvalue, up to 64 eigenvalues at once).
//  3. Eigenvectors of T by inverse iteration (tridiagonal LU with partial pivoting, shifts
//     kept 10 eps ||T|| apart), two sweeps, each followed by a block Cholesky-QR (a second
//     pass when the block was far from orthonormal; in-order Gram-Schmidt if it breaks).
//  4. Back-transformation with the stored reflectors.
template <typename T, bool SM>
__global__ void __launch_bounds__(RR_NT)
    k_rr_eig(int m_full, int K, const double* __restrict__ G, int ldg,
             double* __restrict__ theta, T* __restrict__ Y, T* Ag, T* Zg, T* lu, T* Gsg,
             int* status, int* pflag, int mP, int* nfallback) {
  // a dropped direction block P (trailing mP columns of the basis) shrinks the problem
  const int m = (pflag && *pflag == 0) ? m_full - mP : m_full;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* d = (T*)smraw;
  T* e = d + m;
  T* beta = e + m;
  T* vv = beta + m;
  T* pv = vv + m;
  T* wv = pv + m;
  T* lam = wv + m;   // K
  T* red = lam + K;  // 128
  T* nxt = red + 128;
  T* A = SM ? nxt : Ag;                        // m_full x m_full (row stride m)
  T* Z = SM ? nxt + (long long)m * m : Zg;     // m x K
  __shared__ int sflag;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nw = nt / 32;

  {
    T gmax = 0;  // Gershgorin bound of A: the largest row sum of |a_ij|
    for (int i = warp; i < m; i += nw) {
      T rs = 0;
      for (int j = lane; j < m; j += 32) {
        const T a = (T)(0.5 * (G[(long long)i * ldg + j] + G[(long long)j * ldg + i]));
        A[(long long)i * m + j] = a;
        rs += fabs(a);
      }
      gmax = fmax(gmax, warp_sum(rs));
    }
    if (lane == 0) red[warp] = gmax;
    __syncthreads();
    lift_dropped<T>(m, K, G, ldg, A, m, red, nw);
    __syncthreads();
  }
  RR_MARK(0);
  // ---- 1. tridiagonalization
  long long tsub = clock64();
  for (int k = 0; k + 2 < m; ++k) {
    const int n1 = m - k - 1;
    T* x = A + (long long)k * m + k + 1;
    if (warp == 0) {
      T p0 = 0, p1 = 0;
      int i = lane + 1;
      for (; i + 32 < n1; i += 64) {
        p0 = fma(x[i], x[i], p0);
        p1 = fma(x[i + 32], x[i + 32], p1);
      }
      if (i < n1) p0 = fma(x[i], x[i], p0);
      T sigma = p0 + p1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sigma += __shfl_xor_sync(0xffffffffu, sigma, o);
      T bet = 0, iv0 = 1;
      if (lane == 0) {
        T x0 = x[0], ek;
        if (sigma == (T)0) {
          bet = 0;
          ek = x0;
        } else {
          // x -> ek e1 with ek = -sign(x0) mu: v0 = x0 - ek has |v0| >= mu, so the tail of
          // v = x / v0 stays <= 1 however small sigma is (no cancellation, no overflow)
          T mu = sqrt(x0 * x0 + sigma);
          T v0 = x0 + copysign(mu, x0);
          bet = (T)2 * v0 * v0 / (sigma + v0 * v0);
          iv0 = (T)1 / v0;
          ek = -copysign(mu, x0);
        }
        beta[k] = bet;
        e[k] = ek;
      }
      bet = __shfl_sync(0xffffffffu, bet, 0);
      iv0 = __shfl_sync(0xffffffffu, iv0, 0);
      if (bet != (T)0) {
        for (int q = lane; q < n1; q += 32) {
          T vq = (q == 0) ? (T)1 : x[q] * iv0;
          vv[q] = vq;
          x[q] = vq;
        }
      }
    }
    __syncthreads();
    RR_SUB(0, tsub);
    const T bet = beta[k];
    if (bet == (T)0) continue;  // uniform
    {
      const int g = 8;
      const int rows_pp = nt / g;
      T wpart = 0;
      for (int i0 = 0; i0 < n1; i0 += rows_pp) {
        const int i = i0 + tid / g, sl = tid % g;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        if (i < n1) {
          const T* row = A + (long long)(k + 1 + i) * m + (k + 1);
          int j = sl;
          for (; j + 3 * g < n1; j += 4 * g) {
            a0 = fma(row[j], vv[j], a0);
            a1 = fma(row[j + g], vv[j + g], a1);
            a2 = fma(row[j + 2 * g], vv[j + 2 * g], a2);
            a3 = fma(row[j + 3 * g], vv[j + 3 * g], a3);
          }
          for (; j < n1; j += g) a0 = fma(row[j], vv[j], a0);
        }
        T acc = (a0 + a1) + (a2 + a3);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (i < n1 && sl == 0) {
          pv[i] = bet * acc;
          wpart = fma(bet * acc, vv[i], wpart);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) wpart += __shfl_xor_sync(0xffffffffu, wpart, o);
      if (lane == 0) red[warp] = wpart;
    }
    __syncthreads();
    RR_SUB(1, tsub);
    // p'v: the warp partials reduced by shuffles (same fixed tree in every warp)
    T pdv = lane < nw ? red[lane] : (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pdv += __shfl_xor_sync(0xffffffffu, pdv, o);
    const T kc = bet * (T)0.5 * pdv;
    // this lane's columns j = lane + 32 u of v and w stay in registers for every row
    const int nu = (n1 + 31) >> 5;  // uniform: register slots actually used this step
    T vj[8], wj[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (u >= nu) break;
      const int j = lane + 32 * u;
      vj[u] = j < n1 ? vv[j] : (T)0;
      wj[u] = j < n1 ? pv[j] - kc * vj[u] : (T)0;
    }
    for (int i = warp; i < n1; i += nw) {
      const T vi = vv[i], wi = pv[i] - kc * vi;
      T* arow = A + (long long)(k + 1 + i) * m + (k + 1);
      if (n1 <= 256) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (u >= nu) break;
          const int j = lane + 32 * u;
          if (j < n1) arow[j] -= vi * wj[u] + wi * vj[u];
        }
      } else {
        for (int j = lane; j < n1; j += 32) arow[j] -= vi * (pv[j] - kc * vv[j]) + wi * vv[j];
      }
    }
    __syncthreads();
    RR_SUB(2, tsub);
  }
  (void)tsub;
  for (int i = tid; i < m; i += nt) d[i] = A[(long long)i * m + i];
  if (tid == 0) {
    if (m >= 2) e[m - 2] = A[(long long)(m - 1) * m + (m - 2)];
    e[m - 1] = 0;
  }
  __syncthreads();
  RR_MARK(1);

  // ---- 2. Gershgorin bounds; 17-point multisection, 16 lanes per eigenvalue
  T* e2 = wv;
  {
    T lo_p = (T)3e38, hi_p = (T)-3e38, emax = 0;
    for (int i = tid; i < m; i += nt) {
      T r = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : (T)0);
      lo_p = min(lo_p, d[i] - r);
      hi_p = max(hi_p, d[i] + r);
      emax = max(emax, e[i] * e[i]);
      e2[i] = e[i] * e[i];
      if (!isfinite(d[i]) || !isfinite(e[i])) atomicOr(status, ST_NONFINITE);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo_p = min(lo_p, __shfl_xor_sync(0xffffffffu, lo_p, o));
      hi_p = max(hi_p, __shfl_xor_sync(0xffffffffu, hi_p, o));
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    if (lane == 0) {
      red[warp] = lo_p;
      red[32 + warp] = hi_p;
      red[64 + warp] = emax;
    }
    __syncthreads();
    if (tid == 0) {
      T lo = red[0], hi = red[32], em = red[64];
      for (int w = 1; w < nw; ++w) {
        lo = min(lo, red[w]);
        hi = max(hi, red[32 + w]);
        em = max(em, red[64 + w]);
      }
      red[120] = lo;
      red[121] = hi;
      red[122] = em;
    }
    __syncthreads();
  }
  const T tnorm = max(fabs(red[120]), fabs(red[121]));
  const T pivmin = Lim<T>::tiny() * max((T)1, red[122]);
  const T glo = red[120] - (T)2 * Lim<T>::eps() * tnorm - pivmin;
  const T ghi = red[121] + (T)2 * Lim<T>::eps() * tnorm + pivmin;
  {
    const int grp = tid >> 4, sl = tid & 15;
    const unsigned gmask = 0xFFFFu << (lane & 16);
    for (int j = grp; j < K; j += nt >> 4) {
      T a = glo, b = ghi;
      for (int it = 0; it < 48; ++it) {
        T tol = (T)2 * Lim<T>::eps() * max(fabs(a), fabs(b)) + (T)4 * pivmin;
        if (b - a <= tol) break;
        T h = (b - a) / (T)17;
        int c = sturm_count(m, d, e2, a + h * (T)(sl + 1), pivmin);
        unsigned bal = __ballot_sync(gmask, c > j) >> (lane & 16);
        int first = bal ? (__ffs(bal) - 1) : 16;
        T na = first == 0 ? a : a + h * (T)first;
        T nb = first == 16 ? b : a + h * (T)(first + 1);
        if (!(nb > na)) break;
        a = na;
        b = nb;
      }
      if (sl == 0) lam[j] = (T)0.5 * (a + b);
    }
  }
  __syncthreads();
  RR_MARK(2);

  // ---- 3. inverse iteration
  const T sep = (T)10 * Lim<T>::eps() * tnorm + pivmin;
  T* shift = pv;
  if (tid == 0) {
    T prev = (T)0;
    for (int j = 0; j < K; ++j) {
      T sj = lam[j];
      if (j > 0 && sj < prev + sep) sj = prev + sep;
      shift[j] = sj;
      prev = sj;
    }
  }
  __syncthreads();
  const T small_piv = Lim<T>::eps() * tnorm + pivmin;
#define LU(i, a) lu[((long long)(i) * 5 + (a)) * K + j]
  for (int j = tid; j < K; j += nt) {
    const T sj = shift[j];
    T al = d[0] - sj, bt = m > 1 ? e[0] : (T)0;
    for (int i = 0; i + 1 < m; ++i) {
      const T dl = e[i];
      const T an = d[i + 1] - sj, bn = (i + 2 < m) ? e[i + 1] : (T)0;
      if (fabs(al) >= fabs(dl)) {
        if (al == (T)0) al = small_piv;
        const T mlt = dl / al;
        LU(i, 0) = al; LU(i, 1) = bt; LU(i, 2) = 0; LU(i, 3) = mlt; LU(i, 4) = 0;
        al = an - mlt * bt;
        bt = bn;
      } else {
        const T mlt = al / dl;
        LU(i, 0) = dl; LU(i, 1) = an; LU(i, 2) = bn; LU(i, 3) = mlt; LU(i, 4) = 1;
        al = bt - mlt * an;
        bt = -mlt * bn;
      }
    }
    if (fabs(al) < small_piv) al = al < (T)0 ? -small_piv : small_piv;
    LU(m - 1, 0) = al; LU(m - 1, 1) = 0; LU(m - 1, 2) = 0; LU(m - 1, 3) = 0; LU(m - 1, 4) = 0;
  }
  for (long long idx = tid; idx < (long long)m * K; idx += nt)
    Z[idx] = (T)start_entry((int)(idx / K), (int)(idx % K));
  __syncthreads();
  RR_MARK(3);
  T* Gs = Gsg;          // K x K Gram / factor (global scratch)
  T* Li = Gsg + (size_t)K * K;
  T* rd = pv;           // K reciprocal pivots (pv is free now)
  for (int sweep = 0; sweep < 2; ++sweep) {
    for (int j = tid; j < K; j += nt) {
      for (int i = 0; i + 1 < m; ++i) {
        T bi = Z[(long long)i * K + j], bn = Z[(long long)(i + 1) * K + j];
        if (LU(i, 4) != (T)0) {
          T t = bi; bi = bn; bn = t;
        }
        Z[(long long)i * K + j] = bi;
        Z[(long long)(i + 1) * K + j] = bn - LU(i, 3) * bi;
      }
      T z1 = 0, z2 = 0, mx = 0;
      for (int i = m - 1; i >= 0; --i) {
        T zi = (Z[(long long)i * K + j] - LU(i, 1) * z1 - LU(i, 2) * z2) / LU(i, 0);
        Z[(long long)i * K + j] = zi;
        z2 = z1;
        z1 = zi;
        mx = max(mx, fabs(zi));
      }
      T inv = mx > (T)0 ? (T)1 / mx : (T)1;
      for (int i = 0; i < m; ++i) Z[(long long)i * K + j] *= inv;
    }
    __syncthreads();
    bool ok = true;
    for (int pass = 0; pass < 2 && ok; ++pass) {
      // Gram Z'Z (lower triangle), one thread per entry, four accumulators
      for (int p = tid; p < K * K; p += nt) {
        int a = p / K, b = p % K;
        if (b > a) continue;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int r = 0;
        for (; r + 3 < m; r += 4) {
          a0 = fma(Z[(long long)r * K + a], Z[(long long)r * K + b], a0);
          a1 = fma(Z[(long long)(r + 1) * K + a], Z[(long long)(r + 1) * K + b], a1);
          a2 = fma(Z[(long long)(r + 2) * K + a], Z[(long long)(r + 2) * K + b], a2);
          a3 = fma(Z[(long long)(r + 3) * K + a], Z[(long long)(r + 3) * K + b], a3);
        }
        for (; r < m; ++r) a0 = fma(Z[(long long)r * K + a], Z[(long long)r * K + b], a0);
        Gs[a * K + b] = (a0 + a1) + (a2 + a3);
      }
      __syncthreads();
      // scale to unit diagonal, factor, invert
      for (int a = tid; a < K; a += nt) wv[a] = rsqrt(max(Gs[a * K + a], Lim<T>::tiny()));
      __syncthreads();
      T mindiag = (T)1;
      for (int p = tid; p < K * K; p += nt) {
        int a = p / K, b = p % K;
        if (b <= a) Gs[a * K + b] *= wv[a] * wv[b];
      }
      __syncthreads();
      int fc = blk_chol<T>(K, Gs, K, rd, (T)(sizeof(T) == 4 ? 1e-6 : 1e-14), &sflag);
      if (fc >= 0) {
        ok = false;
        break;
      }
      // minimum pivot decides whether a second pass is needed
      if (tid == 0) {
        for (int a = 0; a < K; ++a) mindiag = min(mindiag, Gs[a * K + a] * Gs[a * K + a]);
        red[44] = mindiag;
      }
      blk_tri_inv<T>(K, Gs, K, rd, Li, K);
      // Z <- Z diag(wv) Li' : out_b = sum_{a <= b} z_a wv_a Li[b][a]; a warp per row, lanes
      // own output columns (buffered in registers until the whole row has been read)
      for (int r = warp; r < m; r += nw) {
        T* zr = Z + (long long)r * K;
        T out[16];
        const int nq = (K + 31) >> 5;  // uniform
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (q >= nq) break;
          const int b = lane + 32 * q;
          T acc = 0;
          if (b < K) {
            const T* lb = Li + b * K;
            for (int a = 0; a <= b; ++a) acc = fma(zr[a] * wv[a], lb[a], acc);
          }
          out[q] = acc;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (q >= nq) break;
          const int b = lane + 32 * q;
          if (b < K) zr[b] = out[q];
        }
        __syncwarp();
      }
      __syncthreads();
      if (red[44] > (T)0.5) break;  // nearly orthonormal input: one pass was enough
    }
    if (!ok) {
      // in-order modified Gram-Schmidt (tight clusters)
      T* coef = vv;
      for (int j = 0; j < K; ++j) {
        for (int pass = 0; pass < 2; ++pass) {
          for (int q = warp; q < j; q += nw) {
            T acc = 0;
            for (int i = lane; i < m; i += 32) acc += Z[(long long)i * K + q] * Z[(long long)i * K + j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) coef[q] = acc;
          }
          __syncthreads();
          for (int i = tid; i < m; i += nt) {
            T acc = 0;
            for (int q = 0; q < j; ++q) acc += coef[q] * Z[(long long)i * K + q];
            Z[(long long)i * K + j] -= acc;
          }
          __syncthreads();
        }
        if (warp == 0) {
          T part = 0;
          for (int i = lane; i < m; i += 32) part += Z[(long long)i * K + j] * Z[(long long)i * K + j];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
          if (lane == 0) red[41] = part > (T)0 ? (T)1 / sqrt(part) : (T)0;
        }
        __syncthreads();
        for (int i = tid; i < m; i += nt) Z[(long long)i * K + j] *= red[41];
        __syncthreads();
      }
    }
  }
#undef LU
  RR_MARK(4);

  // ---- 4. back-transformation Z <- H_0 ... H_{m-3} Z (warp-per-column dots, then update)
  T* coef = vv;
  for (int k = m - 3; k >= 0; --k) {
    const T bet = beta[k];
    if (bet == (T)0) continue;
    const int n1 = m - k - 1;
    const T* v = A + (long long)k * m + k + 1;
    for (int j = warp; j < K; j += nw) {
      T a0 = 0, a1 = 0;
      int i = lane;
      for (; i + 32 < n1; i += 64) {
        a0 = fma(v[i], Z[(long long)(k + 1 + i) * K + j], a0);
        a1 = fma(v[i + 32], Z[(long long)(k + 33 + i) * K + j], a1);
      }
      if (i < n1) a0 = fma(v[i], Z[(long long)(k + 1 + i) * K + j], a0);
      T acc = a0 + a1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) coef[j] = bet * acc;
    }
    __syncthreads();
    for (int i = warp; i < n1; i += nw) {
      const T vi = v[i];
      T* zr = Z + (long long)(k + 1 + i) * K;
#pragma unroll 2
      for (int j = lane; j < K; j += 32) zr[j] -= coef[j] * vi;
    }
    __syncthreads();
  }
  RR_MARK(5);
  for (int j = tid; j < K; j += nt) theta[j] = (double)lam[j];
  for (long long idx = tid; idx < (long long)m_full * K; idx += nt)
    Y[idx] = idx < (long long)m * K ? Z[idx] : (T)0;
  if (pflag && tid == 0) {
    if (*pflag == 0 && nfallback) *nfallback += 1;
    *pflag = 1;  // re-armed for the next pass
  }
  RR_MARK(6);
}


// The K smallest eigenvalues of the tridiagonal (d, e2 = e^2) inside [glo, ghi] by
// (LG + 1)-point multisection on Sturm counts, LG lanes per eigenvalue, to the tolerance
// max(2 eps max(|a|, |b|), abstol) + 4 pivmin.
template <typename T, int NT, int LG>
__device__ void rr_multisect(int m, int K, const T* __restrict__ d, const T* __restrict__ e2,
                             T glo, T ghi, T abstol, T pivmin, T* __restrict__ lam) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int grp = tid / LG, sl = tid % LG;
  const unsigned gmask = (LG == 32 ? 0xffffffffu : ((1u << LG) - 1u)) << (lane & (32 - LG));
  for (int j = grp; j < K; j += NT / LG) {
    T a = glo, b = ghi;
    for (int it = 0; it < 64; ++it) {
      T tol = max((T)2 * Lim<T>::eps() * max(fabs(a), fabs(b)), abstol) + (T)4 * pivmin;
      if (b - a <= tol) break;
      T h = (b - a) / (T)(LG + 1);
      int c = sturm_count(m, d, e2, a + h * (T)(sl + 1), pivmin);
      unsigned bal = __ballot_sync(gmask, c > j) >> (lane & (32 - LG));
      int first = bal ? (__ffs(bal) - 1) : LG;
      T na = first == 0 ? a : a + h * (T)first;
      T nb = first == LG ? b : a + h * (T)(first + 1);
      if (!(nb > na)) break;
      a = na;
      b = nb;
    }
    if (sl == 0) lam[j] = (T)0.5 * (a + b);
  }
}

// ---- phases 2 and 3 of the register-slot Rayleigh-Ritz kernels (shared) ------------------
// Phase 2: Gershgorin bounds of the tridiagonal T = (d, e); the K smallest eigenvalues of T by
// multisection on Sturm counts (rr_multisect), into lam[K].  Outputs the
// norm bound tnorm and the pivot floor pivmin that phase 3 uses.  NT threads take part; red
// holds 3 NW per-warp slots followed by the scalar slots RS ...
template <typename T, int NT>
__device__ void rr_phase_eigvals(int m, int K, const T* __restrict__ d, const T* __restrict__ e,
                                 T* __restrict__ e2, T* red, T* __restrict__ lam, int* status,
                                 T& tnorm, T& pivmin, const T* __restrict__ lam_ext = nullptr) {
  constexpr int NW = NT / 32;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int RS = 3 * NW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  (void)FULL;
  // ---- 2. Gershgorin bounds; multisection
  {
    T lo_p = (T)3e38, hi_p = (T)-3e38, emax = 0;
    for (int i = tid; i < m; i += NT) {
      T r = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : (T)0);
      lo_p = min(lo_p, d[i] - r);
      hi_p = max(hi_p, d[i] + r);
      emax = max(emax, e[i] * e[i]);
      e2[i] = e[i] * e[i];
      if (!isfinite(d[i]) || !isfinite(e[i])) atomicOr(status, ST_NONFINITE);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo_p = min(lo_p, __shfl_xor_sync(FULL, lo_p, o));
      hi_p = max(hi_p, __shfl_xor_sync(FULL, hi_p, o));
      emax = max(emax, __shfl_xor_sync(FULL, emax, o));
    }
    if (lane == 0) {
      red[warp] = lo_p;
      red[NW + warp] = hi_p;
      red[2 * NW + warp] = emax;
    }
    __syncthreads();
    if (tid == 0) {
      T lo = red[0], hi = red[NW], em = red[2 * NW];
      for (int q = 1; q < NW; ++q) {
        lo = min(lo, red[q]);
        hi = max(hi, red[NW + q]);
        em = max(em, red[2 * NW + q]);
      }
      red[RS] = lo;
      red[RS + 1] = hi;
      red[RS + 2] = em;
    }
    __syncthreads();
  }
  tnorm = max(fabs(red[RS]), fabs(red[RS + 1]));
  pivmin = Lim<T>::tiny() * max((T)1, red[RS + 2]);
  const T glo = red[RS] - (T)2 * Lim<T>::eps() * tnorm - pivmin;
  const T ghi = red[RS + 1] + (T)2 * Lim<T>::eps() * tnorm + pivmin;
  const T abstol = Lim<T>::eps() * tnorm;
  if (lam_ext) {  // the eigenvalues were found by k_rr_eigvals_cta: the bounds only
    for (int j = tid; j < K; j += NT) lam[j] = lam_ext[j];
    __syncthreads();
    return;
  }
  // 16 lanes per eigenvalue when the block has a group for each; otherwise 8, so that all K
  // eigenvalues are found in one round
  if (K <= NT / 16)
    rr_multisect<T, NT, 16>(m, K, d, e2, glo, ghi, abstol, pivmin, lam);
  else
    rr_multisect<T, NT, 8>(m, K, d, e2, glo, ghi, abstol, pivmin, lam);
  __syncthreads();
}

// Phase 3: eigenvectors of T for the eigenvalues lam[K] by inverse iteration into Z (m x K):
// LU with partial pivoting of T - sigma I fused with the forward elimination, back
// substitution, RR_SWEEPS sweeps, each followed by a block Cholesky-QR (in-order Gram-Schmidt
// when a tight cluster breaks it).  U (3 m K), Gs (K x K), shift/dd/wv/coef (K), cbuf (2 K)
// are scratch.
template <typename T, int NT>
__device__ void rr_phase_eigvecs(int m, int K, const T* __restrict__ d, const T* __restrict__ e,
                                 const T* __restrict__ lam, T* __restrict__ shift, T* Z, T* U,
                                 T* Gs, T* dd, T* cbuf, T* wv, T* coef, T* red, T tnorm,
                                 T pivmin) {
  constexpr int NW = NT / 32;
  constexpr int RS = 3 * NW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // ---- 3. inverse iteration
  const T sep = (T)10 * Lim<T>::eps() * tnorm + pivmin;
  if (tid == 0) {
    T prev = (T)0;
    for (int j = 0; j < K; ++j) {
      T sj = lam[j];
      if (j > 0 && sj < prev + sep) sj = prev + sep;
      shift[j] = sj;
      prev = sj;
    }
  }
  for (int idx = tid; idx < m * K; idx += NT) Z[idx] = (T)start_entry(idx / K, idx % K);
  __syncthreads();
  RR_MARK(3);
  const T small_piv = Lim<T>::eps() * tnorm + pivmin;
#define UF(i, a) U[((i) * 3 + (a)) * K + j]
  long long tinv = clock64();
  constexpr int kSweeps = sizeof(T) == 4 ? RR_SWEEPS_F32 : RR_SWEEPS;
  for (int sweep = 0; sweep < kSweeps; ++sweep) {
    for (int j = tid; j < K; j += NT) {
      // LU with partial pivoting of T - s I, the right-hand side eliminated alongside
      const T sj = shift[j];
      T al = d[0] - sj, bt = m > 1 ? e[0] : (T)0;
      T bc = Z[j];
      for (int i = 0; i + 1 < m; ++i) {
        const T dl = e[i];
        const T an = d[i + 1] - sj, bn = (i + 2 < m) ? e[i + 1] : (T)0;
        const T bx = Z[(i + 1) * K + j];
        // partial pivoting between rows i and i + 1, written without branches (the choice
        // differs between the lanes of a warp)
        const bool keep = fabs(al) >= fabs(dl);
        if (keep && al == (T)0) al = small_piv;
        const T piv = keep ? al : dl;
        const T mlt = sdiv(keep ? dl : al, piv);
        UF(i, 0) = piv;
        UF(i, 1) = keep ? bt : an;
        UF(i, 2) = keep ? (T)0 : bn;
        Z[i * K + j] = keep ? bc : bx;
        const T bnew = keep ? bx - mlt * bc : bc - mlt * bx;
        const T anew = keep ? an - mlt * bt : bt - mlt * an;
        const T btn = keep ? bn : -mlt * bn;
        bc = bnew;
        al = anew;
        bt = btn;
      }
      if (fabs(al) < small_piv) al = al < (T)0 ? -small_piv : small_piv;
      UF(m - 1, 0) = al;
      UF(m - 1, 1) = 0;
      UF(m - 1, 2) = 0;
      Z[(m - 1) * K + j] = bc;
      T z1 = 0, z2 = 0, mx = 0;
      for (int i = m - 1; i >= 0; --i) {
        const T zi = sdiv(Z[i * K + j] - UF(i, 1) * z1 - UF(i, 2) * z2, UF(i, 0));
        Z[i * K + j] = zi;
        z2 = z1;
        z1 = zi;
        mx = max(mx, fabs(zi));
      }
      const T inv = mx > (T)0 ? (T)1 / mx : (T)1;
      for (int i = 0; i < m; ++i) Z[i * K + j] *= inv;
    }
    __syncthreads();
    RR_INV(0, tinv);
    bool ok = true;
    for (int pass = 0; pass < 2 && ok; ++pass) {
      // Gram Z'Z (lower triangle), one thread per entry, four accumulators
      for (int p = tid; p < K * K; p += NT) {
        const int a = p / K, b = p % K;
        if (b > a) continue;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        int r = 0;
        for (; r + 3 < m; r += 4) {
          a0 = fma(Z[r * K + a], Z[r * K + b], a0);
          a1 = fma(Z[(r + 1) * K + a], Z[(r + 1) * K + b], a1);
          a2 = fma(Z[(r + 2) * K + a], Z[(r + 2) * K + b], a2);
          a3 = fma(Z[(r + 3) * K + a], Z[(r + 3) * K + b], a3);
        }
        for (; r < m; ++r) a0 = fma(Z[r * K + a], Z[r * K + b], a0);
        Gs[a * K + b] = (a0 + a1) + (a2 + a3);
      }
      __syncthreads();
      RR_INV(1, tinv);
      for (int a = tid; a < K; a += NT) wv[a] = rsqrt(max(Gs[a * K + a], Lim<T>::tiny()));
      __syncthreads();
      for (int p = tid; p < K * K; p += NT) {
        const int a = p / K, b = p % K;
        if (b <= a) Gs[a * K + b] *= wv[a] * wv[b];
      }
      __syncthreads();
      int fc;
      if constexpr (sizeof(T) == 4) {
        // the K x K factorization by four warps in registers (the others wait)
        __shared__ int s_fc;
        __shared__ float s_ldlbuf[2 * 64];
        if (K <= 64) {
          if (warp < 4) {
            const int f = ldl_inv_reg<4, 8, 4>(K, Gs, K, dd, s_ldlbuf, 1e-6f, 0, false);
            if (tid == 0) s_fc = f;
          }
          __syncthreads();
          fc = s_fc;
        } else {
          fc = blk_ldl_inv<T>(K, Gs, K, dd, cbuf, (T)1e-6);
        }
      } else {
        fc = blk_ldl_inv<T>(K, Gs, K, dd, cbuf, (T)1e-14);
      }
      __syncthreads();
      RR_INV(2, tinv);
      if (fc >= 0) {
        ok = false;
        break;
      }
      for (int a = tid; a < K; a += NT) cbuf[a] = rsqrt(dd[a]);
      if (tid == 0) {
        T mind = (T)1;
        for (int a = 0; a < K; ++a) mind = min(mind, dd[a]);
        red[RS + 3] = mind;
      }
      // L^-1 transposed into the (unused) upper triangle: Gs[a][b] = (L^-1)_ba for a < b,
      // so lanes that own consecutive output columns b read consecutive addresses
      for (int p = tid; p < K * K; p += NT) {
        const int a = p / K, b = p % K;
        if (b > a) Gs[a * K + b] = Gs[b * K + a];
      }
      __syncthreads();
      // Z <- Z diag(wv) L^-T D^-1/2: out_b = d_b^-1/2 sum_{a <= b} z_a wv_a (L^-1)_ba; a warp
      // per row, lanes own output columns (kept in registers until the row has been read)
      for (int r = warp; r < m; r += NW) {
        T* zr = Z + r * K;
        T out[16];
        const int nq = (K + 31) >> 5;  // uniform
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (q >= nq) break;
          const int b = lane + 32 * q;
          T acc = 0;
          if (b < K) {
            for (int a = 0; a < b; ++a) acc = fma(zr[a] * wv[a], Gs[a * K + b], acc);
            acc = (acc + zr[b] * wv[b]) * cbuf[b];
          }
          out[q] = acc;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          if (q >= nq) break;
          const int b = lane + 32 * q;
          if (b < K) zr[b] = out[q];
        }
        __syncwarp();
      }
      __syncthreads();
      RR_INV(3, tinv);
      if (red[RS + 3] > (T)0.5) break;  // nearly orthonormal input: one pass was enough
    }
    if (!ok) {
      // in-order modified Gram-Schmidt (tight clusters)
      for (int j = 0; j < K; ++j) {
        for (int pass = 0; pass < 2; ++pass) {
          for (int q = warp; q < j; q += NW) {
            T acc = 0;
            for (int i = lane; i < m; i += 32) acc += Z[i * K + q] * Z[i * K + j];
            acc = warp_sum(acc);
            if (lane == 0) coef[q] = acc;
          }
          __syncthreads();
          for (int i = tid; i < m; i += NT) {
            T acc = 0;
            for (int q = 0; q < j; ++q) acc += coef[q] * Z[i * K + q];
            Z[i * K + j] -= acc;
          }
          __syncthreads();
        }
        if (warp == 0) {
          T part = 0;
          for (int i = lane; i < m; i += 32) part += Z[i * K + j] * Z[i * K + j];
          part = warp_sum(part);
          if (lane == 0) red[RS + 4] = part > (T)0 ? (T)1 / sqrt(part) : (T)0;
        }
        __syncthreads();
        for (int i = tid; i < m; i += NT) Z[i * K + j] *= red[RS + 4];
        __syncthreads();
      }
    }
  }
#undef UF
}

// ---------------------------------------------------------------------------------------
// Rayleigh-Ritz, register-slot form for m <= 32 NS: the same four steps as k_rr_eig with
// less synchronization.
//  1. Tridiagonalization with a few threads per row and two barriers per Householder step:
//     the owners of a row form its entries of p = beta A v and apply the rank-2 update to
//     them; the reflector scalars are formed by every thread from one block sum.  The
//     reflector of step k is stored in row k.
//  2. Multisection on Sturm counts as in k_rr_eig, converged to eps ||T|| (the accuracy the
//     reduction itself has).
//  3. Inverse iteration: LU with partial pivoting of T - sigma I fused with the forward
//     elimination of the right-hand side (only U is stored), back substitution; two sweeps,
//     each followed by a block Cholesky-QR through blk_ldl_inv.
//  4. Back-transformation with one warp per column pair, no barriers.
template <typename T, int NS>
__device__ __forceinline__ T slot_sel(const T (&a)[NS], int u) {
  T r = a[0];
#pragma unroll
  for (int q = 1; q < NS; ++q)
    if (q == u) r = a[q];
  return r;
}

// Threads per row in the tridiagonalization of an m x m matrix by nt threads: the largest
// of 8, 4, 2, 1 with m * tpr <= nt.
__host__ __device__ inline int rr_tpr(int m, int nt) {
  int t = 8;
  while (t > 1 && m * t > nt) t >>= 1;
  return t;
}
// Row stride of the matrix: a multiple of tpr, at least m, with an odd quotient, so that the
// tpr parts of 32 / tpr consecutive rows fall in distinct shared-memory banks.  At most
// m + 2 tpr - 1 <= m + 15.
__host__ __device__ inline int rr_lda(int m, int tpr) {
  int l = (m + tpr - 1) / tpr * tpr;
  if ((l / tpr) % 2 == 0) l += tpr;
  return l;
}
// Barrier 1 over the first n threads of the block (n a multiple of 32).
__device__ __forceinline__ void rr_named_sync(int n) {
  asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
}

template <typename T, int NS, int NW, bool SM>
__device__ __forceinline__ void k_rr_eig_reg_body(int m_full, int K, const double* __restrict__ G,
                                                  int ldg, double* __restrict__ theta,
                                                  T* __restrict__ Y, T* Ag, T* Zg, T* Ug, T* Gsg,
                                                  int* status, int* pflag, int mP,
                                                  int* nfallback, const T* dext,
                                                  const T* eext, const T* bext, int ldext,
                                                  const T* lamext, int* mext) {
  // dext != nullptr: the tridiagonal form (d, e, beta) and the reflector rows of Ag (row stride
  // ldext) were computed by the cluster kernel (k_tridiag_cl); the load and phase 1 are skipped
  constexpr int NT = NW * 32;
  constexpr unsigned FULL = 0xffffffffu;
  const int m = (pflag && *pflag == 0) ? m_full - mP : m_full;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* d = (T*)smraw;     // m
  T* e = d + m;         // m
  T* beta = e + m;      // m
  T* e2 = beta + m;     // m
  T* Pb = e2 + m;       // 2 m: p of the current step (double-buffered)
  T* lam = Pb + 2 * m;  // K
  T* shift = lam + K;   // K
  T* dd = shift + K;    // K pivots of the block Cholesky
  T* cbuf = dd + K;     // 2 K
  T* wv = cbuf + 2 * K; // K
  T* coef = wv + K;     // K
  T* red = coef + K;    // 3 NW per-warp parts, then scalar slots RS ..
  T* nxt = red + 3 * NW + 8;
  T* A = SM ? nxt : Ag;                             // m x m (row stride m)
  const bool ext = dext != nullptr;
  const int lda = ext ? ldext : rr_lda(m, rr_tpr(m, NT));  // row stride of the matrix
  T* Z = SM ? A + (size_t)m * lda : Zg;             // m x K
  T* U = SM ? Z + (size_t)m * K : Ug;               // 3 m K
  T* Gs = SM ? U + (size_t)3 * m * K : Gsg;         // K x K
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // red[3 NW + 0..4]: lo, hi, max e^2, min pivot, MGS scale (the shared phases use them)

  if (!ext) {
    T gmax = 0;  // Gershgorin bound of A: the largest row sum of |a_ij|
    for (int i = warp; i < m; i += NW) {
      T rs = 0;
      for (int j = lane; j < m; j += 32) {
        const T a = (T)(0.5 * (G[(long long)i * ldg + j] + G[(long long)j * ldg + i]));
        A[i * lda + j] = a;
        rs += fabs(a);
      }
      gmax = fmax(gmax, warp_sum(rs));
    }
    if (lane == 0) red[warp] = gmax;
    __syncthreads();
    lift_dropped<T>(m, K, G, ldg, A, lda, red, NW);
    __syncthreads();
  }
  RR_MARK(0);

  if (ext) {
    for (int i = tid; i < m; i += NT) {
      d[i] = dext[i];
      e[i] = eext[i];
      beta[i] = bext[i];
    }
  } else {
  // ---- 1. tridiagonalization (Golub & Van Loan Alg. 8.3.1), two barriers per step
  // tpr threads per row: thread t < ntri owns row i = t / tpr and, of the columns j that step
  // k touches, those with j = k + 1 + q (mod tpr), q = t % tpr.  Step k:
  //  (a) the owners of rows j > k publish x_j = a_jk (their own entry) and per-warp sums of
  //      x_j^2 over j > k + 1;
  //  (b) every thread forms the reflector scalars (mu, v0, beta, e_k) from sigma^2 and x_{k+1};
  //      v = e_{k+1} + x / v0 on j > k + 1 goes to row k for the back-transformation;
  //  (c) p_i = beta (A v)_i on the owned rows (parts over q combined by shuffles), published
  //      with per-warp sums of p_i v_i;
  //  (d) w = p - (beta / 2)(p'v) v and the rank-2 update A -= v w' + w v' of the owned
  //      entries, with v_j and w_j formed on the fly from x_j and p_j.
  // The entry a_j,k+1 that row j's owner reads in the next step's (a) is updated by that same
  // thread in (d), so no barrier separates (d) from the next (a).
  {
    const int tpr = rr_tpr(m, NT);
    const int ntri = (m * tpr + 31) / 32 * 32;
    const int nwt = ntri / 32;
    const int ri = tid / tpr, q = tid % tpr;
    const bool own = tid < ntri && ri < m;
    T* __restrict__ pvec = e2;  // p of the current step (e2 is free until step 2)
    if (tid < ntri) {
      for (int k = 0; k + 2 < m; ++k) {
        const int k1 = k + 1;
        T* __restrict__ xs = Pb + (k & 1) * m;  // x of this step (double-buffered)
        // (a)
        T xi = 0, s2 = 0;
        if (own && q == 0) {
          if (ri >= k1) {
            xi = A[ri * lda + k];
            xs[ri] = xi;
            if (ri > k1) s2 = xi * xi;
          } else if (ri == k) {
            d[k] = A[k * lda + k];
          }
        }
        s2 = warp_sum(s2);
        if (lane == 0) red[warp] = s2;
        rr_named_sync(ntri);
        // (b)
        const T sg = warp_sum(lane < nwt ? red[lane] : (T)0);
        const T x0 = xs[k1];
        T bet = 0, iv0 = 0, ek = x0;
        if (sg != (T)0) {
          // x -> ek e1 with ek = -sign(x0) mu: v0 = x0 - ek has |v0| >= mu, so the tail of
          // v = x / v0 stays <= 1 however small sigma is; beta = 2 / (1 + sigma / v0^2)
          const T mu = sqrt(x0 * x0 + sg);
          const T v0 = x0 + copysign(mu, x0);
          iv0 = (T)1 / v0;
          bet = (T)2 / ((T)1 + sg * iv0 * iv0);
          ek = -copysign(mu, x0);
        }
        if (tid == 0) {
          e[k] = ek;
          beta[k] = bet;
        }
        if (own && q == 0 && ri > k1) A[k * lda + ri] = xi * iv0;
        // (c)
        const bool act = own && ri >= k1;
        T sacc = 0;
        if (act) {
          const T* __restrict__ ra = A + ri * lda;
          T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
          int j = k1 + 1 + q;
          for (; j + 3 * tpr < m; j += 4 * tpr) {
            s0 = fma(ra[j], xs[j], s0);
            s1 = fma(ra[j + tpr], xs[j + tpr], s1);
            s2 = fma(ra[j + 2 * tpr], xs[j + 2 * tpr], s2);
            s3 = fma(ra[j + 3 * tpr], xs[j + 3 * tpr], s3);
          }
          for (; j < m; j += tpr) s0 = fma(ra[j], xs[j], s0);
          sacc = (s0 + s1) + (s2 + s3);
        }
        for (int o = 1; o < tpr; o <<= 1) sacc += __shfl_xor_sync(FULL, sacc, o);
        T pi = 0, vi = 0, pvp = 0;
        if (act) {
          pi = bet * (A[ri * lda + k1] + iv0 * sacc);
          vi = ri == k1 ? (T)1 : xs[ri] * iv0;
          if (q == 0) {
            pvec[ri] = pi;
            pvp = pi * vi;
          }
        }
        pvp = warp_sum(pvp);
        if (lane == 0) red[NW + warp] = pvp;
        rr_named_sync(ntri);
        // (d)
        const T pv = warp_sum(lane < nwt ? red[NW + lane] : (T)0);
        const T kc = bet * (T)0.5 * pv;
        if (act) {
          const T wi = pi - kc * vi;
          T* __restrict__ ra = A + ri * lda;
          int j = k1 + q;
          if (q == 0) {  // column k + 1, where v_j = 1
            ra[k1] = ra[k1] - vi * (pvec[k1] - kc) - wi;
            j += tpr;
          }
#pragma unroll 4
          for (; j < m; j += tpr) {
            const T vj = xs[j] * iv0;
            const T wj = pvec[j] - kc * vj;
            ra[j] = ra[j] - vi * wj - wi * vj;
          }
        }
      }
      rr_named_sync(ntri);
      if (tid == 0) {
        // the trailing 2 x 2 block of T (or the 1 x 1 matrix)
        if (m >= 2) {
          d[m - 2] = A[(m - 2) * lda + (m - 2)];
          e[m - 2] = A[(m - 1) * lda + (m - 2)];
          d[m - 1] = A[(m - 1) * lda + (m - 1)];
        } else {
          d[0] = A[0];
        }
        e[m - 1] = 0;
      }
    }
  }
  }
  __syncthreads();
  RR_MARK(1);

  T tnorm, pivmin;
  rr_phase_eigvals<T, NT>(m, K, d, e, e2, red, lam, status, tnorm, pivmin, lamext);
  RR_MARK(2);

  rr_phase_eigvecs<T, NT>(m, K, d, e, lam, shift, Z, U, Gs, dd, cbuf, wv, coef, red, tnorm,
                          pivmin);
  RR_MARK(4);

  // ---- 4. back-transformation Y = H_0 ... H_{m-3} Z, two columns per warp in registers
  // (with mext set it is left to k_rr_back, which spreads the columns over SMs)
  for (int j0 = 2 * warp; !mext && j0 < K; j0 += 2 * NW) {
    const int j1 = j0 + 1;
    const bool two = j1 < K;  // uniform in the warp
    T za[NS], zb[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      const int i = lane + 32 * u;
      za[u] = i < m ? Z[i * K + j0] : (T)0;
      zb[u] = (i < m && two) ? Z[i * K + j1] : (T)0;
    }
    for (int kr = m - 3; kr >= 0; --kr) {
      const T bet = beta[kr];
      if (bet == (T)0) continue;  // uniform
      const int k1 = kr + 1;
      const T* vk = A + kr * lda;
      T cv[NS];
      T sa = 0, sb = 0;
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        const int i = lane + 32 * u;
        cv[u] = (i == k1) ? (T)1 : ((i > k1 && i < m) ? vk[i] : (T)0);
        sa = fma(cv[u], za[u], sa);
        sb = fma(cv[u], zb[u], sb);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(FULL, sa, o);
        sb += __shfl_xor_sync(FULL, sb, o);
      }
      sa *= bet;
      sb *= bet;
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        za[u] = fma(-sa, cv[u], za[u]);
        zb[u] = fma(-sb, cv[u], zb[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      const int i = lane + 32 * u;
      if (i < m_full) {
        Y[(long long)i * K + j0] = i < m ? za[u] : (T)0;
        if (two) Y[(long long)i * K + j1] = i < m ? zb[u] : (T)0;
      }
    }
  }
  RR_MARK(5);
  for (int j = tid; j < K; j += NT) theta[j] = (double)lam[j];
  if (mext) {
    if (tid == 0) *mext = m;  // k_rr_back reads the solved size and re-arms *pflag
  } else if (pflag && tid == 0) {
    if (*pflag == 0 && nfallback) *nfallback += 1;
    *pflag = 1;  // re-armed for the next pass
  }
  RR_MARK(6);
}


template <typename T, int NS, int NW, bool SM>
__global__ void __launch_bounds__(NW * 32)
    k_rr_eig_reg(int m_full, int K, const double* __restrict__ G, int ldg,
                 double* __restrict__ theta, T* __restrict__ Y, T* Ag, T* Zg, T* Ug, T* Gsg,
                 int* status, int* pflag, int mP, int* nfallback, const T* dext = nullptr,
                 const T* eext = nullptr, const T* bext = nullptr, int ldext = 0,
                 const T* lamext = nullptr, int* mext = nullptr) {
  k_rr_eig_reg_body<T, NS, NW, SM>(m_full, K, G, ldg, theta, Y, Ag, Zg, Ug, Gsg, status, pflag,
                                   mP, nfallback, dext, eext, bext, ldext, lamext, mext);
}
// One CTA per descriptor of a lockstep batch (FP32).  With the matrix in global memory the
// working set is Ag (m (m + 16) floats, then Z, U, Gs); with tri set, the tridiagonal form and
// the reflector rows (stride m) come from the cluster kernel.
template <int NS, int NW, bool SM>
__global__ void __launch_bounds__(NW * 32) k_rr_eig_reg_b(const RrDesc* __restrict__ tab) {
  const RrDesc a = tab[blockIdx.x];
  float* Zg = SM ? nullptr : a.Ag + (size_t)a.m * (a.m + 16);
  float* Ug = SM ? nullptr : Zg + (size_t)a.m * a.K;
  float* Gsg = SM ? nullptr : Ug + (size_t)3 * a.m * a.K;
  k_rr_eig_reg_body<float, NS, NW, SM>(a.m, a.K, a.G, a.ldg, a.theta, a.Y, a.Ag, Zg, Ug, Gsg,
                                       a.status, a.pflag, a.mP, a.nfallback, a.tri,
                                       a.tri ? a.tri + a.m : nullptr,
                                       a.tri ? a.tri + 2 * a.m : nullptr, a.tri ? a.m : 0,
                                       a.tri ? a.lamx : nullptr, a.tri ? a.mx : nullptr);
}

// ---- the FP64 Rayleigh-Ritz spread over SMs ---------------------------------------------
// GB300 runs FP64 at 2 FMA per clock per SM, so a one-CTA FP64 solve is bound by one SM's FP64
// pipe.  For 64 < m <= 256 the phases go to many SMs: the cluster tridiagonalization
// (k_tridiag_cl<double>), the eigenvalues here (one CTA per eigenvalue), the eigenvectors in
// k_rr_eig_reg (one CTA: dependent LU chains), and the back-transformation in k_rr_back (one
// CTA per column).
constexpr int EV_MMAX = 512;

// Eigenvalue blockIdx.x of the tridiagonal T = (d, e) (m rows: m_full, less mP when *pflag is
// 0) by 33-point multisection on Sturm counts with the 32 lanes of the CTA's warp (an FP64 warp
// instruction costs the same with 8 lanes or 32), after the Gershgorin bounds of
// rr_phase_eigvals, recomputed by every CTA.
template <typename T>
__device__ __forceinline__ void rr_eigval_one(int j, int m_full, int K, int mP, const int* pflag,
                                              const T* __restrict__ d, const T* __restrict__ e,
                                              T* __restrict__ lam, int* status) {
  constexpr int LG = 32;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ T e2[EV_MMAX];
  const int m = (pflag && *pflag == 0) ? m_full - mP : m_full;
  const int lane = threadIdx.x;
  T lo = (T)3e38, hi = (T)-3e38, emax = 0;
  for (int i = lane; i < m; i += 32) {
    T r = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : (T)0);
    lo = min(lo, d[i] - r);
    hi = max(hi, d[i] + r);
    emax = max(emax, e[i] * e[i]);
    e2[i] = e[i] * e[i];
    if (j == 0 && (!isfinite(d[i]) || !isfinite(e[i]))) atomicOr(status, ST_NONFINITE);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(FULL, lo, o));
    hi = max(hi, __shfl_xor_sync(FULL, hi, o));
    emax = max(emax, __shfl_xor_sync(FULL, emax, o));
  }
  __syncwarp();
  const T tnorm = max(fabs(lo), fabs(hi));
  const T pivmin = Lim<T>::tiny() * max((T)1, emax);
  const T glo = lo - (T)2 * Lim<T>::eps() * tnorm - pivmin;
  const T ghi = hi + (T)2 * Lim<T>::eps() * tnorm + pivmin;
  const T abstol = Lim<T>::eps() * tnorm;
  if (lane >= LG) return;
  const int sl = lane;
  const unsigned gmask = 0xffffffffu;
  T a = glo, b = ghi;
  for (int it = 0; it < 64; ++it) {
    T tol = max((T)2 * Lim<T>::eps() * max(fabs(a), fabs(b)), abstol) + (T)4 * pivmin;
    if (b - a <= tol) break;
    T h = (b - a) / (T)(LG + 1);
    const int c = sturm_count(m, d, e2, a + h * (T)(sl + 1), pivmin);
    unsigned bal = __ballot_sync(gmask, c > j);
    int first = bal ? (__ffs(bal) - 1) : LG;
    T na = first == 0 ? a : a + h * (T)first;
    T nb = first == LG ? b : a + h * (T)(first + 1);
    if (!(nb > na)) break;
    a = na;
    b = nb;
  }
  if (sl == 0) lam[j] = (T)0.5 * (a + b);
}

template <typename T>
__global__ void __launch_bounds__(32)
    k_rr_eigvals_cta(int m_full, int K, int mP, const int* pflag, const T* __restrict__ d,
                     const T* __restrict__ e, T* __restrict__ lam, int* status) {
  rr_eigval_one<T>(blockIdx.x, m_full, K, mP, pflag, d, e, lam, status);
}
// Lockstep batch (FP32 cluster group): CTA (j, q) finds eigenvalue j of descriptor q.
__global__ void __launch_bounds__(32) k_rr_eigvals_cta_b(const RrDesc* __restrict__ tab) {
  const RrDesc a = tab[blockIdx.y];
  if ((int)blockIdx.x >= a.K) return;  // uniform in the CTA
  rr_eigval_one<float>(blockIdx.x, a.m, a.K, a.mP, a.pflag, a.tri, a.tri + a.m, a.lamx, a.status);
}

// Back-transformation Y = H_0 ... H_{m-3} Z of one column per CTA (one warp): the arithmetic
// of k_rr_eig_reg's phase 4 for that column.  The reflectors are the rows of Ag (stride lda),
// m the solved size k_rr_eig_reg left in *mext; CTA 0 then re-arms *pflag (nothing else reads
// it before the next pass).
template <typename T, int NS>
__device__ __forceinline__ void rr_back_one(int j, int m_full, int K, const int* __restrict__ mext,
                                            const T* __restrict__ Ag, int lda,
                                            const T* __restrict__ beta, const T* __restrict__ Z,
                                            T* __restrict__ Y, int* pflag, int* nfallback) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  const int m = *mext;
  T za[NS];
#pragma unroll
  for (int u = 0; u < NS; ++u) {
    const int i = lane + 32 * u;
    za[u] = i < m ? Z[(long long)i * K + j] : (T)0;
  }
  // reflector kr: v_i = 1 at i = kr + 1, the stored row beyond, 0 before; the next one is
  // loaded while the current one's dot product reduces
  auto load_v = [&](int kr, T (&cv)[NS]) {
    const T* vk = Ag + (long long)kr * lda;
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      const int i = lane + 32 * u;
      cv[u] = (i == kr + 1) ? (T)1 : ((i > kr + 1 && i < m) ? vk[i] : (T)0);
    }
  };
  T cv[NS], nv[NS];
  if (m >= 3) load_v(m - 3, cv);
  for (int kr = m - 3; kr >= 0; --kr) {
    const T bet = beta[kr];
    if (kr > 0) load_v(kr - 1, nv);
    if (bet == (T)0) {
#pragma unroll
      for (int u = 0; u < NS; ++u) cv[u] = nv[u];
      continue;
    }
    T sa = 0;
#pragma unroll
    for (int u = 0; u < NS; ++u) sa = fma(cv[u], za[u], sa);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(FULL, sa, o);
    sa *= bet;
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      za[u] = fma(-sa, cv[u], za[u]);
      cv[u] = nv[u];
    }
  }
#pragma unroll
  for (int u = 0; u < NS; ++u) {
    const int i = lane + 32 * u;
    if (i < m_full) Y[(long long)i * K + j] = i < m ? za[u] : (T)0;
  }
  if (j == 0 && lane == 0 && pflag) {
    if (*pflag == 0 && nfallback) *nfallback += 1;
    *pflag = 1;  // re-armed for the next pass
  }
}

template <typename T, int NS>
__global__ void __launch_bounds__(32)
    k_rr_back(int m_full, int K, const int* __restrict__ mext, const T* __restrict__ Ag, int lda,
              const T* __restrict__ beta, const T* __restrict__ Z, T* __restrict__ Y, int* pflag,
              int* nfallback) {
  rr_back_one<T, NS>(blockIdx.x, m_full, K, mext, Ag, lda, beta, Z, Y, pflag, nfallback);
}
// Lockstep batch (FP32 cluster group): CTA (j, q) back-transforms column j of descriptor q.
__global__ void __launch_bounds__(32) k_rr_back_b(const RrDesc* __restrict__ tab) {
  const RrDesc a = tab[blockIdx.y];
  if ((int)blockIdx.x >= a.K) return;  // uniform in the CTA
  const float* Zg = a.Ag + (size_t)a.m * (a.m + 16);
  rr_back_one<float, EV_MMAX / 32>(blockIdx.x, a.m, a.K, a.mx, a.Ag, a.m, a.tri + 2 * a.m, Zg,
                                   a.Y, a.pflag, a.nfallback);
}

// ---------------------------------------------------------------------------------------
// Rayleigh-Ritz with the matrix held in registers, m <= 32 RS, FP32, 16 warps.  Half-warp
// g = 2 warp + lane / 16 (0..31) owns rows g + 32 r (r < RS); lane cl = lane % 16 of it owns
// columns cl + 16 c (c < CS = 2 RS) of those rows.
//  1. Householder tridiagonalization (Golub & Van Loan Alg. 8.3.1), two barriers per step.
//     Step k has q = k / 16, the column slot of k, as a compile-time index: the slots r < q / 2
//     and c < q hold rows and columns <= k only, which the step leaves alone, so they drop out
//     of the loops as the trailing block shrinks.
//      (a) the lanes owning column k publish x_i = a_ik (i > k) into row k of Vs and per
//          half-warp sums of x_i^2 (i > k + 1); the owner of a_kk writes d_k;
//      (b) every thread forms the reflector scalars (mu, v0, beta, e_k) from sigma^2 and
//          x_{k+1}, and v = e_{k+1} + x / v0 on its rows and columns;
//      (c) p_i = beta (A v)_i on the owned rows: register dot products over the owned columns
//          and half-warp butterflies; p and per-half-warp sums of p_i v_i go to shared memory;
//      (d) w = p - (beta / 2)(p'v) v and the rank-2 update A -= v w' + w v' of the owned
//          entries.
//     The lane that reads a_i,k+1 in the next step's (a) is the one that updated it in (d).
//  2. and 3. as in k_rr_eig_reg (rr_phase_eigvals, rr_phase_eigvecs).
//  4. Back-transformation Y = H_0 ... H_{m-3} Z with the reflectors of Vs (v_j = x_j / v0),
//     CPW columns per warp held in registers, the next reflector loaded while the current
//     one's dot products reduce.
template <int N>
__device__ __forceinline__ float halfwarp_sum(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int RT_NW = 16;
constexpr int RT_NT = RT_NW * 32;

// Row stride of the reflector store: the padded width 32 RS, plus one.
__host__ __device__ inline int rt_ldv(int rs) { return 32 * rs + 1; }

// Shared-memory floats of k_rr_eig_rt<RS> for an m x m problem with K wanted pairs.
__host__ __device__ inline size_t rt_smem_floats(int m, int K, int rs) {
  return (size_t)5 * m + 32 * (size_t)rs + 7 * (size_t)K + 3 * RT_NW + 8 + 64 +
         (size_t)m * rt_ldv(rs) + 4 * (size_t)m * K + (size_t)K * K;
}

template <int RS>
__device__ __forceinline__ void k_rr_eig_rt_body(int m_full, int K, const double* __restrict__ G,
                                                 int ldg, double* __restrict__ theta,
                                                 float* __restrict__ Y, int* status, int* pflag,
                                                 int mP, int* nfallback) {
  using T = float;
  constexpr int CS = 2 * RS;
  constexpr unsigned FULL = 0xffffffffu;
  const int m = (pflag && *pflag == 0) ? m_full - mP : m_full;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* d = (T*)smraw;       // m
  T* e = d + m;           // m
  T* beta = e + m;        // m
  T* e2 = beta + m;       // m
  T* ivs = e2 + m;        // m: 1 / v0 of each reflector
  T* pvec = ivs + m;      // 32 RS: p of the current step (padded rows included)
  T* lam = pvec + 32 * RS;  // K
  T* shift = lam + K;     // K
  T* dd = shift + K;      // K
  T* cbuf = dd + K;       // 2 K
  T* wv = cbuf + 2 * K;   // K
  T* coef = wv + K;       // K
  T* red = coef + K;      // 3 NW + 8 (the shared phases' slots)
  T* rs2 = red + 3 * RT_NW + 8;  // 32 half-warp sums of x^2
  T* rpv = rs2 + 32;             // 32 half-warp sums of p_i v_i
  const int ldv = rt_ldv(RS);
  T* Vs = rpv + 32;              // m x ldv: row k = x of reflector k
  T* Z = Vs + (size_t)m * ldv;   // m x K
  T* U = Z + (size_t)m * K;      // 3 m K
  T* Gs = U + (size_t)3 * m * K; // K x K
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = 2 * warp + (lane >> 4), cl = lane & 15;

  // ---- load (symmetrized), Gershgorin bound, lift the diagonal of dropped columns.  G is
  // staged in the (not yet used) reflector / eigenvector region with coalesced row reads when
  // it fits there, so that the symmetrization's transposed reads hit shared memory
  const double* Gsrc = G;
  long long lds = ldg;
  {
    double* Gst = (double*)(((uintptr_t)Vs + 7) & ~(uintptr_t)7);
    const size_t room = (size_t)m * ldv + 4 * (size_t)m * K + (size_t)K * K - 2;
    if ((size_t)2 * m * m <= room) {
      stage_f64(G, ldg, m, m, Gst, tid, RT_NT);
      __syncthreads();
      Gsrc = Gst;
      lds = m;
    }
  }
  T A[RS][CS];
  T gmax = 0;
#pragma unroll
  for (int r = 0; r < RS; ++r) {
    const int i = g + 32 * r;
    T rs = 0;
#pragma unroll
    for (int c = 0; c < CS; ++c) {
      const int j = cl + 16 * c;
      T a = 0;
      if (i < m && j < m) a = (T)(0.5 * (Gsrc[(long long)i * lds + j] + Gsrc[(long long)j * lds + i]));
      A[r][c] = a;
      rs += fabsf(a);
    }
    gmax = fmaxf(gmax, halfwarp_sum<16>(rs));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gmax = fmaxf(gmax, __shfl_xor_sync(FULL, gmax, o));
  if (lane == 0) red[warp] = gmax;
  __syncthreads();
  {
    T big = 0;
    for (int w = 0; w < RT_NW; ++w) big = fmaxf(big, red[w]);
    big = big * (T)1.25 + (T)1;
#pragma unroll
    for (int r = 0; r < RS; ++r)
#pragma unroll
      for (int c = 0; c < CS; ++c) {
        const int i = g + 32 * r, j = cl + 16 * c;
        if (i == j && i >= K && i < m && G[(long long)i * ldg + i] == 0.0) A[r][c] = big;
      }
  }
  __syncthreads();
  RR_MARK(0);

  // ---- 1. tridiagonalization
  // Row k of Vs receives x_i (i > k) in step k and is zero elsewhere (zero-filled here, and
  // padded to 32 RS columns), so that v = x / v0 needs no masks: its entries at i <= k and at
  // i >= m come out zero.  Entries of A outside the trailing block (rows or columns <= k) and
  // the upper / padded slots receive updates that are never read again.
  for (int idx = tid; idx < m * ldv; idx += RT_NT) Vs[idx] = (T)0;
  __syncthreads();
  bool stop = false;
#pragma unroll
  for (int q = 0; q < CS; ++q) {
    if (stop) break;
    const int r0 = q / 2;
    for (int kw = 0; kw < 16; ++kw) {
      const int k = 16 * q + kw;
      if (k + 2 >= m) {
        stop = true;
        break;
      }
      const int k1 = k + 1;
      T* __restrict__ xs = Vs + (size_t)k * ldv;
      // (a)
      if (cl == kw) {
        T s2 = 0;
#pragma unroll
        for (int r = r0; r < RS; ++r) {
          const int i = g + 32 * r;
          const T x = A[r][q];
          if (i > k) xs[i] = x;
          s2 = fmaf(i > k1 ? x : (T)0, x, s2);
        }
        rs2[g] = s2;
        if (g == (k & 31)) d[k] = A[r0][q];
      }
      __syncthreads();
      // (b)
      T sg = rs2[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(FULL, sg, o);
      const T x0 = xs[k1];
      T bet = 0, iv0 = 0, ek = x0;
      if (sg != (T)0) {
        // x -> ek e1 with ek = -sign(x0) mu: v0 = x0 - ek has |v0| >= mu, so the tail of
        // v = x / v0 stays <= 1 however small sigma is; beta = 2 / (1 + sigma / v0^2)
        const T mu = sqrtf(x0 * x0 + sg);
        const T v0 = x0 + copysignf(mu, x0);
        iv0 = __frcp_rn(v0);
        bet = (T)2 * __frcp_rn((T)1 + sg * iv0 * iv0);
        ek = -copysignf(mu, x0);
      }
      if (tid == 0) {
        e[k] = ek;
        beta[k] = bet;
        ivs[k] = iv0;
      }
      T vc[CS], vr[RS], pr[RS];
#pragma unroll
      for (int c = q & ~1; c < CS; ++c) {
        vc[c] = xs[cl + 16 * c] * iv0;  // slot q - 1 (q odd): columns <= k, zero in row k
        if (c >= q && c <= q + 1 && cl + 16 * c == k1) vc[c] = (T)1;  // only slots q, q + 1
      }
#pragma unroll
      for (int r = r0; r < RS; ++r) {
        vr[r] = xs[g + 32 * r] * iv0;
        if (r <= r0 + 1 && g + 32 * r == k1) vr[r] = (T)1;
      }
      // (c)
      T pvp = 0;
      // (the column pairs start at an even slot: slot q - 1, when q is odd, holds columns <= k,
      // whose v entries are zero)
#pragma unroll
      for (int r = r0; r < RS; ++r) {
        float2 sacc2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = q & ~1; c < CS; c += 2)
          sacc2 = __ffma2_rn(make_float2(A[r][c], A[r][c + 1]), make_float2(vc[c], vc[c + 1]), sacc2);
        pr[r] = bet * halfwarp_sum<16>(sacc2.x + sacc2.y);
        pvp = fmaf(pr[r], vr[r], pvp);
      }
      if (cl == 0) {
        rpv[g] = pvp;
#pragma unroll
        for (int r = r0; r < RS; ++r) pvec[g + 32 * r] = pr[r];
      }
      __syncthreads();
      // (d)
      T pv = rpv[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(FULL, pv, o);
      const T kc = bet * (T)0.5 * pv;
      T wr[RS];
#pragma unroll
      for (int r = r0; r < RS; ++r) wr[r] = fmaf(-kc, vr[r], pr[r]);
      // rank-2 update, two columns per packed FMA (each half rounds as fmaf; the pair that
      // starts at slot q - 1 updates dead entries)
#pragma unroll
      for (int c = q & ~1; c < CS; c += 2) {
        const float2 vc2 = make_float2(vc[c], vc[c + 1]);
        const float2 wj2 = __ffma2_rn(make_float2(-kc, -kc), vc2,
                                      make_float2(pvec[cl + 16 * c], pvec[cl + 16 * (c + 1)]));
#pragma unroll
        for (int r = r0; r < RS; ++r) {
          const float2 a = __ffma2_rn(make_float2(-vr[r], -vr[r]), wj2,
                                      __ffma2_rn(make_float2(-wr[r], -wr[r]), vc2,
                                                 make_float2(A[r][c], A[r][c + 1])));
          A[r][c] = a.x;
          A[r][c + 1] = a.y;
        }
      }
    }
  }
  __syncthreads();
  // the trailing 2 x 2 block of T (or the 1 x 1 matrix), from the owners of its entries
#pragma unroll
  for (int r = 0; r < RS; ++r)
#pragma unroll
    for (int c = 0; c < CS; ++c) {
      const int i = g + 32 * r, j = cl + 16 * c;
      if (m >= 2) {
        if (i == m - 2 && j == m - 2) d[m - 2] = A[r][c];
        if (i == m - 1 && j == m - 2) e[m - 2] = A[r][c];
        if (i == m - 1 && j == m - 1) d[m - 1] = A[r][c];
      } else if (i == 0 && j == 0) {
        d[0] = A[r][c];
      }
    }
  if (tid == 0) e[m - 1] = 0;
  __syncthreads();
  RR_MARK(1);

  // ---- 2. and 3.
  T tnorm, pivmin;
  rr_phase_eigvals<T, RT_NT>(m, K, d, e, e2, red, lam, status, tnorm, pivmin);
  RR_MARK(2);
  rr_phase_eigvecs<T, RT_NT>(m, K, d, e, lam, shift, Z, U, Gs, dd, cbuf, wv, coef, red, tnorm,
                             pivmin);
  RR_MARK(4);

  // ---- 4. back-transformation Y = H_0 ... H_{m-3} Z, CPW columns per warp in registers
  {
    constexpr int CPW = 3;
    for (int j0 = CPW * warp; j0 < K; j0 += CPW * RT_NW) {
      T z[CPW][RS];
#pragma unroll
      for (int t = 0; t < CPW; ++t)
#pragma unroll
        for (int u = 0; u < RS; ++u) {
          const int i = lane + 32 * u, j = j0 + t;
          z[t][u] = (i < m && j < K) ? Z[i * K + j] : (T)0;
        }
      // reflector kr: v_i = 1 at i = kr + 1, x_i / v0 beyond, 0 before
      auto load_v = [&](int kr, T (&cv)[RS]) {
        const T* __restrict__ xk = Vs + (size_t)kr * ldv;
        const T iv = ivs[kr];
#pragma unroll
        for (int u = 0; u < RS; ++u) {
          const int i = lane + 32 * u;
          cv[u] = i == kr + 1 ? (T)1 : xk[i] * iv;  // zero at i <= kr and i >= m
        }
      };
      T cv[RS], nv[RS];
      int kr = m - 3;
      if (kr >= 0) load_v(kr, cv);
      for (; kr >= 0; --kr) {
        const T bet = beta[kr];
        if (kr > 0) load_v(kr - 1, nv);
        if (bet != (T)0) {  // uniform
          T sa[CPW];
#pragma unroll
          for (int t = 0; t < CPW; ++t) {
            float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u + 1 < RS; u += 2)
              acc2 = __ffma2_rn(make_float2(cv[u], cv[u + 1]), make_float2(z[t][u], z[t][u + 1]), acc2);
            if (RS % 2) acc2.x = fmaf(cv[RS - 1], z[t][RS - 1], acc2.x);
            sa[t] = acc2.x + acc2.y;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int t = 0; t < CPW; ++t) sa[t] += __shfl_xor_sync(FULL, sa[t], o);
#pragma unroll
          for (int t = 0; t < CPW; ++t) {
            const T f = bet * sa[t];
#pragma unroll
            for (int u = 0; u + 1 < RS; u += 2) {
              const float2 zz = __ffma2_rn(make_float2(-f, -f), make_float2(cv[u], cv[u + 1]),
                                           make_float2(z[t][u], z[t][u + 1]));
              z[t][u] = zz.x;
              z[t][u + 1] = zz.y;
            }
            if (RS % 2) z[t][RS - 1] = fmaf(-f, cv[RS - 1], z[t][RS - 1]);
          }
        }
#pragma unroll
        for (int u = 0; u < RS; ++u) cv[u] = nv[u];
      }
#pragma unroll
      for (int t = 0; t < CPW; ++t)
#pragma unroll
        for (int u = 0; u < RS; ++u) {
          const int i = lane + 32 * u, j = j0 + t;
          if (i < m_full && j < K) Y[(long long)i * K + j] = i < m ? z[t][u] : (T)0;
        }
    }
  }
  RR_MARK(5);
  for (int j = tid; j < K; j += RT_NT) theta[j] = (double)lam[j];
  if (pflag && tid == 0) {
    if (*pflag == 0 && nfallback) *nfallback += 1;
    *pflag = 1;  // re-armed for the next pass
  }
  RR_MARK(6);
}


template <int RS>
__global__ void __launch_bounds__(RT_NT, 1)
    k_rr_eig_rt(int m_full, int K, const double* __restrict__ G, int ldg,
                double* __restrict__ theta, float* __restrict__ Y, int* status, int* pflag,
                int mP, int* nfallback) {
  k_rr_eig_rt_body<RS>(m_full, K, G, ldg, theta, Y, status, pflag, mP, nfallback);
}
// One CTA per descriptor of a lockstep batch.
template <int RS>
__global__ void __launch_bounds__(RT_NT, 1) k_rr_eig_rt_b(const RrDesc* __restrict__ tab) {
  const RrDesc a = tab[blockIdx.x];
  k_rr_eig_rt_body<RS>(a.m, a.K, a.G, a.ldg, a.theta, a.Y, a.status, a.pflag, a.mP, a.nfallback);
}

// Cholesky-QR transform in FP32 with the factorization in registers (ldl_inv_reg, four warps,
// ka <= min(8 RS, 16 CS)): the same arithmetic as k_chol_inv (scaled FP64 Gram, in-place LDL'
// with L^-1 formed alongside, column drops, floors, the direction-block fallback).
constexpr int CR_NW = 4;
template <int RS, int CS>
__device__ __forceinline__ void k_chol_inv_rt_body(int ka, const double* __restrict__ G, int ldg,
                                                   float* __restrict__ Tm, int* status,
                                                   int* fail_col, double pivot_tol, int keep,
                                                   int* pflag, int ndrop, int* ndropped,
                                                   double rfloor, double pfloor) {
  using T = float;
  constexpr int NTH = CR_NW * 32;
  extern __shared__ __align__(16) unsigned char craw[];
  T* s = (T*)craw;                 // ka scale factors
  T* dd = s + ka;                  // ka pivots
  T* buf = dd + ka;                // 2 x 16 CS
  T* W = buf + 2 * 16 * CS;        // ka x ka
  double* Gs = (double*)(((uintptr_t)(W + (size_t)ka * ka) + 15) & ~(uintptr_t)15);  // ka x ka
  __shared__ int sfc;
  const int tid = threadIdx.x;
  // the FP64 Gram staged with coalesced row reads (the symmetrization reads its transpose)
  stage_f64(G, ldg, ka, ka, Gs, tid, NTH);
  __syncthreads();
  for (int i = tid; i < ka; i += NTH) {
    const double dgi = Gs[i * ka + i];
    const double fl = i < keep ? rfloor * rfloor : pfloor * pfloor;
    s[i] = dgi > fl ? (T)rsqrt(dgi) : (T)0;
  }
  __syncthreads();
  for (int idx = tid; idx < ka * ka; idx += NTH) {
    const int i = idx / ka, j = idx % ka;
    if (j > i) continue;
    const double gg = 0.5 * (Gs[i * ka + j] + Gs[j * ka + i]);
    W[i * ka + j] = (T)gg * s[i] * s[j];
  }
  __syncthreads();
  const int f = ldl_inv_reg<CR_NW, RS, CS>(ka, W, ka, dd, buf, (T)pivot_tol, ndrop, ndrop > 0);
  if (tid == 0) sfc = f;
  __syncthreads();
  const int fc = sfc;
  if (ndropped && tid == 0) {
    const int lim = fc >= 0 ? fc : ka;
    int cnt = 0;
    for (int k = 0; k < lim; ++k) cnt += dd[k] == (T)0;
    if (cnt) atomicAdd(ndropped, cnt);
  }
  int kk = ka;  // size of the leading block whose transform is returned
  if (fc >= 0) {
    if (pflag && keep > 0 && fc >= keep) {
      kk = keep;
      if (tid == 0) *pflag = 0;
    } else {
      if (tid == 0) {
        atomicOr(status, ST_CHOL_FAIL);
        if (fail_col) *fail_col = fc;
      }
      return;
    }
  }
  for (int i = tid; i < kk; i += NTH) buf[i] = dd[i] > (T)0 ? rsqrtf(dd[i]) : (T)0;
  __syncthreads();
  // Tm[r][c] = s_r (L^-1)_cr d_c^-1/2 for r <= c < kk, else 0
  for (int idx = tid; idx < ka * ka; idx += NTH) {
    const int r = idx / ka, c = idx % ka;
    T v = 0;
    if (r <= c && c < kk) v = s[r] * (r == c ? (T)1 : W[c * ka + r]) * buf[c];
    Tm[(long long)r * ka + c] = v;
  }
}

template <int RS, int CS>
__global__ void __launch_bounds__(CR_NW * 32, 1)
    k_chol_inv_rt(int ka, const double* __restrict__ G, int ldg, float* __restrict__ Tm,
                  int* status, int* fail_col, double pivot_tol, int keep, int* pflag, int ndrop,
                  int* ndropped, double rfloor, double pfloor) {
  k_chol_inv_rt_body<RS, CS>(ka, G, ldg, Tm, status, fail_col, pivot_tol, keep, pflag, ndrop,
                             ndropped, rfloor, pfloor);
}
// One CTA per descriptor of a lockstep batch.
template <int RS, int CS>
__global__ void __launch_bounds__(CR_NW * 32, 1) k_chol_inv_rt_b(const CholDesc* __restrict__ tab) {
  const CholDesc a = tab[blockIdx.x];
  k_chol_inv_rt_body<RS, CS>(a.ka, a.G, a.ldg, a.Tm, a.status, a.fail_col, a.pivot_tol, a.keep,
                             a.pflag, a.ndrop, a.ndropped, a.rfloor, a.pfloor);
}

}  // namespace

template <typename T>
cudaError_t chol_inv_nt(cudaStream_t st, Alloc& al, int ka, const double* G, int ldg, T* Tm,
                        int* d_status, double pivot_tol, int* fail_col, int keep, int* pflag,
                        int ndrop, int* ndropped, double rfloor, double pfloor,
                        int nthreads);


template <int RS, int CS>
cudaError_t chol_inv_rt(cudaStream_t st, int ka, const double* G, int ldg, float* Tm,
                        int* d_status, double pivot_tol, int* fail_col, int keep, int* pflag,
                        int ndrop, int* ndropped, double rfloor, double pfloor) {
  const size_t sm = sizeof(float) * ((size_t)2 * ka + 32 * CS + (size_t)ka * ka) + 16 +
                    sizeof(double) * (size_t)ka * ka;
  auto kern = k_chol_inv_rt<RS, CS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  ProfScope ps(st, "chol_inv");
  kern<<<1, CR_NW * 32, sm, st>>>(ka, G, ldg, Tm, d_status, fail_col, pivot_tol, keep, pflag,
                                  ndrop, ndropped, rfloor, pfloor);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t chol_inv(cudaStream_t st, Alloc& al, int ka, const double* G, int ldg, T* Tm,
                     int* d_status, double pivot_tol, int* fail_col, int keep, int* pflag,
                     int ndrop, int* ndropped, double rfloor, double pfloor) {
  if constexpr (sizeof(T) == 4) {
    if (ka >= 1 && ka <= 64)
      return chol_inv_rt<8, 4>(st, ka, G, ldg, Tm, d_status, pivot_tol, fail_col, keep, pflag,
                               ndrop, ndropped, rfloor, pfloor);
    if (ka <= 96)
      return chol_inv_rt<12, 6>(st, ka, G, ldg, Tm, d_status, pivot_tol, fail_col, keep, pflag,
                                ndrop, ndropped, rfloor, pfloor);
    if (ka <= 128)
      return chol_inv_rt<16, 8>(st, ka, G, ldg, Tm, d_status, pivot_tol, fail_col, keep, pflag,
                                ndrop, ndropped, rfloor, pfloor);
  }
  return chol_inv_nt<T>(st, al, ka, G, ldg, Tm, d_status, pivot_tol, fail_col, keep, pflag, ndrop,
                        ndropped, rfloor, pfloor, 512);
}

template <typename T>
cudaError_t chol_inv_nt(cudaStream_t st, Alloc& al, int ka, const double* G, int ldg, T* Tm,
                        int* d_status, double pivot_tol, int* fail_col, int keep, int* pflag,
                        int ndrop, int* ndropped, double rfloor, double pfloor,
                        int nthreads) {
  size_t base = sizeof(T) * (4 * (size_t)ka);
  size_t wbytes = sizeof(T) * (size_t)ka * ka;
  int in_smem = base + wbytes <= 200 * 1024;
  size_t sm = base + (in_smem ? wbytes : 0);
  T* Wg = nullptr;
  if (!in_smem) {
    Wg = al.get<T>((size_t)ka * ka);
    if (!Wg) return cudaErrorMemoryAllocation;
  }
  auto kern = in_smem ? k_chol_inv<T, true> : k_chol_inv<T, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  ProfScope ps(st, "chol_inv");
  kern<<<1, nthreads, sm, st>>>(ka, G, ldg, Tm, Wg, d_status, fail_col, pivot_tol, keep, pflag,
                                ndrop, ndropped, rfloor, pfloor);
  note_launch();
  e = cudaGetLastError();
  al.put(Wg);
  return e;
}

// Register-slot Rayleigh-Ritz: shared-memory sizes and launch for one (NS, NW) shape.
template <typename T, int NS, int NW>
cudaError_t rr_eig_reg(cudaStream_t st, Alloc& al, int m, int K, const double* G, int ldg,
                       double* theta, T* Y, int* d_status, int* pflag, int mP, int* nfallback) {
  const size_t base = sizeof(T) * ((size_t)6 * m + 7 * (size_t)K + 3 * NW + 8);
  if (m > NW * 32) return cudaErrorInvalidValue;
  // the matrix rows are padded to rr_lda(m', tpr) <= m' + 15 for the m' <= m the kernel solves
  const size_t big = sizeof(T) * ((size_t)m * (m + 16) + 4 * (size_t)m * K + (size_t)K * K);
  constexpr bool can_sm = sizeof(T) == 4 && NS == 5;  // the only shape whose blocks fit
  const bool insm = can_sm && base + big <= 220 * 1024;
  const size_t sm = base + (insm ? big : 0);
  T* Ag = nullptr;
  if (!insm) {
    Ag = al.get<T>((size_t)m * (m + 16) + 4 * (size_t)m * K + (size_t)K * K);
    if (!Ag) return cudaErrorMemoryAllocation;
  }
  T* Zg = insm ? nullptr : Ag + (size_t)m * (m + 16);
  T* Ug = insm ? nullptr : Zg + (size_t)m * K;
  T* Gsg = insm ? nullptr : Ug + (size_t)3 * m * K;
  auto kern = k_rr_eig_reg<T, NS, NW, false>;
  if constexpr (can_sm) {
    if (insm) kern = k_rr_eig_reg<T, NS, NW, true>;
  }
  // FP64 (64 < m <= 256) and FP32 (160 < m <= 512): the phases spread over SMs
  // (tridiagonalization on a cluster, one CTA per eigenvalue, the eigenvectors here, one CTA
  // per back-transformed column)
  {
    constexpr bool f64 = sizeof(T) == 8;
    if (!insm && (f64 ? (m > 64 && m <= 256) : (m > 160 && m <= EV_MMAX))) {
      T* tri = al.get<T>((size_t)3 * m + K);  // d, e, beta, eigenvalues
      int* mx = al.get<int>(1);
      cudaError_t e = (tri && mx) ? cudaSuccess : cudaErrorMemoryAllocation;
      if (e == cudaSuccess)
        e = tridiag_cluster(st, m, K, G, ldg, Ag, m, tri, tri + m, tri + 2 * m, pflag, mP);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e == cudaSuccess) {
        ProfScope ps(st, "rr_eig");
        k_rr_eigvals_cta<T><<<K, 32, 0, st>>>(m, K, mP, pflag, tri, tri + m, tri + 3 * m,
                                               d_status);
        note_launch();
        kern<<<1, NW * 32, sm, st>>>(m, K, G, ldg, theta, Y, Ag, Zg, Ug, Gsg, d_status, pflag, mP,
                                     nfallback, tri, tri + m, tri + 2 * m, m, tri + 3 * m, mx);
        note_launch();
        k_rr_back<T, (f64 ? 256 : EV_MMAX) / 32><<<K, 32, 0, st>>>(m, K, mx, Ag, m, tri + 2 * m,
                                                                   Zg, Y, pflag, nfallback);
        note_launch();
        e = cudaGetLastError();
      }
      al.put(mx);
      al.put(tri);
      al.put(Ag);
      return e;
    }
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess) {
    ProfScope ps(st, "rr_eig");
    kern<<<1, NW * 32, sm, st>>>(m, K, G, ldg, theta, Y, Ag, Zg, Ug, Gsg, d_status, pflag, mP,
                                 nfallback, nullptr, nullptr, nullptr, 0, nullptr, nullptr);
    note_launch();
    e = cudaGetLastError();
  }
  al.put(Ag);
  return e;
}


// Register-resident Rayleigh-Ritz (FP32, m <= 32 RS): launch with the whole working set in
// shared memory.  Returns cudaErrorNotSupported when it does not fit (the caller falls back).
template <int RS>
cudaError_t rr_eig_rt(cudaStream_t st, int m, int K, const double* G, int ldg, double* theta,
                      float* Y, int* d_status, int* pflag, int mP, int* nfallback) {
  const size_t sm = sizeof(float) * rt_smem_floats(m, K, RS);
  if (m > 32 * RS || sm > 225 * 1024) return cudaErrorNotSupported;
  auto kern = k_rr_eig_rt<RS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  ProfScope ps(st, "rr_eig");
  kern<<<1, RT_NT, sm, st>>>(m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t rr_eig(cudaStream_t st, Alloc& al, int m, int K, const double* G, int ldg,
                   double* theta, T* Y, int* d_status, int* pflag, int mP, int* nfallback) {
  if (m < 1 || K < 1 || K > m) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    // register-resident tridiagonalization when the working set fits in shared memory
    cudaError_t e = cudaErrorNotSupported;
    if (m <= 64) e = rr_eig_rt<2>(st, m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
    else if (m <= 96) e = rr_eig_rt<3>(st, m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
    else if (m <= 128) e = rr_eig_rt<4>(st, m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
    else if (m <= 160) e = rr_eig_rt<5>(st, m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
    if (e != cudaErrorNotSupported) return e;
  }
  // m <= 480: register-slot kernel (m = 3K up to K = 160)
  if (m <= 160) {
    if constexpr (sizeof(T) == 4)
      return rr_eig_reg<T, 5, 32>(st, al, m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
    else
      return rr_eig_reg<T, 5, 16>(st, al, m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
  }
  if (m <= 320)
    return rr_eig_reg<T, 10, 16>(st, al, m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
  if (m <= 480)
    return rr_eig_reg<T, 15, 16>(st, al, m, K, G, ldg, theta, Y, d_status, pflag, mP, nfallback);
  size_t base = sizeof(T) * ((size_t)6 * m + K + 128);
  size_t abytes = sizeof(T) * (size_t)m * m;
  size_t zbytes = sizeof(T) * (size_t)m * K;
  const size_t cap = 220 * 1024;
  const bool insm = base + abytes + zbytes <= cap;
  size_t sm = base + (insm ? abytes + zbytes : 0);
  T* Ag = insm ? nullptr : al.get<T>((size_t)m * m);
  T* Zg = insm ? nullptr : al.get<T>((size_t)m * K);
  T* lu = al.get<T>((size_t)K * 5 * m);
  T* Gs = al.get<T>((size_t)K * K * 2);
  cudaError_t e = cudaSuccess;
  if ((!insm && (!Ag || !Zg)) || !lu || !Gs) {
    e = cudaErrorMemoryAllocation;
  } else {
    auto kern = insm ? k_rr_eig<T, true> : k_rr_eig<T, false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
      ProfScope ps(st, "rr_eig");
      kern<<<1, RR_NT, sm, st>>>(m, K, G, ldg, theta, Y, Ag, Zg, lu, Gs, d_status, pflag, mP,
                                 nfallback);
      note_launch();
      e = cudaGetLastError();
    }
  }
  al.put(Ag);
  al.put(Zg);
  al.put(lu);
  al.put(Gs);
  return e;
}

// ---- lockstep batches ------------------------------------------------------------------
// Groups of the batched Cholesky-QR transforms (FP32): kind 0 = the four-warp register form
// (ka <= 128; param = the register shape of the group's largest ka), kind 1 = the shared-memory
// form, kind 2 = the global-memory form (Wg per descriptor).  The register shapes differ only in
// unused slots, so a factorization gives the same bits in any of them.
static int chol_rt_shape(int ka) { return ka <= 64 ? 0 : ka <= 96 ? 1 : 2; }
static size_t chol_rt_smem(int ka, int shape) {
  const int CS = shape == 0 ? 4 : shape == 1 ? 6 : 8;
  return sizeof(float) * ((size_t)2 * ka + 32 * CS + (size_t)ka * ka) + 16 +
         sizeof(double) * (size_t)ka * ka;
}
static size_t chol_nt_base(int ka) { return sizeof(float) * 4 * (size_t)ka; }
static bool chol_nt_insm(int ka) {
  return chol_nt_base(ka) + sizeof(float) * (size_t)ka * ka <= 200 * 1024;
}
size_t chol_batch_scratch(int ka) { return (ka > 128 && !chol_nt_insm(ka)) ? (size_t)ka * ka : 0; }

void chol_batch_plan(std::vector<CholDesc>& d, std::vector<BatchGroup>& groups,
                     std::vector<int>& single) {
  auto kind = [](const CholDesc& a) { return a.ka <= 128 ? 0 : chol_nt_insm(a.ka) ? 1 : 2; };
  std::stable_sort(d.begin(), d.end(),
                   [&](const CholDesc& x, const CholDesc& y) { return kind(x) < kind(y); });
  groups.clear();
  single.clear();
  for (int i = 0; i < (int)d.size();) {
    const int k = kind(d[i]);
    int j = i, kamax = 0;
    while (j < (int)d.size() && kind(d[j]) == k) kamax = std::max(kamax, d[j++].ka);
    BatchGroup gr{k, i, j - i, 0, 0, 0};
    if (k == 0) {
      gr.param = chol_rt_shape(kamax);
      for (int q = i; q < j; ++q) gr.smem = std::max(gr.smem, chol_rt_smem(d[q].ka, gr.param));
    } else {
      gr.smem = chol_nt_base(kamax) + (k == 1 ? sizeof(float) * (size_t)kamax * kamax : 0);
    }
    groups.push_back(gr);
    i = j;
  }
}

cudaError_t chol_batch_launch(cudaStream_t st, const CholDesc* dtab,
                              const std::vector<BatchGroup>& groups) {
  for (const BatchGroup& g : groups) {
    if (g.count <= 0) continue;
    const CholDesc* t = dtab + g.first;
    cudaError_t e = cudaSuccess;
    ProfScope ps(st, "chol_inv");
    if (g.kind == 0) {
      auto kern = g.param == 0 ? k_chol_inv_rt_b<8, 4>
                  : g.param == 1 ? k_chol_inv_rt_b<12, 6> : k_chol_inv_rt_b<16, 8>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
      if (e == cudaSuccess) kern<<<g.count, CR_NW * 32, g.smem, st>>>(t);
    } else {
      auto kern = g.kind == 1 ? k_chol_inv_b<true> : k_chol_inv_b<false>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
      if (e == cudaSuccess) kern<<<g.count, 512, g.smem, st>>>(t);
    }
    note_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Groups of the batched Rayleigh-Ritz solves (FP32): kind 0 = the register-resident kernel
// (param = RS of the group's largest m), kind 1 / 2 = the register-slot kernel of 1,024 threads
// with its working set in shared / global memory (m <= 160), kind 3 = the cluster
// tridiagonalization and the register-slot kernel in its external-input mode (160 < m <= 480).
// Larger m run one by one.  Wider register shapes only add zero slots: the same bits.
static int rr_rt_rs(int m) { return m <= 64 ? 2 : m <= 96 ? 3 : m <= 128 ? 4 : 5; }
static size_t rr_rt_bytes(int m, int K, int rs) { return sizeof(float) * rt_smem_floats(m, K, rs); }
static size_t rr_reg5_base(int m, int K) { return sizeof(float) * ((size_t)6 * m + 7 * (size_t)K + 3 * 32 + 8); }
static size_t rr_reg_big(int m, int K) {
  return sizeof(float) * ((size_t)m * (m + 16) + 4 * (size_t)m * K + (size_t)K * K);
}
static int rr_kind(int m, int K) {
  if (m <= 160 && rr_rt_bytes(m, K, rr_rt_rs(m)) <= 225 * 1024) return 0;
  if (m <= 160) return rr_reg5_base(m, K) + rr_reg_big(m, K) <= 220 * 1024 ? 1 : 2;
  if (m <= 480) return 3;
  return 4;
}
bool rr_batch_cluster(int m) { return m > 160 && m <= 480; }
size_t rr_batch_scratch(int m, int K) {
  const int k = rr_kind(m, K);
  return (k == 2 || k == 3) ? rr_reg_big(m, K) / sizeof(float) : 0;
}

void rr_batch_plan(std::vector<RrDesc>& d, std::vector<BatchGroup>& groups,
                   std::vector<int>& single) {
  std::vector<RrDesc> in = d;
  d.clear();
  groups.clear();
  single.clear();
  for (int k = 0; k < 4; ++k) {
    const int first = (int)d.size();
    int mmax = 0;
    for (const RrDesc& a : in)
      if (rr_kind(a.m, a.K) == k) mmax = std::max(mmax, a.m);
    BatchGroup gr{k, first, 0, 0, 0, 0};
    if (k == 0) gr.param = rr_rt_rs(mmax);
    for (const RrDesc& a : in) {
      if (rr_kind(a.m, a.K) != k) continue;
      size_t need = 0;
      if (k == 0) need = rr_rt_bytes(a.m, a.K, gr.param);
      else if (k == 1) need = rr_reg5_base(a.m, a.K) + rr_reg_big(a.m, a.K);
      else if (k == 2) need = rr_reg5_base(a.m, a.K);
      else need = sizeof(float) * ((size_t)6 * a.m + 7 * (size_t)a.K + 3 * 16 + 8);
      if (k == 0 && need > 225 * 1024) continue;  // does not fit the group's register shape
      gr.smem = std::max(gr.smem, need);
      gr.aux = std::max(gr.aux, a.K);
      d.push_back(a);
    }
    gr.count = (int)d.size() - first;
    if (gr.count > 0) {
      if (k == 3) gr.param = mmax;
      groups.push_back(gr);
    }
  }
  // the rest (m > 480, or a kernel shape the group's cannot hold) one by one, after the groups
  for (const RrDesc& a : in) {
    bool placed = false;
    for (const RrDesc& b : d) placed = placed || (b.theta == a.theta);
    if (!placed) {
      single.push_back((int)d.size());
      d.push_back(a);
    }
  }
}

cudaError_t rr_batch_launch(cudaStream_t st, const RrDesc* dtab,
                            const std::vector<BatchGroup>& groups) {
  for (const BatchGroup& g : groups) {
    if (g.count <= 0) continue;
    const RrDesc* t = dtab + g.first;
    cudaError_t e = cudaSuccess;
    if (g.kind == 3) {
      e = tridiag_cluster_batch(st, g.count, t, g.param);
      if (e != cudaSuccess) return e;
      ProfScope ps(st, "rr_eig");
      k_rr_eigvals_cta_b<<<dim3(g.aux, g.count), 32, 0, st>>>(t);
      note_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    ProfScope ps(st, "rr_eig");
    if (g.kind == 0) {
      auto kern = g.param == 2 ? k_rr_eig_rt_b<2>
                  : g.param == 3 ? k_rr_eig_rt_b<3>
                  : g.param == 4 ? k_rr_eig_rt_b<4> : k_rr_eig_rt_b<5>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
      if (e == cudaSuccess) kern<<<g.count, RT_NT, g.smem, st>>>(t);
    } else if (g.kind == 1 || g.kind == 2) {
      auto kern = g.kind == 1 ? k_rr_eig_reg_b<5, 32, true> : k_rr_eig_reg_b<5, 32, false>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
      if (e == cudaSuccess) kern<<<g.count, 32 * 32, g.smem, st>>>(t);
    } else {
      auto kern = k_rr_eig_reg_b<15, 16, false>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
      if (e == cudaSuccess) kern<<<g.count, 16 * 32, g.smem, st>>>(t);
      if (e == cudaSuccess) e = cudaGetLastError();
      note_launch();
      if (e == cudaSuccess) {
        k_rr_back_b<<<dim3(g.aux, g.count), 32, 0, st>>>(t);
      }
    }
    note_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t chol_inv<float>(cudaStream_t, Alloc&, int, const double*, int, float*,
                                     int*, double, int*, int, int*, int, int*, double, double);
template cudaError_t chol_inv<double>(cudaStream_t, Alloc&, int, const double*, int, double*,
                                      int*, double, int*, int, int*, int, int*, double, double);
template cudaError_t rr_eig<float>(cudaStream_t, Alloc&, int, int, const double*, int, double*,
                                   float*, int*, int*, int, int*);
template cudaError_t rr_eig<double>(cudaStream_t, Alloc&, int, int, const double*, int,
                                    double*, double*, int*, int*, int, int*);

}  // namespace sc

#ifdef SC_RR_PHASES
// Debug builds only: the clock64() marks of the last Rayleigh-Ritz launch (phase starts).
// out[0..7]: phase marks; out[8..11]: accumulated eigenvector sub-phase clocks (LU solves,
// Gram, factorization, transform) since the previous call, which clears them.
extern "C" int sc_debug_rr_phases(long long* out) {
  if (cudaMemcpyFromSymbol(out, sc::g_rr_phase, sizeof(long long) * 8) != cudaSuccess) return -6;
  if (cudaMemcpyFromSymbol(out + 8, sc::g_rr_inv, sizeof(long long) * 4) != cudaSuccess) return -6;
  long long z[4] = {0, 0, 0, 0};
  return cudaMemcpyToSymbol(sc::g_rr_inv, z, sizeof(z)) == cudaSuccess ? 0 : -6;
}
#endif
