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

constexpr int NT = 1024;

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
// Cholesky-QR transform (FP64).  W is ka x ka FP64 workspace (shared or global).
template <typename T>
__global__ void __launch_bounds__(NT)
    k_chol_inv(int ka, const double* __restrict__ G, int ldg, T* __restrict__ Tm,
               double* Wg, int in_smem, int* status, double pivot_tol) {
  extern __shared__ __align__(16) double dsm[];
  double* s = dsm;                 // ka scale factors
  double* red = s + ka;            // 34
  double* W = in_smem ? red + 34 : Wg;
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < ka; i += blockDim.x) {
    double d = G[(long long)i * ldg + i];
    s[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    if (!(d > 0.0)) fail = 1;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ka * ka; idx += blockDim.x) {
    int i = idx / ka, j = idx % ka;
    double g = 0.5 * (G[(long long)i * ldg + j] + G[(long long)j * ldg + i]);
    W[idx] = g * s[i] * s[j];
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle in place
  for (int k = 0; k < ka && !fail; ++k) {
    double piv = W[k * ka + k];
    if (!(piv > pivot_tol)) {
      __syncthreads();
      if (threadIdx.x == 0) fail = 1;
      __syncthreads();
      break;
    }
    double ck = sqrt(piv);
    for (int i = k + 1 + threadIdx.x; i < ka; i += blockDim.x) W[i * ka + k] /= ck;
    __syncthreads();
    if (threadIdx.x == 0) W[k * ka + k] = ck;
    int nr = ka - k - 1;
    for (int idx = threadIdx.x; idx < nr * nr; idx += blockDim.x) {
      int i = k + 1 + idx / nr, j = k + 1 + idx % nr;
      if (j <= i) W[i * ka + j] -= W[i * ka + k] * W[j * ka + k];
    }
    __syncthreads();
  }
  if (fail) {
    if (threadIdx.x == 0) atomicOr(status, ST_CHOL_FAIL);
    return;
  }
  // inverse of the lower factor, column j by thread j (forward substitution), stored in
  // the strict upper triangle transposed: U[j][i] = Linv[i][j] for i >= j.
  for (int j = threadIdx.x; j < ka; j += blockDim.x) {
    // Linv[j][j]
    double xj = 1.0 / W[j * ka + j];
    Tm[(long long)j * ka + j] = (T)(s[j] * xj);
    // x_i for i > j go to the (free) strict upper triangle: W[j][i] = Linv[i][j]
    for (int i = j + 1; i < ka; ++i) {
      double acc = W[i * ka + j] * xj;
      for (int q = j + 1; q < i; ++q) acc += W[i * ka + q] * W[j * ka + q];
      double xi = -acc / W[i * ka + i];
      W[j * ka + i] = xi;  // strictly upper part is free (lower holds C)
    }
  }
  __syncthreads();
  // Tm[i][j] = s_i * (C^-1)[j][i] for j >= i  (C^-1 stored as W[col][row] above diagonal)
  for (int idx = threadIdx.x; idx < ka * ka; idx += blockDim.x) {
    int i = idx / ka, j = idx % ka;
    T v = 0;
    if (j > i) v = (T)(s[i] * W[i * ka + j]);
    if (j != i) Tm[(long long)i * ka + j] = v;
  }
}

// ---------------------------------------------------------------------------------------
template <typename T>
__device__ int sturm_count(int m, const T* d, const T* e2, T x, T pivmin) {
  int c = 0;
  T q = d[0] - x;
  if (fabs(q) <= pivmin) q = -pivmin;
  if (q <= 0) ++c;
  for (int i = 1; i < m; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) <= pivmin) q = -pivmin;
    if (q <= 0) ++c;
  }
  return c;
}

// Pseudo-random start entries in (-1, 1) for inverse iteration (SplitMix64 output mix).
__device__ inline double start_entry(int i, int j) {
  unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(i * 7919 + j * 104729 + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

template <typename T>
__global__ void __launch_bounds__(NT)
    k_rr_eig(int m, int K, const double* __restrict__ G, int ldg, double* __restrict__ theta,
             T* __restrict__ Y, T* Ag, T* Zg, T* lu, int a_smem, int z_smem, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* d = (T*)smraw;
  T* e = d + m;
  T* beta = e + m;
  T* vv = beta + m;
  T* pv = vv + m;
  T* wv = pv + m;
  T* lam = wv + m;   // K
  T* red = lam + K;  // 64
  T* nxt = red + 64;
  T* A = a_smem ? nxt : Ag;
  if (a_smem) nxt += (long long)m * m;
  T* Z = z_smem ? nxt : Zg;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;

  for (int idx = tid; idx < m * m; idx += nt) {
    int i = idx / m, j = idx % m;
    A[idx] = (T)(0.5 * (G[(long long)i * ldg + j] + G[(long long)j * ldg + i]));
  }
  __syncthreads();

  // 1. Householder tridiagonalization; reflector k stored in row k, cols k+1..m-1 (v0 = 1)
  for (int k = 0; k + 2 < m; ++k) {
    const int n1 = m - k - 1;
    T* x = A + (long long)k * m + k + 1;
    T part = 0;
    for (int i = tid + 1; i < n1; i += nt) part += x[i] * x[i];
    T sigma = block_sum(part, red);
    if (tid == 0) {
      T x0 = x[0], bet, ek, v0 = 1;
      if (sigma == (T)0) {
        bet = 0;
        ek = x0;
      } else {
        T mu = sqrt(x0 * x0 + sigma);
        v0 = (x0 <= (T)0) ? x0 - mu : -sigma / (x0 + mu);
        bet = (T)2 * v0 * v0 / (sigma + v0 * v0);
        ek = mu;
      }
      beta[k] = bet;
      e[k] = ek;
      red[40] = v0;
    }
    __syncthreads();
    const T bet = beta[k];
    const T v0 = red[40];
    if (bet == (T)0) continue;  // uniform
    for (int i = tid; i < n1; i += nt) vv[i] = (i == 0) ? (T)1 : x[i] / v0;
    __syncthreads();
    for (int i = tid; i < n1; i += nt) x[i] = vv[i];
    // p = bet * A' v (A' symmetric trailing block; thread groups of g lanes per row)
    int g = 32;
    while (g > 1 && n1 * g > nt) g >>= 1;
    const int rows_pp = nt / g;
    for (int i0 = 0; i0 < n1; i0 += rows_pp) {
      int i = i0 + tid / g, sl = tid % g;
      T acc = 0;
      if (i < n1) {
        const T* col = A + (long long)(k + 1) * m + (k + 1 + i);
        for (int j = sl; j < n1; j += g) acc += col[(long long)j * m] * vv[j];
      }
      for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, g);
      if (i < n1 && sl == 0) pv[i] = bet * acc;
    }
    __syncthreads();
    part = 0;
    for (int i = tid; i < n1; i += nt) part += pv[i] * vv[i];
    T pdv = block_sum(part, red);
    T kc = bet * (T)0.5 * pdv;
    for (int i = tid; i < n1; i += nt) wv[i] = pv[i] - kc * vv[i];
    __syncthreads();
    const long long tot = (long long)n1 * n1;
    for (long long idx = tid; idx < tot; idx += nt) {
      int i = (int)(idx / n1), j = (int)(idx % n1);
      T* a = A + (long long)(k + 1 + i) * m + (k + 1 + j);
      *a -= vv[i] * wv[j] + wv[i] * vv[j];
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += nt) d[i] = A[(long long)i * m + i];
  if (tid == 0 && m >= 2) {
    e[m - 2] = A[(long long)(m - 1) * m + (m - 2)];
    if (m - 2 >= 0) beta[m - 2] = 0;
  }
  if (tid == 0) e[m - 1] = 0;
  __syncthreads();

  // 2. Gershgorin bounds and multisection for eigenvalues 0..K-1
  T* e2 = wv;
  T lo_p = (T)3e38, hi_p = (T)-3e38, emax = 0;
  for (int i = tid; i < m; i += nt) {
    T r = fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : (T)0);
    lo_p = min(lo_p, d[i] - r);
    hi_p = max(hi_p, d[i] + r);
    emax = max(emax, e[i] * e[i]);
    if (!isfinite(d[i]) || !isfinite(e[i])) atomicOr(status, ST_NONFINITE);
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) e2[i] = e[i] * e[i];
  T lo = -block_max(-lo_p, red);
  T hi = block_max(hi_p, red);
  emax = block_max(emax, red);
  const T tnorm = max(fabs(lo), fabs(hi));
  const T pivmin = Lim<T>::tiny() * max((T)1, emax);
  lo -= (T)2 * Lim<T>::eps() * tnorm + pivmin;
  hi += (T)2 * Lim<T>::eps() * tnorm + pivmin;
  for (int j = warp; j < K; j += nt / 32) {
    T a = lo, b = hi;
    for (int it = 0; it < 40; ++it) {
      T tol = (T)2 * Lim<T>::eps() * max(fabs(a), fabs(b)) + (T)4 * pivmin;
      if (b - a <= tol) break;
      T h = (b - a) / (T)33;
      T xq = a + h * (T)(lane + 1);
      int c = sturm_count(m, d, e2, xq, pivmin);
      unsigned bal = __ballot_sync(0xffffffffu, c > j);
      int first = bal ? (__ffs(bal) - 1) : 32;
      T na = first == 0 ? a : a + h * (T)first;
      T nb = first == 32 ? b : a + h * (T)(first + 1);
      if (!(nb > na)) break;
      a = na;
      b = nb;
    }
    if (lane == 0) lam[j] = (T)0.5 * (a + b);
  }
  __syncthreads();

  // 3. inverse iteration: shifts separated by sep, LU of (T - s I) per eigenvalue
  const T sep = (T)10 * Lim<T>::eps() * tnorm + pivmin;
  T* shift = pv;  // K <= m
  if (tid == 0) {
    T prev = (T)0;
    for (int j = 0; j < K; ++j) {
      T s = lam[j];
      if (j > 0 && s < prev + sep) s = prev + sep;
      shift[j] = s;
      prev = s;
    }
  }
  __syncthreads();
  const T small_piv = Lim<T>::eps() * tnorm + pivmin;
  for (int j = tid; j < K; j += nt) {
    T* u0 = lu + (long long)j * 5 * m;
    T* u1 = u0 + m;
    T* u2 = u1 + m;
    T* ml = u2 + m;
    T* sw = ml + m;  // 1 = rows i, i+1 swapped
    T s = shift[j];
    T al = d[0] - s, bt = m > 1 ? e[0] : (T)0;
    for (int i = 0; i + 1 < m; ++i) {
      T dl = e[i];                                   // (i+1, i)
      T an = d[i + 1] - s, bn = (i + 2 < m) ? e[i + 1] : (T)0;  // row i+1: diag, super
      if (fabs(al) >= fabs(dl)) {
        if (al == (T)0) al = small_piv;
        T mlt = dl / al;
        u0[i] = al; u1[i] = bt; u2[i] = 0; ml[i] = mlt; sw[i] = 0;
        al = an - mlt * bt;
        bt = bn;
      } else {
        T mlt = al / dl;
        u0[i] = dl; u1[i] = an; u2[i] = bn; ml[i] = mlt; sw[i] = 1;
        al = bt - mlt * an;
        bt = -mlt * bn;
      }
    }
    if (fabs(al) < small_piv) al = al < (T)0 ? -small_piv : small_piv;
    u0[m - 1] = al;
    u1[m - 1] = 0;
    u2[m - 1] = 0;
    ml[m - 1] = 0;
    sw[m - 1] = 0;
    for (int i = 0; i < m; ++i) Z[(long long)i * K + j] = (T)start_entry(i, j);
  }
  __syncthreads();
  for (int sweep = 0; sweep < 2; ++sweep) {
    for (int j = tid; j < K; j += nt) {
      const T* u0 = lu + (long long)j * 5 * m;
      const T* u1 = u0 + m;
      const T* u2 = u1 + m;
      const T* ml = u2 + m;
      const T* sw = ml + m;
      // forward: apply row swaps and multipliers
      for (int i = 0; i + 1 < m; ++i) {
        T bi = Z[(long long)i * K + j], bn = Z[(long long)(i + 1) * K + j];
        if (sw[i] != (T)0) {
          T t = bi; bi = bn; bn = t;
        }
        Z[(long long)i * K + j] = bi;
        Z[(long long)(i + 1) * K + j] = bn - ml[i] * bi;
      }
      // back substitution with U (diag u0, super u1, second super u2)
      T z1 = 0, z2 = 0, mx = 0;
      for (int i = m - 1; i >= 0; --i) {
        T zi = (Z[(long long)i * K + j] - u1[i] * z1 - u2[i] * z2) / u0[i];
        Z[(long long)i * K + j] = zi;
        z2 = z1;
        z1 = zi;
        mx = max(mx, fabs(zi));
      }
      T inv = mx > (T)0 ? (T)1 / mx : (T)1;
      for (int i = 0; i < m; ++i) Z[(long long)i * K + j] *= inv;
    }
    __syncthreads();
    // classical Gram-Schmidt twice per column, in eigenvalue order, then normalize
    T* coef = vv;  // K <= m
    for (int j = 0; j < K; ++j) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int q = warp; q < j; q += nt / 32) {
          T acc = 0;
          for (int i = lane; i < m; i += 32) acc += Z[(long long)i * K + q] * Z[(long long)i * K + j];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) coef[q] = acc;
        }
        __syncthreads();
        if (j > 0) {
          for (int i = tid; i < m; i += nt) {
            T acc = 0;
            for (int q = 0; q < j; ++q) acc += coef[q] * Z[(long long)i * K + q];
            Z[(long long)i * K + j] -= acc;
          }
        }
        __syncthreads();
      }
      T part = 0;
      for (int i = tid; i < m; i += nt) {
        T z = Z[(long long)i * K + j];
        part += z * z;
      }
      T nrm2 = block_sum(part, red);
      T inv = nrm2 > (T)0 ? (T)1 / sqrt(nrm2) : (T)0;
      for (int i = tid; i < m; i += nt) Z[(long long)i * K + j] *= inv;
      __syncthreads();
    }
  }

  // 4. back-transformation Z <- H_0 ... H_{m-3} Z
  T* coef = vv;
  for (int k = m - 3; k >= 0; --k) {
    const T bet = beta[k];
    if (bet == (T)0) continue;
    const int n1 = m - k - 1;
    const T* v = A + (long long)k * m + k + 1;
    for (int j = warp; j < K; j += nt / 32) {
      T acc = 0;
      for (int i = lane; i < n1; i += 32) acc += v[i] * Z[(long long)(k + 1 + i) * K + j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) coef[j] = bet * acc;
    }
    __syncthreads();
    const long long tot = (long long)n1 * K;
    for (long long idx = tid; idx < tot; idx += nt) {
      int i = (int)(idx / K), j = (int)(idx % K);
      Z[(long long)(k + 1 + i) * K + j] -= coef[j] * v[i];
    }
    __syncthreads();
  }
  for (int j = tid; j < K; j += nt) theta[j] = (double)lam[j];
  for (long long idx = tid; idx < (long long)m * K; idx += nt) Y[idx] = Z[idx];
}

}  // namespace

template <typename T>
cudaError_t chol_inv(cudaStream_t st, Alloc& al, int ka, const double* G, int ldg, T* Tm,
                     int* d_status, double pivot_tol) {
  size_t base = sizeof(double) * ((size_t)ka + 34);
  size_t wbytes = sizeof(double) * (size_t)ka * ka;
  int in_smem = base + wbytes <= 200 * 1024;
  size_t sm = base + (in_smem ? wbytes : 0);
  double* Wg = nullptr;
  if (!in_smem) {
    Wg = al.get<double>((size_t)ka * ka);
    if (!Wg) return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaFuncSetAttribute(k_chol_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  ProfScope ps(st, "chol_inv");
  k_chol_inv<T><<<1, NT, sm, st>>>(ka, G, ldg, Tm, Wg, in_smem, d_status, pivot_tol);
  note_launch();
  e = cudaGetLastError();
  al.put(Wg);
  return e;
}

template <typename T>
cudaError_t rr_eig(cudaStream_t st, Alloc& al, int m, int K, const double* G, int ldg,
                   double* theta, T* Y, int* d_status) {
  if (m < 1 || K < 1 || K > m) return cudaErrorInvalidValue;
  size_t base = sizeof(T) * ((size_t)6 * m + K + 64);
  size_t abytes = sizeof(T) * (size_t)m * m;
  size_t zbytes = sizeof(T) * (size_t)m * K;
  const size_t cap = 220 * 1024;
  int a_smem = base + abytes <= cap;
  int z_smem = a_smem && base + abytes + zbytes <= cap;
  size_t sm = base + (a_smem ? abytes : 0) + (z_smem ? zbytes : 0);
  T* Ag = a_smem ? nullptr : al.get<T>((size_t)m * m);
  T* Zg = z_smem ? nullptr : al.get<T>((size_t)m * K);
  T* lu = al.get<T>((size_t)K * 5 * m);
  cudaError_t e = cudaSuccess;
  if ((!a_smem && !Ag) || (!z_smem && !Zg) || !lu) {
    e = cudaErrorMemoryAllocation;
  } else {
    e = cudaFuncSetAttribute(k_rr_eig<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
      ProfScope ps(st, "rr_eig");
      k_rr_eig<T><<<1, NT, sm, st>>>(m, K, G, ldg, theta, Y, Ag, Zg, lu, a_smem, z_smem,
                                     d_status);
      note_launch();
      e = cudaGetLastError();
    }
  }
  al.put(Ag);
  al.put(Zg);
  al.put(lu);
  return e;
}

template cudaError_t chol_inv<float>(cudaStream_t, Alloc&, int, const double*, int, float*,
                                     int*, double);
template cudaError_t chol_inv<double>(cudaStream_t, Alloc&, int, const double*, int, double*,
                                      int*, double);
template cudaError_t rr_eig<float>(cudaStream_t, Alloc&, int, int, const double*, int, double*,
                                   float*, int*);
template cudaError_t rr_eig<double>(cudaStream_t, Alloc&, int, int, const double*, int,
                                    double*, double*, int*);

}  // namespace sc
