// Householder tridiagonalization (Golub & Van Loan Alg. 8.3.1) of the Rayleigh-Ritz matrix of a
// wide LOBPCG block (Knyazev 2001; m = 3K up to 512) on a cluster of CL CTAs, FP32.
//
// One SM's registers cannot hold a 480 x 480 matrix, so the rows are spread over the cluster:
// warp h = 16 rank + w (128 in all) owns rows h + 128 r (r < 4); lane l owns columns l + 32 c
// (c < 16) of those rows, so each warp holds whole rows and the row dot products
// p_i = beta (A v)_i need no exchange.  Per step k (q = k / 32 a compile-time index of the
// unrolled outer loop; column slots c < q hold columns <= k only and drop out):
//  (a) the owners of column k write x_i (0 for i <= k) into the x vector of every CTA, and their
//      warp's partial sum of x_i^2 (i > k + 1) into every CTA's table of partials;
//      cluster barrier;
//  (b) every thread sums the partials in a fixed order, forms the reflector scalars and v on
//      its rows and columns;
//  (c) p_i on the owned rows; lane 0 of each warp writes p_i and the p_i v_i partial into every
//      CTA, and the owners of column k write the scaled reflector v_i = x_i / v0 (i > k + 1)
//      to row k of the reflector matrix in global memory; cluster barrier;
//  (d) w = p - (beta / 2)(p'v) v and the rank-2 update of the owned entries.
// Outputs: the diagonal d, off-diagonal e, beta of every reflector and the reflector rows, in
// the layout the single-CTA Rayleigh-Ritz kernel takes them for the eigenvalue, eigenvector and
// back-transformation phases.  Dropped basis columns (zero diagonal of G at i >= K) are lifted
// above the Gershgorin bound first, as in the single-CTA kernels.  The exchanges go through
// distributed shared memory; the cluster barrier orders them (release / acquire), and a final
// barrier keeps every CTA's shared memory alive until the others are done with it.
#include <algorithm>

#include "common.cuh"

namespace sc {
namespace {

constexpr int TC_CL = 8;        // CTAs per cluster
constexpr int TC_NW = 16;       // warps per CTA
constexpr int TC_RS = 4;        // row slots per warp
constexpr int TC_CS = 16;       // column slots per lane
constexpr int TC_NH = TC_CL * TC_NW;  // warps in the cluster (128): each owns whole rows
constexpr int TC_MMAX = TC_NH * TC_RS;  // 512

// A store into the shared memory of CTA t of the cluster (distributed shared memory).
__device__ __forceinline__ void st_remote(float* p, int t, float v) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(t));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v) : "memory");
}
__device__ __forceinline__ void st_remote(double* p, int t, double v) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p), ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(t));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
// FP64: the reciprocal estimate refined by two Newton steps r <- r + r (1 - x r) (within a few
// ulps; the correctly rounded __drcp_rn is a long instruction sequence at the FP64 rate)
__device__ __forceinline__ double rcp_rn(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  return fma(r, fma(-x, r, 1.0), r);
}
// Cluster-wide barrier; its release / acquire orders the distributed shared memory stores.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" :::
                   "memory");
}

template <typename T>
__device__ __forceinline__ T hw_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Ag[i][j] = 0.5 (G_ij + G_ji) in FP32 (i, j < m): the cluster kernel's input, read back row
// by row with coalesced loads.  The same buffer then receives the reflector rows; the cluster
// barrier after the load separates the two uses.
template <typename T>
__global__ void k_sym(int m, const double* __restrict__ G, int ldg, T* __restrict__ Ag, int lda) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)m * m;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    Ag[(long long)i * lda + j] = (T)(0.5 * (G[(long long)i * ldg + j] + G[(long long)j * ldg + i]));
  }
}

template <typename T, int RS, int CS>
__device__ __forceinline__ void k_tridiag_cl_body(int m_full, int K, const double* __restrict__ G,
                                                  int ldg, T* __restrict__ Ag, int lda,
                                                  T* __restrict__ d_out, T* __restrict__ e_out,
                                                  T* __restrict__ b_out, const int* pflag,
                                                  int mP) {
  constexpr int MMAX = TC_NH * RS;
  constexpr bool kF64 = sizeof(T) == 8;
  __shared__ T vsc[kF64 ? MMAX : 1];  // FP64: the scaled reflector v of the step
  __shared__ T sh_bet, sh_iv0, sh_kc;
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ T xs[MMAX];      // x of the current step (every row)
  __shared__ T pvec[MMAX];    // p of the current step (every row)
  __shared__ T rs2all[TC_NH];    // per-warp partial sums of x_i^2
  __shared__ T rpvall[TC_NH];    // per-warp partial sums of p_i v_i
  __shared__ T gmx[TC_CL];       // per-CTA Gershgorin partial maxima
  __shared__ T wmax[TC_NW];
  unsigned rank_u;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank_u));
  const int rank = (int)rank_u;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int h = rank * TC_NW + warp, cl = lane;  // warp h of the cluster, lane = column owner
  const int m = (pflag && *pflag == 0) ? m_full - mP : m_full;

  // ---- load (symmetrized), Gershgorin bound over the cluster, lift dropped columns
  T A[RS][CS];
  T gm = (T)0;
#pragma unroll
  for (int r = 0; r < RS; ++r) {
    const int i = h + TC_NH * r;
    T rs = (T)0;
#pragma unroll
    for (int c = 0; c < CS; ++c) {
      const int j = cl + 32 * c;
      T a = (T)0;
      if (i < m && j < m) a = Ag[(long long)i * lda + j];  // symmetrized FP32 copy of G
      A[r][c] = a;
      rs += fabs(a);
    }
    gm = fmax(gm, hw_sum(rs));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(FULL, gm, o));
  if (lane == 0) wmax[warp] = gm;
  __syncthreads();
  if (tid == 0) {
    T mx = (T)0;
    for (int w = 0; w < TC_NW; ++w) mx = fmax(mx, wmax[w]);
    for (int t = 0; t < TC_CL; ++t) st_remote(&gmx[rank], t, mx);
  }
  cluster_sync();
  {
    T big = (T)0;
    for (int t = 0; t < TC_CL; ++t) big = fmax(big, gmx[t]);
    big = big * (T)1.25 + (T)1;
#pragma unroll
    for (int r = 0; r < RS; ++r)
#pragma unroll
      for (int c = 0; c < CS; ++c) {
        const int i = h + TC_NH * r, j = cl + 32 * c;
        if (i == j && i >= K && i < m && G[(long long)i * ldg + i] == 0.0) A[r][c] = big;
      }
  }

  // ---- the Householder steps
  bool stop = false;
#pragma unroll
  for (int q = 0; q < CS; ++q) {
    if (stop) break;
    const int r0 = q >> 2;  // row slot r holds rows 128 r .. 128 r + 127, dead once k >= 128 r + 127
    for (int kw = 0; kw < 32; ++kw) {
      const int k = 32 * q + kw;
      if (k + 2 >= m) {
        stop = true;
        break;
      }
      const int k1 = k + 1;
      // (a)
      if (cl == kw) {
        T s2 = (T)0;
#pragma unroll
        for (int r = 0; r < RS; ++r) {
          const int i = h + TC_NH * r;
          const T x = A[r][q];
          const T val = i > k ? x : (T)0;
          for (int t = 0; t < TC_CL; ++t) st_remote(&xs[i], t, val);
          s2 = fma(i > k1 ? x : (T)0, x, s2);
        }
        for (int t = 0; t < TC_CL; ++t) st_remote(&rs2all[h], t, s2);
        if (h == (k & (TC_NH - 1))) d_out[k] = A[q >> 2][q];
      }
      cluster_sync();
      // (b)
      T bet = (T)0, iv0 = (T)0;
      auto scalars = [&]() {
        T sg = (T)0;
#pragma unroll
        for (int j = 0; j < TC_NH / 32; ++j) sg += rs2all[lane + 32 * j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(FULL, sg, o);
        const T x0 = xs[k1];
        T ek = x0;
        if (sg != (T)0) {
          const T mu = sqrt(x0 * x0 + sg);
          const T v0 = x0 + copysign(mu, x0);
          iv0 = rcp_rn(v0);
          bet = (T)2 * rcp_rn((T)1 + sg * iv0 * iv0);
          ek = -copysign(mu, x0);
        }
        if (rank == 0 && tid == 0) {
          e_out[k] = ek;
          b_out[k] = bet;
        }
      };
      if constexpr (kF64) {
        // FP64 runs at 2 FMA per clock per SM: warp 0 forms the reflector scalars and the
        // scaled v once for the CTA instead of every thread doing so
        if (warp == 0) {
          scalars();
          if (lane == 0) {
            sh_bet = bet;
            sh_iv0 = iv0;
          }
          for (int i = lane; i < MMAX; i += 32) vsc[i] = i == k1 ? (T)1 : xs[i] * iv0;
        }
        __syncthreads();
        bet = sh_bet;
        iv0 = sh_iv0;
      } else {
        scalars();
      }
      // v on the owned columns is re-read from xs where it is needed (registers hold A)
      auto vcol = [&](int c) {
        if constexpr (kF64) return vsc[cl + 32 * c];
        const T v = xs[cl + 32 * c] * iv0;
        return (c <= q + 1 && cl + 32 * c == k1) ? (T)1 : v;
      };
      T vr[RS], pr[RS];
#pragma unroll
      for (int r = 0; r < RS; ++r) {
        const int i = h + TC_NH * r;
        if constexpr (kF64) vr[r] = vsc[i];
        else vr[r] = i == k1 ? (T)1 : xs[i] * iv0;
      }
      // (c)
      T sacc[RS];
#pragma unroll
      for (int r = 0; r < RS; ++r) sacc[r] = (T)0;
#pragma unroll
      for (int c = q; c < CS; ++c) {
        const T vc = vcol(c);
#pragma unroll
        for (int r = r0; r < RS; ++r)
          if (h + TC_NH * r < m) sacc[r] = fma(A[r][c], vc, sacc[r]);  // rows >= m stay zero
      }
      T pvp = (T)0;
#pragma unroll
      for (int r = r0; r < RS; ++r) {
        pr[r] = bet * hw_sum(sacc[r]);
        pvp = fma(pr[r], vr[r], pvp);
      }
      if (cl == 0) {
#pragma unroll
        for (int r = r0; r < RS; ++r)
          for (int t = 0; t < TC_CL; ++t) st_remote(&pvec[h + TC_NH * r], t, pr[r]);
        for (int t = 0; t < TC_CL; ++t) st_remote(&rpvall[h], t, pvp);
      }
      if (cl == kw) {
        // the scaled reflector: row k of Ag holds v_i for i > k + 1 (v_{k+1} = 1 is implied)
#pragma unroll
        for (int r = r0; r < RS; ++r) {
          const int i = h + TC_NH * r;
          if (i > k1 && i < m) Ag[(long long)k * lda + i] = A[r][q] * iv0;
        }
      }
      cluster_sync();
      // (d)
      auto pvsum = [&]() {
        T pv = (T)0;
#pragma unroll
        for (int j = 0; j < TC_NH / 32; ++j) pv += rpvall[lane + 32 * j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(FULL, pv, o);
        return bet * (T)0.5 * pv;
      };
      T kc;
      if constexpr (kF64) {
        if (warp == 0) {
          const T t = pvsum();
          if (lane == 0) sh_kc = t;
        }
        __syncthreads();
        kc = sh_kc;
      } else {
        kc = pvsum();
      }
      T wr[RS];
#pragma unroll
      for (int r = r0; r < RS; ++r) wr[r] = fma(-kc, vr[r], pr[r]);
#pragma unroll
      for (int c = q; c < CS; ++c) {
        const T vc = vcol(c);
        const T wj = fma(-kc, vc, pvec[cl + 32 * c]);
#pragma unroll
        for (int r = r0; r < RS; ++r)
          if (h + TC_NH * r < m) A[r][c] = fma(-vr[r], wj, fma(-wr[r], vc, A[r][c]));
      }
    }
  }
  // the trailing 2 x 2 block of T (or the 1 x 1 matrix), from the owners of its entries
#pragma unroll
  for (int r = 0; r < RS; ++r)
#pragma unroll
    for (int c = 0; c < CS; ++c) {
      const int i = h + TC_NH * r, j = cl + 32 * c;
      if (m >= 2) {
        if (i == m - 2 && j == m - 2) d_out[m - 2] = A[r][c];
        if (i == m - 1 && j == m - 2) e_out[m - 2] = A[r][c];
        if (i == m - 1 && j == m - 1) d_out[m - 1] = A[r][c];
      } else if (i == 0 && j == 0) {
        d_out[0] = A[r][c];
      }
    }
  if (rank == 0 && tid == 0 && m >= 1) e_out[m - 1] = (T)0;
  cluster_sync();  // no CTA leaves while another may still touch its shared memory
}

// FP32 for m <= 512 (4 row slots, 16 column slots); FP64 for m <= 256 (2 and 8: the FP64
// entries take two registers each).
template <typename T, int RS, int CS>
__global__ void __launch_bounds__(TC_NW * 32, 1)
    k_tridiag_cl(int m_full, int K, const double* __restrict__ G, int ldg, T* __restrict__ Ag,
                 int lda, T* __restrict__ d_out, T* __restrict__ e_out, T* __restrict__ b_out,
                 const int* pflag, int mP) {
  k_tridiag_cl_body<T, RS, CS>(m_full, K, G, ldg, Ag, lda, d_out, e_out, b_out, pflag, mP);
}

// Lockstep batch: cluster c of the grid (TC_CL CTAs) tridiagonalizes descriptor c's matrix;
// the reflector rows go to its Ag (stride m), d, e, beta to its tri.
__global__ void __launch_bounds__(TC_NW * 32, 1) k_tridiag_cl_b(const RrDesc* __restrict__ tab) {
  const RrDesc a = tab[blockIdx.x / TC_CL];
  k_tridiag_cl_body<float, TC_RS, TC_CS>(a.m, a.K, a.G, a.ldg, a.Ag, a.m, a.tri, a.tri + a.m,
                                         a.tri + 2 * a.m, a.pflag, a.mP);
}

// Lockstep batch: blockIdx.y = descriptor; its symmetrized FP32 matrix into Ag (stride m).
__global__ void k_sym_f32_b(const RrDesc* __restrict__ tab) {
  const RrDesc a = tab[blockIdx.y];
  const int m = a.m;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)m * m;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    a.Ag[(long long)i * m + j] =
        (float)(0.5 * (a.G[(long long)i * a.ldg + j] + a.G[(long long)j * a.ldg + i]));
  }
}

}  // namespace

// Tridiagonalization of the symmetric m x m FP64 matrix G (symmetrized on the fly) on one
// cluster of 8 CTAs, in the arithmetic of T (FP32: m <= 512; FP64: m <= 256): d, e (m each),
// beta (m) and the scaled reflectors in rows 0 .. m - 3 of Ag (row stride lda), as the
// register-slot Rayleigh-Ritz kernel takes them in its external-input mode.
template <typename T>
static cudaError_t tridiag_cluster_t(cudaStream_t st, int m, int K, const double* G, int ldg,
                                     T* Ag, int lda, T* d, T* e, T* beta, const int* pflag,
                                     int mP) {
  constexpr bool f32 = sizeof(T) == 4;
  if (m < 1 || m > (f32 ? TC_NH * TC_RS : TC_NH * 2)) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(TC_CL, 1, 1);
  cfg.blockDim = dim3(TC_NW * 32, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = TC_CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ProfScope ps(st, "rr_eig");
  k_sym<T><<<(unsigned)std::min<long long>(((long long)m * m + 255) / 256, 1024), 256, 0, st>>>(
      m, G, ldg, Ag, lda);
  note_launch();
  cudaError_t e0 = cudaGetLastError();
  if (e0 != cudaSuccess) return e0;
  if constexpr (f32)
    e0 = cudaLaunchKernelEx(&cfg, k_tridiag_cl<float, TC_RS, TC_CS>, m, K, G, ldg, Ag, lda, d, e,
                            beta, pflag, mP);
  else if (m <= 160)  // FP64 pays for every column slot: the narrowest shape that holds m
    e0 = cudaLaunchKernelEx(&cfg, k_tridiag_cl<double, 2, 5>, m, K, G, ldg, Ag, lda, d, e, beta,
                            pflag, mP);
  else
    e0 = cudaLaunchKernelEx(&cfg, k_tridiag_cl<double, 2, 8>, m, K, G, ldg, Ag, lda, d, e, beta,
                            pflag, mP);
  note_launch();
  return e0;
}

cudaError_t tridiag_cluster(cudaStream_t st, int m, int K, const double* G, int ldg, float* Ag,
                            int lda, float* d, float* e, float* beta, const int* pflag, int mP) {
  return tridiag_cluster_t<float>(st, m, K, G, ldg, Ag, lda, d, e, beta, pflag, mP);
}
cudaError_t tridiag_cluster(cudaStream_t st, int m, int K, const double* G, int ldg, double* Ag,
                            int lda, double* d, double* e, double* beta, const int* pflag, int mP) {
  return tridiag_cluster_t<double>(st, m, K, G, ldg, Ag, lda, d, e, beta, pflag, mP);
}

// The same for every descriptor of a lockstep batch (m <= mmax <= 512 each): one launch of
// the symmetrization, one of count clusters.
cudaError_t tridiag_cluster_batch(cudaStream_t st, int count, const RrDesc* dtab, int mmax) {
  if (count <= 0) return cudaSuccess;
  if (mmax < 1 || mmax > TC_MMAX) return cudaErrorInvalidValue;
  ProfScope ps(st, "rr_eig");
  const unsigned bx = (unsigned)std::min<long long>(((long long)mmax * mmax + 255) / 256, 256);
  k_sym_f32_b<<<dim3(bx, (unsigned)count), 256, 0, st>>>(dtab);
  note_launch();
  cudaError_t e0 = cudaGetLastError();
  if (e0 != cudaSuccess) return e0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(TC_CL * (unsigned)count, 1, 1);
  cfg.blockDim = dim3(TC_NW * 32, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = TC_CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e0 = cudaLaunchKernelEx(&cfg, k_tridiag_cl_b, dtab);
  note_launch();
  return e0;
}

}  // namespace sc
