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
// Cluster-wide barrier; its release / acquire orders the distributed shared memory stores.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" :::
                   "memory");
}

__device__ __forceinline__ float hw_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Ag[i][j] = 0.5 (G_ij + G_ji) in FP32 (i, j < m): the cluster kernel's input, read back row
// by row with coalesced loads.  The same buffer then receives the reflector rows; the cluster
// barrier after the load separates the two uses.
__global__ void k_sym_f32(int m, const double* __restrict__ G, int ldg, float* __restrict__ Ag,
                          int lda) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)m * m;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    Ag[(long long)i * lda + j] = (float)(0.5 * (G[(long long)i * ldg + j] + G[(long long)j * ldg + i]));
  }
}

__device__ __forceinline__ void k_tridiag_cl_body(int m_full, int K, const double* __restrict__ G,
                                                  int ldg, float* __restrict__ Ag, int lda,
                                                  float* __restrict__ d_out,
                                                  float* __restrict__ e_out,
                                                  float* __restrict__ b_out, const int* pflag,
                                                  int mP) {
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ float xs[TC_MMAX];      // x of the current step (every row)
  __shared__ float pvec[TC_MMAX];    // p of the current step (every row)
  __shared__ float rs2all[TC_NH];    // per-warp partial sums of x_i^2
  __shared__ float rpvall[TC_NH];    // per-warp partial sums of p_i v_i
  __shared__ float gmx[TC_CL];       // per-CTA Gershgorin partial maxima
  __shared__ float wmax[TC_NW];
  unsigned rank_u;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank_u));
  const int rank = (int)rank_u;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int h = rank * TC_NW + warp, cl = lane;  // warp h of the cluster, lane = column owner
  const int m = (pflag && *pflag == 0) ? m_full - mP : m_full;

  // ---- load (symmetrized), Gershgorin bound over the cluster, lift dropped columns
  float A[TC_RS][TC_CS];
  float gm = 0.f;
#pragma unroll
  for (int r = 0; r < TC_RS; ++r) {
    const int i = h + TC_NH * r;
    float rs = 0.f;
#pragma unroll
    for (int c = 0; c < TC_CS; ++c) {
      const int j = cl + 32 * c;
      float a = 0.f;
      if (i < m && j < m) a = Ag[(long long)i * lda + j];  // symmetrized FP32 copy of G
      A[r][c] = a;
      rs += fabsf(a);
    }
    gm = fmaxf(gm, hw_sum(rs));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(FULL, gm, o));
  if (lane == 0) wmax[warp] = gm;
  __syncthreads();
  if (tid == 0) {
    float mx = 0.f;
    for (int w = 0; w < TC_NW; ++w) mx = fmaxf(mx, wmax[w]);
    for (int t = 0; t < TC_CL; ++t) st_remote(&gmx[rank], t, mx);
  }
  cluster_sync();
  {
    float big = 0.f;
    for (int t = 0; t < TC_CL; ++t) big = fmaxf(big, gmx[t]);
    big = big * 1.25f + 1.f;
#pragma unroll
    for (int r = 0; r < TC_RS; ++r)
#pragma unroll
      for (int c = 0; c < TC_CS; ++c) {
        const int i = h + TC_NH * r, j = cl + 32 * c;
        if (i == j && i >= K && i < m && G[(long long)i * ldg + i] == 0.0) A[r][c] = big;
      }
  }

  // ---- the Householder steps
  bool stop = false;
#pragma unroll
  for (int q = 0; q < TC_CS; ++q) {
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
        float s2 = 0.f;
#pragma unroll
        for (int r = 0; r < TC_RS; ++r) {
          const int i = h + TC_NH * r;
          const float x = A[r][q];
          const float val = i > k ? x : 0.f;
          for (int t = 0; t < TC_CL; ++t) st_remote(&xs[i], t, val);
          s2 = fmaf(i > k1 ? x : 0.f, x, s2);
        }
        for (int t = 0; t < TC_CL; ++t) st_remote(&rs2all[h], t, s2);
        if (h == (k & (TC_NH - 1))) d_out[k] = A[q >> 2][q];
      }
      cluster_sync();
      // (b)
      float sg = 0.f;
#pragma unroll
      for (int j = 0; j < TC_NH / 32; ++j) sg += rs2all[lane + 32 * j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(FULL, sg, o);
      const float x0 = xs[k1];
      float bet = 0.f, iv0 = 0.f, ek = x0;
      if (sg != 0.f) {
        const float mu = sqrtf(x0 * x0 + sg);
        const float v0 = x0 + copysignf(mu, x0);
        iv0 = __frcp_rn(v0);
        bet = 2.f * __frcp_rn(1.f + sg * iv0 * iv0);
        ek = -copysignf(mu, x0);
      }
      if (rank == 0 && tid == 0) {
        e_out[k] = ek;
        b_out[k] = bet;
      }
      // v on the owned columns is re-read from xs where it is needed (registers hold A)
      auto vcol = [&](int c) {
        const float v = xs[cl + 32 * c] * iv0;
        return (c <= q + 1 && cl + 32 * c == k1) ? 1.f : v;
      };
      float vr[TC_RS], pr[TC_RS];
#pragma unroll
      for (int r = 0; r < TC_RS; ++r) {
        const int i = h + TC_NH * r;
        vr[r] = i == k1 ? 1.f : xs[i] * iv0;
      }
      // (c)
      float sacc[TC_RS];
#pragma unroll
      for (int r = 0; r < TC_RS; ++r) sacc[r] = 0.f;
#pragma unroll
      for (int c = q; c < TC_CS; ++c) {
        const float vc = vcol(c);
#pragma unroll
        for (int r = r0; r < TC_RS; ++r) sacc[r] = fmaf(A[r][c], vc, sacc[r]);
      }
      float pvp = 0.f;
#pragma unroll
      for (int r = r0; r < TC_RS; ++r) {
        pr[r] = bet * hw_sum(sacc[r]);
        pvp = fmaf(pr[r], vr[r], pvp);
      }
      if (cl == 0) {
#pragma unroll
        for (int r = r0; r < TC_RS; ++r)
          for (int t = 0; t < TC_CL; ++t) st_remote(&pvec[h + TC_NH * r], t, pr[r]);
        for (int t = 0; t < TC_CL; ++t) st_remote(&rpvall[h], t, pvp);
      }
      if (cl == kw) {
        // the scaled reflector: row k of Ag holds v_i for i > k + 1 (v_{k+1} = 1 is implied)
#pragma unroll
        for (int r = r0; r < TC_RS; ++r) {
          const int i = h + TC_NH * r;
          if (i > k1 && i < m) Ag[(long long)k * lda + i] = A[r][q] * iv0;
        }
      }
      cluster_sync();
      // (d)
      float pv = 0.f;
#pragma unroll
      for (int j = 0; j < TC_NH / 32; ++j) pv += rpvall[lane + 32 * j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(FULL, pv, o);
      const float kc = bet * 0.5f * pv;
      float wr[TC_RS];
#pragma unroll
      for (int r = r0; r < TC_RS; ++r) wr[r] = fmaf(-kc, vr[r], pr[r]);
#pragma unroll
      for (int c = q; c < TC_CS; ++c) {
        const float vc = vcol(c);
        const float wj = fmaf(-kc, vc, pvec[cl + 32 * c]);
#pragma unroll
        for (int r = r0; r < TC_RS; ++r) A[r][c] = fmaf(-vr[r], wj, fmaf(-wr[r], vc, A[r][c]));
      }
    }
  }
  // the trailing 2 x 2 block of T (or the 1 x 1 matrix), from the owners of its entries
#pragma unroll
  for (int r = 0; r < TC_RS; ++r)
#pragma unroll
    for (int c = 0; c < TC_CS; ++c) {
      const int i = h + TC_NH * r, j = cl + 32 * c;
      if (m >= 2) {
        if (i == m - 2 && j == m - 2) d_out[m - 2] = A[r][c];
        if (i == m - 1 && j == m - 2) e_out[m - 2] = A[r][c];
        if (i == m - 1 && j == m - 1) d_out[m - 1] = A[r][c];
      } else if (i == 0 && j == 0) {
        d_out[0] = A[r][c];
      }
    }
  if (rank == 0 && tid == 0 && m >= 1) e_out[m - 1] = 0.f;
  cluster_sync();  // no CTA leaves while another may still touch its shared memory
}

__global__ void __launch_bounds__(TC_NW * 32, 1)
    k_tridiag_cl(int m_full, int K, const double* __restrict__ G, int ldg, float* __restrict__ Ag,
                 int lda, float* __restrict__ d_out, float* __restrict__ e_out,
                 float* __restrict__ b_out, const int* pflag, int mP) {
  k_tridiag_cl_body(m_full, K, G, ldg, Ag, lda, d_out, e_out, b_out, pflag, mP);
}

// Lockstep batch: cluster c of the grid (TC_CL CTAs) tridiagonalizes descriptor c's matrix;
// the reflector rows go to its Ag (stride m), d, e, beta to its tri.
__global__ void __launch_bounds__(TC_NW * 32, 1) k_tridiag_cl_b(const RrDesc* __restrict__ tab) {
  const RrDesc a = tab[blockIdx.x / TC_CL];
  k_tridiag_cl_body(a.m, a.K, a.G, a.ldg, a.Ag, a.m, a.tri, a.tri + a.m, a.tri + 2 * a.m,
                    a.pflag, a.mP);
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

// Tridiagonalization of the symmetric m x m FP64 matrix G (m <= 512, symmetrized on the fly) on
// one cluster of 8 CTAs: d, e (m floats each), beta (m) and the scaled reflectors in rows
// 0 .. m - 3 of Ag (row stride lda), as the single-CTA Rayleigh-Ritz kernel expects them.
cudaError_t tridiag_cluster(cudaStream_t st, int m, int K, const double* G, int ldg, float* Ag,
                            int lda, float* d, float* e, float* beta, const int* pflag, int mP) {
  if (m < 1 || m > TC_MMAX) return cudaErrorInvalidValue;
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
  k_sym_f32<<<(unsigned)std::min<long long>(((long long)m * m + 255) / 256, 1024), 256, 0, st>>>(
      m, G, ldg, Ag, lda);
  note_launch();
  cudaError_t e0 = cudaGetLastError();
  if (e0 != cudaSuccess) return e0;
  e0 = cudaLaunchKernelEx(&cfg, k_tridiag_cl, m, K, G, ldg, Ag, lda, d, e, beta, pflag, mP);
  note_launch();
  return e0;
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
