// Cluster assignment by QR with column pivoting of the eigenvector block (Sec. II.A, the
// method of Damle, Minden & Ying that the paper names beside k-means++).  FP64 throughout:
//  1. Greedy column pivoting of Y' (K x n), i.e. of the rows of Y: K steps, each choosing
//     the row of the current residual with the largest norm (lowest index on ties), then
//     projecting every residual row off its direction.  Per step one grid kernel (projection,
//     fresh row norms, per-block argmax) and one single-CTA kernel (global argmax, the
//     normalized direction q).
//  2. Q = C (C'C)^-1/2, the polar factor of C = Y'[:, pivots], through the symmetric
//     eigensolver (C'C = W diag(theta) W').
//  3. label_i = argmax_j |(Y Q)_ij| (lowest j on ties), one thread per row.
#include <cuda_runtime.h>

#include <cfloat>
#include <climits>

#include "common.cuh"

namespace sc {
namespace {

constexpr int CB = 256;  // rows per block in the grid kernels

// Block argmax of (v, i) pairs: larger v wins, the lower index on equal v.
__device__ void block_argmax(double v, int i, int out_slot, double* gv, int* gi) {
  __shared__ double sv[CB / 32];
  __shared__ int si[CB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
  if (lane == 0) {
    sv[w] = v;
    si[w] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bvv = sv[0];
    int bii = si[0];
    for (int q = 1; q < CB / 32; ++q)
      if (sv[q] > bvv || (sv[q] == bvv && si[q] < bii)) {
        bvv = sv[q];
        bii = si[q];
      }
    gv[out_slot] = bvv;
    gi[out_slot] = bii;
  }
}

// Residual rows A = Y (FP64) and their squared norms; per-block argmax of the norms.
__global__ void __launch_bounds__(CB)
    k_cpqr_init(long long n, int K, const float* __restrict__ Y, long long ldy,
                double* __restrict__ A, double* __restrict__ nrm, double* bval, int* bidx) {
  const long long i = (long long)blockIdx.x * CB + threadIdx.x;
  double s = -1.0;
  if (i < n) {
    s = 0.0;
    for (int c = 0; c < K; ++c) {
      const double a = (double)Y[i * ldy + c];
      A[i * K + c] = a;
      s = fma(a, a, s);
    }
    nrm[i] = s;
  }
  block_argmax(s, i < n ? (int)i : INT_MAX, blockIdx.x, bval, bidx);
}

// Step t: the global argmax over the block partials is pivot t; q = its residual row,
// normalized (zero when the row is zero); the pivot row is retired (norm -1).
__global__ void __launch_bounds__(CB)
    k_cpqr_pick(int nb, const double* __restrict__ bval, const int* __restrict__ bidx,
                const double* __restrict__ A, int K, double* nrm, double* q, int* piv, int t) {
  __shared__ double sv[CB / 32];
  __shared__ int si[CB / 32];
  __shared__ int sj;
  double v = -2.0;
  int i = INT_MAX;
  for (int b = threadIdx.x; b < nb; b += CB) {
    const double bvv = bval[b];
    const int bii = bidx[b];
    if (bvv > v || (bvv == v && bii < i)) {
      v = bvv;
      i = bii;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
  if (lane == 0) {
    sv[w] = v;
    si[w] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bvv = sv[0];
    int bii = si[0];
    for (int qq = 1; qq < CB / 32; ++qq)
      if (sv[qq] > bvv || (sv[qq] == bvv && si[qq] < bii)) {
        bvv = sv[qq];
        bii = si[qq];
      }
    sj = bii;
    piv[t] = bii;
  }
  __syncthreads();
  const int j = sj;
  const double nj2 = nrm[j];
  const double inv = nj2 > 0.0 ? 1.0 / sqrt(nj2) : 0.0;
  for (int c = threadIdx.x; c < K; c += CB) q[c] = A[(long long)j * K + c] * inv;
  __syncthreads();
  if (threadIdx.x == 0) nrm[j] = -1.0;
}

// Project every live residual row off q, refresh its squared norm, per-block argmax.
__global__ void __launch_bounds__(CB)
    k_cpqr_proj(long long n, int K, double* __restrict__ A, double* __restrict__ nrm,
                const double* __restrict__ q, double* bval, int* bidx) {
  extern __shared__ double qs[];
  for (int c = threadIdx.x; c < K; c += CB) qs[c] = q[c];
  __syncthreads();
  const long long i = (long long)blockIdx.x * CB + threadIdx.x;
  double s = -1.0;
  if (i < n) {
    s = nrm[i];
    if (s >= 0.0) {
      double* a = A + i * K;
      double d = 0.0;
      for (int c = 0; c < K; ++c) d = fma(qs[c], a[c], d);
      s = 0.0;
      for (int c = 0; c < K; ++c) {
        const double v = fma(-d, qs[c], a[c]);
        a[c] = v;
        s = fma(v, v, s);
      }
      nrm[i] = s;
    }
  }
  block_argmax(s, i < n ? (int)i : INT_MAX, blockIdx.x, bval, bidx);
}

// C (K x K, column j = row piv[j] of Y) and M = C'C.
__global__ void __launch_bounds__(CB)
    k_cpqr_gram(int K, const float* __restrict__ Y, long long ldy, const int* __restrict__ piv,
                double* __restrict__ Cm, double* __restrict__ M) {
  for (int idx = threadIdx.x; idx < K * K; idx += CB) {
    const int c = idx / K, j = idx % K;
    Cm[idx] = (double)Y[(long long)piv[j] * ldy + c];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < K * K; idx += CB) {
    const int a = idx / K, b = idx % K;
    double s = 0.0;
    for (int c = 0; c < K; ++c) s = fma(Cm[c * K + a], Cm[c * K + b], s);
    M[idx] = s;
  }
}

// Q = C W diag(theta)^-1/2 W' (the polar factor of C), B = W diag(theta)^-1/2 W' first.
__global__ void __launch_bounds__(CB)
    k_cpqr_polar(int K, const double* __restrict__ Cm, const double* __restrict__ W,
                 const double* __restrict__ theta, double* __restrict__ B, double* __restrict__ Q) {
  for (int idx = threadIdx.x; idx < K * K; idx += CB) {
    const int a = idx / K, b = idx % K;
    double s = 0.0;
    for (int e = 0; e < K; ++e) {
      const double th = theta[e];
      const double f = th > 0.0 ? 1.0 / sqrt(th) : 0.0;
      s = fma(W[a * K + e] * f, W[b * K + e], s);
    }
    B[idx] = s;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < K * K; idx += CB) {
    const int c = idx / K, j = idx % K;
    double s = 0.0;
    for (int a = 0; a < K; ++a) s = fma(Cm[c * K + a], B[a * K + j], s);
    Q[idx] = s;
  }
}

// label_i = argmax_j |sum_c Y_ic Q_cj| (lowest j on ties), Q in shared memory when it fits.
__global__ void __launch_bounds__(CB)
    k_cpqr_label(long long n, int K, const float* __restrict__ Y, long long ldy,
                 const double* __restrict__ Q, int* __restrict__ labels, int use_smem) {
  extern __shared__ double qsm[];
  if (use_smem) {
    for (int idx = threadIdx.x; idx < K * K; idx += CB) qsm[idx] = Q[idx];
    __syncthreads();
  }
  const double* qm = use_smem ? qsm : Q;
  const long long i = (long long)blockIdx.x * CB + threadIdx.x;
  if (i >= n) return;
  const float* y = Y + i * ldy;
  double best = -1.0;
  int bj = 0;
  for (int j = 0; j < K; ++j) {
    double s = 0.0;
    for (int c = 0; c < K; ++c) s = fma((double)y[c], qm[c * K + j], s);
    const double a = fabs(s);
    if (a > best) {
      best = a;
      bj = j;
    }
  }
  labels[i] = bj;
}

}  // namespace

cudaError_t cpqr_assign(cudaStream_t st, Alloc& al, long long n, int K, const float* Y,
                        long long ldy, int* piv, int* labels, int* d_status) {
  if (n == 0 || K == 0) return cudaSuccess;
  const int nb = (int)((n + CB - 1) / CB);
  double* A = al.get<double>((size_t)n * K);
  double* nrm = al.get<double>((size_t)n);
  double* bval = al.get<double>((size_t)nb);
  int* bidx = al.get<int>((size_t)nb);
  double* q = al.get<double>((size_t)K);
  double* Cm = al.get<double>((size_t)K * K);
  double* M = al.get<double>((size_t)K * K);
  double* W = al.get<double>((size_t)K * K);
  double* B = al.get<double>((size_t)K * K);
  double* Q = al.get<double>((size_t)K * K);
  double* theta = al.get<double>((size_t)K);
  cudaError_t e = cudaSuccess;
  if (!A || !nrm || !bval || !bidx || !q || !Cm || !M || !W || !B || !Q || !theta) {
    e = cudaErrorMemoryAllocation;
  } else {
    ProfScope ps(st, "cpqr");
    k_cpqr_init<<<nb, CB, 0, st>>>(n, K, Y, ldy, A, nrm, bval, bidx);
    note_launch();
    for (int t = 0; t < K && e == cudaSuccess; ++t) {
      k_cpqr_pick<<<1, CB, 0, st>>>(nb, bval, bidx, A, K, nrm, q, piv, t);
      note_launch();
      if (t + 1 < K) {
        k_cpqr_proj<<<nb, CB, sizeof(double) * K, st>>>(n, K, A, nrm, q, bval, bidx);
        note_launch();
      }
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_cpqr_gram<<<1, CB, 0, st>>>(K, Y, ldy, piv, Cm, M);
      note_launch();
      e = rr_eig<double>(st, al, K, K, M, K, theta, W, d_status);
    }
    if (e == cudaSuccess) {
      k_cpqr_polar<<<1, CB, 0, st>>>(K, Cm, W, theta, B, Q);
      note_launch();
      size_t qb = sizeof(double) * (size_t)K * K;
      const int use_smem = qb <= 160 * 1024;
      if (!use_smem) qb = 0;
      if (qb > 48 * 1024)
        e = cudaFuncSetAttribute(k_cpqr_label, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)qb);
      if (e == cudaSuccess) {
        k_cpqr_label<<<nb, CB, qb, st>>>(n, K, Y, ldy, Q, labels, use_smem);
        note_launch();
        e = cudaGetLastError();
      }
    }
  }
  al.put(A);
  al.put(nrm);
  al.put(bval);
  al.put(bidx);
  al.put(q);
  al.put(Cm);
  al.put(M);
  al.put(W);
  al.put(B);
  al.put(Q);
  al.put(theta);
  return e;
}

}  // namespace sc
