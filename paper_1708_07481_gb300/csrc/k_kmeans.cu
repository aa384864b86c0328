// k-means on the unit-normalized rows of the eigenvector block (Sec. II.A: the rows are
// clustered, traditionally by k-means++).
//
// Seeding (Arthur & Vassilvitskii 2007), k sequential rounds, decisions in FP64:
//   update: D2_i <- min(D2_i, ||E_i - c_t||^2) in FP64 (FP32 data promoted exactly), with
//           FP64 block sums in a fixed tree order;
//   pick:   one CTA scans the block sums and then the chosen block's D2 to find the first i
//           whose running sum exceeds u_t * sum(D2) (clamped to the last row with D2 > 0;
//           sum(D2) = 0 -> lowest unchosen row).
// Lloyd rounds:
//   assign: FP32 distance ||c||^2 - 2 e.c to every centroid with a running best/second best;
//           rows whose margin is below a threshold are re-decided with direct FP64 distances
//           ||e - c||^2 (ties -> lowest index), so the labels are those of FP64 arithmetic;
//   update: per-CTA FP64 sums accumulated in row order (one thread per column), the last
//           CTA adds the CTA partials in fixed order and divides; empty clusters keep their
//           centroid.  Deterministic for a given n.
#include <algorithm>
#include <cstdio>

#include "common.cuh"

namespace sc {
namespace {

constexpr int PB = 256;  // rows per seeding block (one CTA each; the pick CTA has PB threads)

__device__ double block_sum_d(double v, double* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sh[32] = s;
  }
  __syncthreads();
  double r = sh[32];
  __syncthreads();
  return r;
}

// inclusive scan of doubles across the block (fixed order: warp scan + warp-total scan)
__device__ double block_incl_scan_d(double v, double* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    double s = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      double y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  double r = x + (wid > 0 ? sh[wid - 1] : 0.0);
  __syncthreads();
  return r;
}

__global__ void k_pp_first(int n, const double* u, int* seeds, int* chosen) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long i = (long long)floor(u[0] * (double)n);
    if (i > n - 1) i = n - 1;
    if (i < 0) i = 0;
    seeds[0] = (int)i;
    chosen[i] = 1;
  }
}

// Shared memory of the D2 update: the seed row in FP64 (cs, d) and FP32 (cs32), block-sum slots
// (sh, 40), the rows' new FP64 distances (dv, PB) and the list of rows to compute (lst, PB + 1).
struct PpSmem {
  double *cs, *sh, *dv;
  float* cs32;
  int* lst;
};
__host__ __device__ inline size_t pp_smem_bytes(int d) {
  return sizeof(double) * ((size_t)d + 40 + PB) + sizeof(float) * (size_t)((d + 1) & ~1) +
         sizeof(int) * (PB + 1);
}
__device__ inline PpSmem pp_smem(void* raw, int d) {
  PpSmem m;
  m.cs = (double*)raw;
  m.sh = m.cs + d;
  m.dv = m.sh + 40;
  m.cs32 = (float*)(m.dv + PB);
  m.lst = (int*)(m.cs32 + ((d + 1) & ~1));
  return m;
}

// Block b of the D2 update: D2_i <- min(D2_i, ||E_i - c||^2) for the PB rows of block b, c in
// cs (FP64), and the block's sum into bsum[b].  After the first round a row is screened first
// with its FP32 distance s: with unit rounding u = 2^-24, the FP32 sum of d squared differences
// is within a relative gamma = (d + 2) u of the exact one (all terms are nonnegative), so when
// s (1 - 2 gamma) > D2_i the exact distance exceeds D2_i and the row keeps D2_i.  The other rows
// get the FP64 distance, gathered into a list so that the FP64 warp instructions (GB300 runs an
// FP64 warp instruction at 2 FMA per clock per SM, lanes masked off or not) run on full warps.
// Every row ends with the value the plain FP64 update gives.
__device__ __forceinline__ void pp_update_block(int b, int n, int d, const float* __restrict__ E,
                                                long long lde, int t, const PpSmem& sm,
                                                double* D2, double* bsum) {
  const long long i = (long long)b * PB + threadIdx.x;
  if (threadIdx.x == 0) sm.lst[PB] = 0;
  __syncthreads();
  double old = 0.0;
  bool need = false;
  if (i < n) {
    if (t == 0) {
      need = true;
    } else {
      old = D2[i];
      const float* e = E + i * lde;
      float sf = 0.f;
      for (int c = 0; c < d; ++c) {
        const float df = e[c] - sm.cs32[c];
        sf = fmaf(df, df, sf);
      }
      const double gam = (double)(d + 2) * 0x1p-24;
      need = !((double)sf * (1.0 - 2.0 * gam) > old);
    }
  }
  if (need) sm.lst[atomicAdd(&sm.lst[PB], 1)] = threadIdx.x;
  __syncthreads();
  const int cnt = sm.lst[PB];
  for (int q = threadIdx.x; q < cnt; q += PB) {
    const int r = sm.lst[q];
    const long long ii = (long long)b * PB + r;
    const float* e = E + ii * lde;
    double acc = 0.0;
    for (int c = 0; c < d; ++c) {
      double df = (double)e[c] - sm.cs[c];
      acc = fma(df, df, acc);
    }
    const double nv = (t == 0) ? acc : fmin(D2[ii], acc);
    D2[ii] = nv;
    sm.dv[r] = nv;
  }
  __syncthreads();
  const double v = i < n ? (need ? sm.dv[threadIdx.x] : old) : 0.0;
  double bs = block_sum_d(v, sm.sh);
  if (threadIdx.x == 0) bsum[b] = bs;
}

__global__ void __launch_bounds__(PB)
    k_pp_update(int n, int d, const float* __restrict__ E, long long lde, const int* seeds, int t,
                double* D2, double* bsum) {
  extern __shared__ double pp_raw[];  // pp_smem_bytes(d)
  const PpSmem sm = pp_smem(pp_raw, d);
  const int s = seeds[t];
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    const float x = E[(long long)s * lde + c];
    sm.cs[c] = (double)x;
    sm.cs32[c] = x;
  }
  __syncthreads();
  pp_update_block(blockIdx.x, n, d, E, lde, t, sm, D2, bsum);
}

// The pick of round t by one CTA of PB threads.  D2 and the block sums are read through L2
// (__ldcg): in the persistent seeding they were written by other CTAs of the same launch.
__device__ __forceinline__ void pp_pick_body(int n, int nb, const double* __restrict__ D2,
                                             const double* __restrict__ bsum, const double* u,
                                             int t, int* seeds, int* chosen) {
  __shared__ double sh[40];
  __shared__ int sel;
  __shared__ double base_sh;
  // total over block sums in fixed order (thread-strided partial sums, then the tree)
  double p = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) p += __ldcg(bsum + b);
  double total = block_sum_d(p, sh);
  if (threadIdx.x == 0) sel = -1;
  __syncthreads();
  if (total > 0.0) {
    double target = u[t] * total;
    // running sum over blocks, PB blocks at a time
    double carry = 0.0;
    int bstar = -1;
    for (int b0 = 0; b0 < nb && bstar < 0; b0 += PB) {
      int b = b0 + threadIdx.x;
      double v = b < nb ? __ldcg(bsum + b) : 0.0;
      double inc = block_incl_scan_d(v, sh) + carry;
      double exc = inc - v;
      if (b < nb && exc <= target && target < inc) {
        sel = b;
        base_sh = exc;
      }
      __syncthreads();
      bstar = sel;
      double tot = block_sum_d(v, sh);
      carry += tot;
      __syncthreads();
    }
    if (bstar >= 0) {
      if (threadIdx.x == 0) sel = -1;
      __syncthreads();
      double base = base_sh;
      long long i = (long long)bstar * PB + threadIdx.x;
      double v = i < n ? __ldcg(D2 + i) : 0.0;
      double inc = block_incl_scan_d(v, sh) + base;
      if (i < n && inc > target && inc - v <= target) sel = (int)i;
      __syncthreads();
      bstar = sel;
    }
    if (threadIdx.x == 0) {
      int pick = bstar;
      if (pick < 0) {  // rounding put the target past the end: last row with D2 > 0
        for (long long i = n - 1; i >= 0; --i)
          if (__ldcg(D2 + i) > 0.0) {
            pick = (int)i;
            break;
          }
      }
      seeds[t] = pick;
      chosen[pick] = 1;
    }
  } else {
    // all remaining rows coincide with chosen seeds: lowest unchosen row
    if (threadIdx.x == 0) sel = n;
    __syncthreads();
    for (long long i = threadIdx.x; i < n; i += blockDim.x)
      if (!chosen[i]) {
        atomicMin(&sel, (int)i);
        break;
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      int pick = sel < n ? sel : 0;
      seeds[t] = pick;
      chosen[pick] = 1;
    }
  }
}

__global__ void __launch_bounds__(PB)
    k_pp_pick(int n, int nb, const double* __restrict__ D2, const double* __restrict__ bsum,
              const double* u, int t, int* seeds, int* chosen) {
  pp_pick_body(n, nb, D2, bsum, u, t, seeds, chosen);
}

// Grid-wide barrier of a cooperative launch (every CTA resident): an arrival counter bar[0]
// and a generation word bar[1] in global memory.  The wait is bounded (about two seconds of SM
// clocks); a CTA that gives up sets *flag, and every CTA that sees the flag returns false.
constexpr long long GB_WAIT_CLOCKS = 4LL << 30;
__device__ bool grid_barrier(unsigned* bar, int* flag) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = atomicAdd(bar + 1, 0u);
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (atomicAdd(bar + 1, 0u) == gen) {
        if (clock64() - t0 > GB_WAIT_CLOCKS) {
          ok = 0;
          atomicOr(flag, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (atomicAdd(flag, 0) != 0) ok = 0;
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// k-means++ seeding in one cooperative launch: the first seed, then rounds t = 0 .. k - 2 of
// (D2 update with seed t by every CTA over blocks b = blockIdx.x, blockIdx.x + gridDim.x, ...;
// pick of seed t + 1 by CTA 0), with a grid barrier after each phase.  The blocks, their sums
// and the pick are those of k_pp_update / k_pp_pick, so the seeds are the same.
__global__ void __launch_bounds__(PB)
    k_pp_all(int n, int d, int k, const float* __restrict__ E, long long lde, const double* u,
             int* seeds, int* chosen, double* D2, double* bsum, unsigned* bar, int* flag) {
  extern __shared__ double pp_raw[];  // pp_smem_bytes(d)
  const PpSmem sm = pp_smem(pp_raw, d);
  const int nb = (n + PB - 1) / PB;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    long long i = (long long)floor(u[0] * (double)n);
    if (i > n - 1) i = n - 1;
    if (i < 0) i = 0;
    seeds[0] = (int)i;
    chosen[i] = 1;
  }
  if (!grid_barrier(bar, flag)) return;
  for (int t = 0; t + 1 < k; ++t) {
    const int sd = __ldcg(seeds + t);
    for (int c = threadIdx.x; c < d; c += PB) {
      const float x = E[(long long)sd * lde + c];
      sm.cs[c] = (double)x;
      sm.cs32[c] = x;
    }
    __syncthreads();
    for (int b = blockIdx.x; b < nb; b += gridDim.x)
      pp_update_block(b, n, d, E, lde, t, sm, D2, bsum);
    if (!grid_barrier(bar, flag)) return;
    if (blockIdx.x == 0) pp_pick_body(n, nb, D2, bsum, u, t + 1, seeds, chosen);
    if (!grid_barrier(bar, flag)) return;
  }
}

// ---- Lloyd ---------------------------------------------------------------------------------

__global__ void k_init_cent(int d, int k, const float* __restrict__ E, long long lde,
                            const int* seeds, double* C64, float* C32, float* cn) {
  int j = blockIdx.x;
  if (j >= k) return;
  const float* e = E + (long long)seeds[j] * lde;
  float s = 0.f;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    C64[(long long)j * d + c] = (double)e[c];
    C32[(long long)j * d + c] = e[c];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < d; ++c) s = fmaf(C32[(long long)j * d + c], C32[(long long)j * d + c], s);
    cn[j] = s;
  }
}

constexpr int ACH = 64;  // centroids per shared-memory chunk in the assignment

// One row per thread; the row lives in registers (D >= d, D a multiple of 4), the centroids
// stream through shared memory in chunks of ACH.
// SUM: the CTA also forms its rows' per-cluster FP64 column sums and counts (the partial of the
// centroid update, one per CTA of 256 rows, rows in order) into part / pcnt, so that no separate
// pass over E is needed; its shared memory then holds the rows (256 d floats), the sums (k d
// doubles), the labels and the counts after the centroid chunks.
template <int D, bool SUM>
__global__ void __launch_bounds__(256)
    k_assign(int n, int d, int k, const float* __restrict__ E, long long lde,
             const float* __restrict__ C32, const float* __restrict__ cn,
             const double* __restrict__ C64, int* labels, int* changes, int first, double tie,
             const int* ctl, double* part = nullptr, int* pcnt = nullptr) {
  if (ctl[0]) return;  // converged in an earlier round (uniform: written by an earlier kernel)
  extern __shared__ float csm[];  // ACH * D
  __shared__ int nchg;
  if (threadIdx.x == 0) nchg = 0;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float ev[D];
#pragma unroll
  for (int q = 0; q < D; ++q) ev[q] = (i < n && q < d) ? E[i * lde + q] : 0.f;
  float best = 3.4e38f, second = 3.4e38f;
  int bj = 0;
  for (int j0 = 0; j0 < k; j0 += ACH) {
    int nj = min(ACH, k - j0);
    __syncthreads();
    for (int q = threadIdx.x; q < nj * D; q += blockDim.x) {
      int jj = q / D, c = q % D;
      csm[q] = c < d ? C32[(long long)(j0 + jj) * d + c] : 0.f;
    }
    __syncthreads();
    for (int jj = 0; jj < nj; ++jj) {
      const float4* c4 = reinterpret_cast<const float4*>(csm + jj * D);
      float dot = 0.f;
#pragma unroll
      for (int q = 0; q < D / 4; ++q) {
        float4 cv = c4[q];
        dot = fmaf(ev[4 * q], cv.x, dot);
        dot = fmaf(ev[4 * q + 1], cv.y, dot);
        dot = fmaf(ev[4 * q + 2], cv.z, dot);
        dot = fmaf(ev[4 * q + 3], cv.w, dot);
      }
      float dist = fmaf(-2.f, dot, cn[j0 + jj]);
      if (dist < best) {
        second = best;
        best = dist;
        bj = j0 + jj;
      } else if (dist < second) {
        second = dist;
      }
    }
  }
  if (i < n) {
    if (k > 1 && second - best < (float)tie) {
      // near tie: re-decide among the centroids within the margin, with direct FP64
      // distances ||e - c||^2 to the FP64 centroids (ties -> lowest index).  The FP32
      // distances are recomputed exactly as above (same order), from the centroids still in
      // shared memory when they all fit in one chunk.
      double bd = 1e300;
      int bb = 0;
      for (int j = 0; j < k; ++j) {
        float dot = 0.f;
        if (k <= ACH) {
          const float4* c4 = reinterpret_cast<const float4*>(csm + j * D);
#pragma unroll
          for (int q = 0; q < D / 4; ++q) {
            float4 cv = c4[q];
            dot = fmaf(ev[4 * q], cv.x, dot);
            dot = fmaf(ev[4 * q + 1], cv.y, dot);
            dot = fmaf(ev[4 * q + 2], cv.z, dot);
            dot = fmaf(ev[4 * q + 3], cv.w, dot);
          }
        } else {
          const float* cj = C32 + (long long)j * d;
#pragma unroll
          for (int q = 0; q < D; ++q) dot = fmaf(ev[q], q < d ? cj[q] : 0.f, dot);
        }
        float dist = fmaf(-2.f, dot, cn[j]);
        if (dist - best >= (float)tie) continue;
        const double* c = C64 + (long long)j * d;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < D; ++q) {
          if (q < d) {
            double df = (double)ev[q] - c[q];
            acc = fma(df, df, acc);
          }
        }
        if (acc < bd) {
          bd = acc;
          bb = j;
        }
      }
      bj = bb;
    }
    int old = labels[i];
    if (first || old != bj) atomicAdd(&nchg, 1);
    labels[i] = bj;
  }
  if constexpr (SUM) {
    float* rows = csm + (size_t)ACH * D;                      // 256 x d
    double* acc = reinterpret_cast<double*>(rows + 256 * d);  // k x d
    int* lab = reinterpret_cast<int*>(acc + (size_t)k * d);   // 256
    int* cnt = lab + 256;                                     // k
    const int t = threadIdx.x;
#pragma unroll
    for (int q = 0; q < D; ++q)
      if (q < d) rows[t * d + q] = ev[q];
    lab[t] = i < n ? bj : -1;
    for (int q = t; q < k * d; q += 256) acc[q] = 0.0;
    for (int j = t; j < k; j += 256) cnt[j] = 0;
    __syncthreads();
    if (i < n) atomicAdd(&cnt[bj], 1);  // integer counts: any order gives the same total
    if (t < d) {
      for (int r = 0; r < 256; ++r) {
        const int l = lab[r];
        if (l >= 0) acc[(size_t)l * d + t] += (double)rows[r * d + t];
      }
    }
    __syncthreads();
    double* pb = part + (size_t)blockIdx.x * k * d;
    for (int q = t; q < k * d; q += 256) pb[q] = acc[q];
    for (int j = t; j < k; j += 256) pcnt[(size_t)blockIdx.x * k + j] = cnt[j];
  }
  __syncthreads();
  if (threadIdx.x == 0 && nchg) atomicAdd(changes, nchg);
}

using AssignFn = void (*)(int, int, int, const float*, long long, const float*, const float*,
                          const double*, int*, int*, int, double, const int*, double*, int*);

inline AssignFn assign_for(int d, int* D, bool sum) {
#define SC_ASSIGN_PICK(DD)                                          \
  {                                                                 \
    *D = DD;                                                        \
    return sum ? k_assign<DD, true> : k_assign<DD, false>;          \
  }
  if (d <= 16) SC_ASSIGN_PICK(16)
  if (d <= 32) SC_ASSIGN_PICK(32)
  if (d <= 48) SC_ASSIGN_PICK(48)
  if (d <= 64) SC_ASSIGN_PICK(64)
  if (d <= 96) SC_ASSIGN_PICK(96)
  if (d <= 128) SC_ASSIGN_PICK(128)
  if (d <= 192) SC_ASSIGN_PICK(192)
  SC_ASSIGN_PICK(512)
#undef SC_ASSIGN_PICK
}

// Per-CTA FP64 cluster sums over a contiguous row range.  Rows pass through shared memory in
// chunks of CR (the labels and the d columns, loaded coalesced).  The CTA's threads form `sub`
// groups; group g accumulates rows g, g + sub, ... of each chunk in row order into its own
// shared accumulator (one thread per column), and the sub accumulators are added in group
// order at the end, so the summation order depends only on n, d and the launch shape.
// Counts are integers (shared atomics; any order gives the same total).
constexpr int CR = 64;

__global__ void k_cent_partial(int n, int d, int k, const float* __restrict__ E, long long lde,
                               const int* __restrict__ labels, long long rows_per_cta,
                               double* part, int* pcnt, int use_smem, int sub, const int* ctl,
                               const int* chg, int it) {
  if (ctl[0] || (it > 0 && *chg == 0)) return;  // no update this round
  extern __shared__ double acc_sm[];  // sub x k*d (when use_smem), then CR x d floats, CR
                                      // labels, k counts
  const long long kd = (long long)k * d;
  double* acc = use_smem ? acc_sm : part + (long long)blockIdx.x * kd;  // sub == 1 unless smem
  float* stg = reinterpret_cast<float*>(acc_sm + (use_smem ? (size_t)sub * kd : 0));
  int* lab = reinterpret_cast<int*>(stg + CR * d);
  int* cnt = lab + CR;
  const int gs = blockDim.x / sub, grp = threadIdx.x / gs, gt = threadIdx.x % gs;
  double* mine = acc + grp * kd;
  for (long long q = threadIdx.x; q < (long long)sub * kd; q += blockDim.x) acc[q] = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) cnt[j] = 0;
  const long long r0 = blockIdx.x * rows_per_cta, r1 = min((long long)n, r0 + rows_per_cta);
  for (long long r = r0; r < r1; r += CR) {
    const int nr = (int)min((long long)CR, r1 - r);
    __syncthreads();  // the previous chunk has been consumed
    for (int q = threadIdx.x; q < nr * d; q += blockDim.x) {
      const int rr = q / d;
      stg[q] = E[(r + rr) * lde + (q - rr * d)];
    }
    for (int q = threadIdx.x; q < nr; q += blockDim.x) lab[q] = labels[r + q];
    __syncthreads();
    if (grp < sub) {
      for (int rr = grp; rr < nr; rr += sub) {
        const int l = lab[rr];
        if ((unsigned)l >= (unsigned)k) continue;  // never written by an assignment: skip
        for (int c = gt; c < d; c += gs) mine[(long long)l * d + c] += (double)stg[rr * d + c];
        if (gt == 0) atomicAdd(&cnt[l], 1);
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) pcnt[(long long)blockIdx.x * k + j] = cnt[j];
  if (use_smem)
    for (long long q = threadIdx.x; q < kd; q += blockDim.x) {
      double v = acc[q];
      for (int g = 1; g < sub; ++g) v += acc[g * kd + q];
      part[(long long)blockIdx.x * kd + q] = v;
    }
}

// Centroid j = (sum of the CTA partials) / count, empty clusters kept.  Warp w of the CTA sums
// the partials w, w + 8, ... (two accumulators, even and odd steps) for 32 columns at a time;
// the 8 warp sums are added in warp order.
__global__ void __launch_bounds__(256)
    k_cent_reduce(int d, int k, int nct, const double* __restrict__ part,
                  const int* __restrict__ pcnt, double* C64, float* C32, float* cn, int* ctl,
                  const int* chg, int it) {
  const int j = blockIdx.x;
  // a round without label changes ends the iteration (before any centroid update); ctl[0]
  // is only ever set on that path, where every CTA returns without writing
  if (ctl[0]) return;
  if (it > 0 && *chg == 0) {
    if (j == 0 && threadIdx.x == 0) ctl[0] = 1;
    return;
  }
  if (j == 0 && threadIdx.x == 0) ctl[1] = it + 1;  // rounds with a centroid update
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ long long tot;
  __shared__ double ps[8][33];
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  {
    long long t = 0;  // integer counts: any summation order gives the same total
    for (int c = threadIdx.x; c < nct; c += blockDim.x) t += pcnt[(long long)c * k + j];
    atomicAdd((unsigned long long*)&tot, (unsigned long long)t);
  }
  __syncthreads();
  float s = 0.f;
  for (int c0 = 0; c0 < d; c0 += 32) {
    const int c = c0 + lane;
    double t0 = 0.0, t1 = 0.0;
    if (tot > 0 && c < d) {
      int q = w;
      for (; q + 8 < nct; q += 16) {
        t0 += part[((long long)q * k + j) * d + c];
        t1 += part[((long long)(q + 8) * k + j) * d + c];
      }
      if (q < nct) t0 += part[((long long)q * k + j) * d + c];
    }
    ps[w][lane] = t0 + t1;
    __syncthreads();
    if (w == 0 && c < d) {
      if (tot > 0) {
        double v = ps[0][lane];
#pragma unroll
        for (int q = 1; q < 8; ++q) v += ps[q][lane];
        const double mval = v / (double)tot;
        C64[(long long)j * d + c] = mval;
        C32[(long long)j * d + c] = (float)mval;
      }
      const float f = C32[(long long)j * d + c];
      s = fmaf(f, f, s);
    }
    __syncthreads();
  }
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) cn[j] = s;
  }
}

__global__ void k_inertia(int n, int d, int k, const float* __restrict__ E, long long lde,
                          const int* __restrict__ labels, const double* __restrict__ C64,
                          double* part) {
  __shared__ double sh[40];
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int l = labels[i];
    if ((unsigned)l >= (unsigned)k) continue;
    const double* c = C64 + (long long)l * d;
    for (int q = 0; q < d; ++q) {
      double df = (double)E[i * lde + q] - c[q];
      v = fma(df, df, v);
    }
  }
  double b = block_sum_d(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

}  // namespace

cudaError_t kmeanspp(cudaStream_t st, Alloc& al, int n, int d, int k, const float* E,
                     long long lde, const double* u_host, int* seeds) {
  int nb = (n + PB - 1) / PB;
  double* u = al.get<double>(k);
  double* D2 = al.get<double>(n);
  double* bsum = al.get<double>(nb);
  int* chosen = al.get<int>(n);
  int* bar = al.get<int>(4);  // grid barrier: arrivals, generation, time-out flag
  cudaError_t e = cudaSuccess;
  if (!u || !D2 || !bsum || !chosen || !bar) {
    e = cudaErrorMemoryAllocation;
  } else {
    cudaMemcpyAsync(u, u_host, sizeof(double) * k, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(chosen, 0, sizeof(int) * n, st);
    size_t sm = pp_smem_bytes(d);
    // one cooperative launch for every round when the device runs one (all CTAs resident)
    bool persistent = false;
    if (bar) {
      cudaMemsetAsync(bar, 0, sizeof(int) * 4, st);
      int dev = 0, nsm = 0, per = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pp_all, PB, sm) == cudaSuccess &&
          per > 0 && nsm > 0) {
        int grid = std::min(nb, per * nsm);
        unsigned* barp = (unsigned*)bar;
        int* flag = bar + 2;
        void* args[] = {&n, &d, &k, (void*)&E, &lde, &u, &seeds, &chosen, &D2, &bsum, &barp, &flag};
        ProfScope ps(st, "kmeanspp_update");
        persistent = cudaLaunchCooperativeKernel((const void*)k_pp_all, dim3(grid), dim3(PB), args,
                                                 sm, st) == cudaSuccess;
        note_launch();
        if (!persistent) cudaGetLastError();
      }
    }
    if (!persistent) {
      k_pp_first<<<1, 32, 0, st>>>(n, u, seeds, chosen);
      note_launch();
    }
    for (int t = 0; t < k && !persistent; ++t) {
      if (t > 0) {
        k_pp_pick<<<1, PB, 0, st>>>(n, nb, D2, bsum, u, t, seeds, chosen);
        note_launch();
      }
      if (t + 1 < k) {
        ProfScope ps(st, "kmeanspp_update");
        k_pp_update<<<nb, PB, sm, st>>>(n, d, E, lde, seeds, t, D2, bsum);
        note_launch();
      }
    }
    e = cudaGetLastError();
    // u_host may be a stack array of the caller: make sure the copy finished
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && persistent) {
      int hf = 0;
      e = cudaMemcpy(&hf, bar + 2, sizeof(int), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && hf) e = cudaErrorTimeout;  // a grid barrier gave up
    }
  }
  al.put(bar);
  al.put(u);
  al.put(D2);
  al.put(bsum);
  al.put(chosen);
  return e;
}

cudaError_t lloyd(cudaStream_t st, Alloc& al, int n, int d, int k, const float* E,
                  long long lde, const int* seeds, int iters, int* labels, double* C64,
                  int* iters_run, double* inertia) {
  float* C32 = al.get<float>((size_t)k * d);
  float* cn = al.get<float>(k);
  int* changes = al.get<int>((size_t)iters + 2);  // per-round change counts, then stop / done
  long long nct = 152 * 2;
  if (nct > n) nct = n > 0 ? n : 1;
  long long rpc = (n + nct - 1) / nct;
  nct = (n + rpc - 1) / rpc;
  if (nct < 1) nct = 1;
  const long long nab = (n + 255) / 256;  // assignment CTAs: the partials when they are fused
  const long long npart = std::max(nct, nab);
  double* part = al.get<double>((size_t)npart * k * d);
  int* pcnt = al.get<int>((size_t)npart * k);
  double* ipart = al.get<double>(152);
  int* tstat = al.get<int>(1);  // time-outs of the tensor-core assignment's bounded waits
  // The assignment runs on tensor cores (assign_tc) for large n k d, or when SC_TUNE_ASSIGN=1;
  // SC_TUNE_ASSIGN=0 keeps the CUDA-core kernel.  Both give the labels of FP64 arithmetic.
  const int forced = tune_override("assign");
  bool use_tc = forced >= 0 ? forced == 1 : (long long)n * k * d >= (1LL << 28);
  cudaError_t e = cudaSuccess;
  int done = 0;
  if (!C32 || !cn || !changes || !part || !pcnt || !ipart || !tstat) {
    e = cudaErrorMemoryAllocation;
    goto out;
  }
  {
    k_init_cent<<<k, 128, 0, st>>>(d, k, E, lde, seeds, C64, C32, cn);
    note_launch();
    int Dp = 0;
    AssignFn afn = assign_for(d, &Dp, false);
    size_t asm_bytes = sizeof(float) * (size_t)ACH * Dp;
    // The CUDA-core assignment also forms the centroid update's partial sums when its rows,
    // the k x d FP64 sums, the labels and the counts fit beside the centroid chunks
    const size_t fused_bytes = asm_bytes + sizeof(float) * 256 * (size_t)d +
                               sizeof(double) * (size_t)k * d + sizeof(int) * (256 + (size_t)k);
    const bool fuse = fused_bytes <= 100 * 1024;
    AssignFn afn_sum = assign_for(d, &Dp, true);
    if (fuse) {
      e = cudaFuncSetAttribute(afn_sum, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fused_bytes);
      if (e != cudaSuccess) goto out;
    }
    // opt in above 40 KB: the kernel's static shared memory comes on top of the dynamic part,
    // and the two together may not exceed the 48 KB default without the attribute
    if (asm_bytes > 40 * 1024) {
      e = cudaFuncSetAttribute(afn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asm_bytes);
      if (e != cudaSuccess) goto out;
    }
    const size_t stg_bytes = sizeof(float) * (size_t)CR * d + sizeof(int) * ((size_t)CR + k);
    const size_t kdb = sizeof(double) * (size_t)k * d;
    int sub = 4;
    while (sub > 1 && sub * kdb + stg_bytes > 160 * 1024) sub /= 2;
    int use_smem = sub * kdb + stg_bytes <= 160 * 1024;
    if (!use_smem) sub = 1;
    size_t psm = (use_smem ? sub * kdb : 0) + stg_bytes;
    if (psm > 40 * 1024) {
      e = cudaFuncSetAttribute(k_cent_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psm);
      if (e != cudaSuccess) goto out;
    }
    unsigned ab = (unsigned)((n + 255) / 256);
    int* ctl = changes + iters;
    cudaMemsetAsync(changes, 0, sizeof(int) * ((size_t)iters + 2), st);
    // Rounds are issued without waiting: a round that changes no label sets the stop flag on
    // the device and every later kernel returns at once; the host looks every 4 rounds.
    cudaMemsetAsync(tstat, 0, sizeof(int), st);
    for (int it = 0; it < iters; ++it) {
      // FP32 distances of unit rows to centroids of norm <= 1 carry at most ~2.5e-7 d of
      // rounding each; margins below twice that (plus slack) are re-decided in FP64.  The
      // tensor cores' 3-term split TF32 products and their FP32 accumulation are held to four
      // times that margin.
      const double tie = 2e-5 + 5e-7 * d;
      bool on_tc = false;
      if (use_tc) {
        const cudaError_t et = assign_tc(st, n, d, k, E, lde, C32, cn, C64, labels,
                                         changes + it, it == 0, (float)tie, ctl, tstat);
        if (et == cudaSuccess) {
          on_tc = true;
        } else if (et == cudaErrorNotSupported) {
          use_tc = false;
          cudaGetLastError();
        } else {
          e = et;
          goto out;
        }
      }
      const bool fused = !on_tc && fuse;
      if (!on_tc) {
        ProfScope ps(st, "kmeans_assign");
        if (fused)
          afn_sum<<<ab, 256, fused_bytes, st>>>(n, d, k, E, lde, C32, cn, C64, labels,
                                                changes + it, it == 0, tie, ctl, part, pcnt);
        else
          afn<<<ab, 256, asm_bytes, st>>>(n, d, k, E, lde, C32, cn, C64, labels, changes + it,
                                           it == 0, tie, ctl, nullptr, nullptr);
        note_launch();
      }
      // a launch that did not start leaves the labels unwritten: stop here
      if ((e = cudaGetLastError()) != cudaSuccess) goto out;
      if (!fused) {
        k_cent_partial<<<(unsigned)nct, 64 * sub, psm, st>>>(n, d, k, E, lde, labels, rpc, part,
                                                             pcnt, use_smem, sub, ctl,
                                                             changes + it, it);
        note_launch();
      }
      k_cent_reduce<<<k, 256, 0, st>>>(d, k, (int)(fused ? nab : nct), part, pcnt, C64, C32, cn,
                                       ctl, changes + it, it);
      note_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) goto out;
      if ((it + 1) % 4 == 0 && it + 1 < iters) {
        int h = 0;
        cudaMemcpyAsync(&h, ctl, sizeof(int), cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto out;
        if (h) break;
      }
    }
    cudaMemcpyAsync(&done, ctl + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    k_inertia<<<152, 256, 0, st>>>(n, d, k, E, lde, labels, C64, ipart);
    note_launch();
    double hp[152];
    cudaMemcpyAsync(hp, ipart, sizeof(hp), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto out;
    double s = 0.0;
    for (int q = 0; q < 152; ++q) s += hp[q];
    if (inertia) *inertia = s;
    if (iters_run) *iters_run = done;
    int ht = 0;
    if ((e = cudaMemcpy(&ht, tstat, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) goto out;
    if (ht) e = cudaErrorTimeout;  // a bounded wait of the tensor-core assignment gave up
  }
out:
  if (e == cudaSuccess) e = cudaGetLastError();
  al.put(C32);
  al.put(cn);
  al.put(changes);
  al.put(part);
  al.put(pcnt);
  al.put(ipart);
  al.put(tstat);
  return e;
}

}  // namespace sc
