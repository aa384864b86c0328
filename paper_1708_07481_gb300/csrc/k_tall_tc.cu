// Tall-skinny LOBPCG updates on tcgen05 tensor cores (Sec. IV: the O(n l) multi-vector
// work): out (n x b) = beta Cin + [A_0 A_1 A_2] W for FP32 blocks, as the update
// [X R P] Y, the projections R - X F and the Cholesky-QR transforms V Tm of one pass.
//
// 3-term split TF32 as in the Gram kernel: x = x_big + x_small, x_big = tf32(x),
// x_small = tf32(x - x_big); A W ~ Ab Wb + Ab Ws + As Wb, FP32 accumulation in tensor memory.
//
// Operands (both K-major, 128-byte swizzle), in chunks of 32 columns of A (= 32 rows of W):
//   A side (M = 128 rows of the tall block): a TMA tiled load of the FP32 rows with
//   SWIZZLE_128B lands exactly in the K-major SW128 layout the MMA reads, so the split is an
//   in-place sweep over the staged tile (big overwrites the FP32 values, small goes to a second
//   buffer at the same offsets);
//   B side (N = output columns rounded up to 16): W^T is split once per call by a small kernel
//   into an image of per-chunk big / small SW128 tiles in global memory, and each chunk's tile
//   comes with the A chunk as one bulk copy completing on the same mbarrier.
// Each A segment is cut into chunks of 32 columns (the last one zero-filled by the TMA past
// the segment's width; the matching rows of W^T are zero).  A persistent CTA walks row tiles
// of 128 with up to six staged chunks in flight (as many as fit beside each other).  Two
// kernels:
//   k_tall_ws (the update): copies, the split, the MMA issue (4 K-steps x 3 products per
//   chunk) and the epilogue run on separate warps, with two tensor-memory accumulators so
//   that a tile's epilogue overlaps the next tile's MMAs;
//   k_tall_tc (the k-means assignment mode): every thread splits each chunk, one thread issues
//   the copies and the MMAs, commits per stage and per tile, and refills the previous chunk's
//   stage; eight warps read the accumulator with tcgen05.ld (warp w: rows 32 (w % 4) .. +32,
//   columns 32 (w / 4) + 64 j .. +32) for the assignment epilogue.
// Every wait is bounded; on a time-out a CTA records ST_TIMEOUT, waits (bounded) for its
// copies and MMAs in flight, frees its tensor memory and returns.
#include <algorithm>
#include <cstring>

#include "tc.cuh"

namespace sc {
namespace {

constexpr int TT_M = 128;     // rows per tile (MMA M)
constexpr int TT_K = 32;      // columns per chunk (one 128-byte swizzle row of FP32)
constexpr int TT_MAXSTG = 6;  // staged chunks in flight, at most
constexpr int TT_NTH = 256;   // eight warps: warps w, w + 4 share lane quarter w % 4
constexpr int TT_ATILE = TT_M * TT_K * 4;             // 16 KB: one FP32 (then big) A chunk
constexpr int TT_SMEM = 225 * 1024;                   // dynamic shared memory of a CTA
constexpr int TT_AM_BYTES = TT_M * 12;                // assignment mode: the upper warps' part
constexpr int TT_SMEM_USE = TT_SMEM - 1024 - 256 - TT_AM_BYTES;  // stages (after alignment,
                                                                  // barriers, assignment part)

#ifdef SC_TT_PHASES
// Debug builds only: clock64() time of CTA thread 0 in each part of k_tall_tc's chunk loop,
// summed over CTAs (0 chunk wait, 1 split, 2 MMA issue, 3 accumulator wait, 4 epilogue,
// 5 whole loop, 6 CTAs, 7 chunks, 8 wait for the previous chunk's MMAs, 9 refill issue).
__device__ long long g_tt_phase[10];
#define TT_T(i)                        \
  do {                                 \
    if (tid == 0) {                    \
      const long long t1_ = clock64(); \
      tt_acc[i] += t1_ - tt_t0;        \
      tt_t0 = t1_;                     \
    }                                  \
  } while (0)
// The same for k_tall_ws, per role (the first thread of the role's first warp): 0 copies:
// wait for a free stage, 1 copies: issue, 2 split: wait for a chunk, 3 split: work,
// 4 MMA: wait for a split chunk, 5 MMA: wait for a free accumulator, 6 MMA: issue,
// 7 epilogue: wait for an accumulator, 8 epilogue: work, 9 the CTA's loop, 10 CTAs, 11 chunks.
__device__ long long g_tw_phase[12];
#define TW_T(i)                        \
  do {                                 \
    if (tw_me) {                       \
      const long long t1_ = clock64(); \
      tw_acc[i] += t1_ - tw_t0;        \
      tw_t0 = t1_;                     \
    }                                  \
  } while (0)
#else
#define TT_T(i) \
  do {          \
  } while (0)
#define TW_T(i) \
  do {          \
  } while (0)
#endif

struct TcTall {
  int nseg;
  int nch[3];     // chunks of each A segment
  int cseg[3];    // columns of each A segment
  int wrow[3];    // first logical row of W for each segment
  int nchunks;    // total chunks
  int nn;         // MMA N: output columns rounded up to 16
  int nstg;       // stages
  int stage;      // bytes per stage: A big + A small + W^T chunk (big + small)
  long long n;
  int ntiles;
  const uint8_t* wimg;  // W^T image: per chunk nn x 128 B big, then nn x 128 B small
  // outputs: columns [0, b0) -> segment 0, [b0, b) -> segment 1
  float* out[2];
  long long ldo[2];
  const float* cin[2];
  long long ldc[2];
  const float* w[2];
  int ldw[2];
  int wskip[2];
  int vec[2];
  int b0, b;
  float beta;
  // W given transposed (W[lr][col] = w[col * ldw + lr]), as the centroid matrix in k-means
  int wt;
  // k-means assignment mode (amode): the accumulator holds e_i . c_j for the k = b centroids;
  // the epilogue turns it into labels instead of writing it (see k_tall_tc)
  int amode, first, d;
  float tie;  // margin of the tensor-core distances (at least twice their error)
  const float* cn;      // ||c_j||^2 (FP32)
  const double* C64;    // FP64 centroids, k x d
  const float* E;       // the rows, n x d (stride lde)
  long long lde;
  int* labels;
  int* changes;
  const int* ctl;       // ctl[0] != 0: converged in an earlier round (nothing to do)
};

__device__ __forceinline__ float tt_w(const TcTall& p, int lr, int col) {
  if (col >= p.b) return 0.f;
  const bool s1 = col >= p.b0;
  const int skip = s1 ? p.wskip[1] : p.wskip[0];
  if (lr < skip) return 0.f;
  const float* w = s1 ? p.w[1] : p.w[0];
  const int ldw = s1 ? p.ldw[1] : p.ldw[0];
  const int c = s1 ? col - p.b0 : col;
  return p.wt ? w[(long long)c * ldw + (lr - skip)] : w[(long long)(lr - skip) * ldw + c];
}

// The W^T image: for chunk ch (segment q, local chunk cc), operand row r (output column) and
// k < 32, logical row lr = wrow[q] + 32 cc + k of W; entries past the segment's width are 0.
__global__ void k_tall_wsplit(const __grid_constant__ TcTall p, uint8_t* __restrict__ img) {
  if (p.amode && p.ctl && *p.ctl) return;  // uniform: written by an earlier kernel
  const long long tot = (long long)p.nchunks * p.nn * TT_K;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % TT_K), r = (int)((idx / TT_K) % p.nn);
    const int ch = (int)(idx / ((long long)TT_K * p.nn));
    int q = 0, cc = ch;
    while (q + 1 < p.nseg && cc >= p.nch[q]) cc -= p.nch[q++];
    const int lc = cc * TT_K + kk;
    const float wv = lc < p.cseg[q] ? tt_w(p, p.wrow[q] + lc, r) : 0.f;
    const uint32_t bgv = to_tf32(wv);
    const uint32_t smv = to_tf32(wv - __uint_as_float(bgv));
    uint8_t* base = img + (size_t)ch * 2 * p.nn * 128;
    const uint32_t off = sw128_off(r, kk);
    *reinterpret_cast<uint32_t*>(base + off) = bgv;
    *reinterpret_cast<uint32_t*>(base + (size_t)p.nn * 128 + off) = smv;
  }
}

// Bulk copy of `bytes` contiguous bytes (16-byte aligned, a multiple of 16) into shared
// memory, completing on an mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Reads 32 accumulator columns c0 .. c0 + 31 of the warp's lane quarter (row 32 (w % 4) + l).
__device__ __forceinline__ void tt_ld32(uint32_t tmem, int warp, int c0, uint32_t (&v)[32]) {
  const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Writes accumulator columns c0 .. c0 + 31 of one row (v = the 32 values of a tcgen05.ld):
// out = beta Cin + acc, float4 stores where the output segment allows them.
__device__ __forceinline__ void tt_store32(const TcTall& p, const uint32_t (&v)[32],
                                           long long row, int c0) {
  if (row >= p.n) return;
#pragma unroll
  for (int j4 = 0; j4 < 8; ++j4) {
    const int col = c0 + 4 * j4;
    if (col >= p.b) break;
    const int s1 = col >= p.b0 ? 1 : 0;
    const int cs = s1 ? col - p.b0 : col;
    const int bs = s1 ? p.b - p.b0 : p.b0;
    float r4[4] = {__uint_as_float(v[4 * j4]), __uint_as_float(v[4 * j4 + 1]),
                   __uint_as_float(v[4 * j4 + 2]), __uint_as_float(v[4 * j4 + 3])};
    if (p.vec[s1] && cs + 3 < bs) {
      const float* cin = p.cin[s1];
      if (cin) {
        const float4 cv = *reinterpret_cast<const float4*>(cin + row * p.ldc[s1] + cs);
        r4[0] = fmaf(p.beta, cv.x, r4[0]);
        r4[1] = fmaf(p.beta, cv.y, r4[1]);
        r4[2] = fmaf(p.beta, cv.z, r4[2]);
        r4[3] = fmaf(p.beta, cv.w, r4[3]);
      }
      *reinterpret_cast<float4*>(p.out[s1] + row * p.ldo[s1] + cs) =
          make_float4(r4[0], r4[1], r4[2], r4[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cj = col + j;
        if (cj >= p.b) break;
        const int t1 = cj >= p.b0 ? 1 : 0;
        const int ct = t1 ? cj - p.b0 : cj;
        const float* cn = p.cin[t1];
        float x = r4[j];
        if (cn) x = fmaf(p.beta, cn[row * p.ldc[t1] + ct], x);
        p.out[t1][row * p.ldo[t1] + ct] = x;
      }
    }
  }
}

// Assignment epilogue of a tile (every thread of the CTA calls it).  Thread (warp w, lane l)
// owns row 32 (w % 4) + l and the accumulator columns 32 (w / 4) + 64 j: for each it forms the
// FP32 distance ||c_j||^2 - 2 e.c_j and keeps the best (lowest index among equal values) and
// the second best; the upper four warps hand theirs to the lower four through shared memory,
// which merge them.  A row whose margin (second - best) is below p.tie is re-decided with
// exact FP64 distances ||e - c_j||^2 for the centroids whose tensor-core distance lies within
// p.tie of the best (ties -> lowest index): p.tie is at least twice the error of the 3-term
// split TF32 distances, so the exact nearest centroid is among them and the labels are those
// of FP64 arithmetic.  The candidates are read back from tensor memory by both warps of the
// row; their FP64 minima are merged like the FP32 ones.
__device__ __forceinline__ void assign_epilogue(const TcTall& p, uint32_t tmem, int warp, int lane,
                                                long long row, float* sb, float* ss, int* sj,
                                                int* nchg) {
  float best = 3.4e38f, second = 3.4e38f;
  int bj = 0;
  for (int c0 = 32 * (warp >> 2); c0 < p.b; c0 += 64) {  // uniform in the warp
    uint32_t v[32];
    tt_ld32(tmem, warp, c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int col = c0 + j;
      if (col < p.b) {
        const float dist = fmaf(-2.f, __uint_as_float(v[j]), p.cn[col]);
        if (dist < best) {
          second = best;
          best = dist;
          bj = col;
        } else if (dist < second) {
          second = dist;
        }
      }
    }
  }
  const int r = 32 * (warp & 3) + lane;
  if (warp >= 4) {
    sb[r] = best;
    ss[r] = second;
    sj[r] = bj;
  }
  __syncthreads();
  bool tie = false;
  if (warp < 4) {
    // merge with the upper warp's columns
    const float b2 = sb[r], s2 = ss[r];
    const int j2 = sj[r];
    if (b2 < best || (b2 == best && j2 < bj)) {
      second = fminf(s2, best);
      best = b2;
      bj = j2;
    } else {
      second = fminf(second, b2);
    }
    tie = row < p.n && p.b > 1 && second - best < p.tie;
  }
  __syncthreads();
  if (warp < 4) {
    sb[r] = best;          // the row's best, for the candidates of both warps
    sj[r] = tie ? 1 : 0;
  }
  __syncthreads();
  if (warp >= 4) {
    best = sb[r];
    tie = sj[r] != 0;
  }
  // FP64 distances of the candidates (warps with a near-tie row only)
  double bd = 1e300;
  int bb = 0x7fffffff;
  if (__any_sync(0xffffffffu, tie)) {
    const float* e = p.E + (tie ? row : 0) * p.lde;
    for (int c0 = 32 * (warp >> 2); c0 < p.b; c0 += 64) {
      uint32_t v[32];
      tt_ld32(tmem, warp, c0, v);
      if (tie) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = c0 + j;
          if (col >= p.b) break;
          const float dist = fmaf(-2.f, __uint_as_float(v[j]), p.cn[col]);
          if (dist - best >= p.tie) continue;
          const double* c = p.C64 + (long long)col * p.d;
          double acc = 0.0;
          for (int q = 0; q < p.d; ++q) {
            const double df = (double)e[q] - c[q];
            acc = fma(df, df, acc);
          }
          if (acc < bd) {  // columns ascend within a warp: the first minimum is the lowest
            bd = acc;
            bb = col;
          }
        }
      }
    }
  }
  __syncthreads();  // every read of sb / ss / sj is done: the area takes the FP64 minima
  double* sd = reinterpret_cast<double*>(sb);  // 128 doubles over sb and ss
  if (warp >= 4) {
    sd[r] = bd;
    sj[r] = bb;
  }
  __syncthreads();
  if (warp < 4 && row < p.n) {
    if (tie) {
      const double bd2 = sd[r];
      const int bb2 = sj[r];
      if (bd2 < bd || (bd2 == bd && bb2 < bb)) {
        bd = bd2;
        bb = bb2;
      }
      bj = bb;
    }
    const int old = p.labels[row];
    if (p.first || old != bj) atomicAdd(nchg, 1);
    p.labels[row] = bj;
  }
}

__global__ void __launch_bounds__(TT_NTH, 1)
    k_tall_tc(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
              const __grid_constant__ CUtensorMap map2, const __grid_constant__ TcTall p,
              int* status) {
  if (p.amode && p.ctl && *p.ctl) return;  // uniform: written by an earlier kernel
  extern __shared__ __align__(1024) uint8_t tt_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)tt_raw + 1023) & ~(uintptr_t)1023);
  __shared__ int am_chg;
  const int nstg = p.nstg, sb = p.stage, wbytes = p.nn * 128;
  uint64_t* bars = (uint64_t*)(base + (size_t)nstg * sb);
  uint64_t* full = bars;                   // [nstg] A chunk and W^T chunk landed
  uint64_t* mdone = bars + TT_MAXSTG;      // [nstg] MMAs reading the stage finished
  uint64_t* accd = bars + 2 * TT_MAXSTG;   // accumulator of the tile complete
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * TT_MAXSTG + 1);
  float* am_best = (float*)((uint8_t*)bars + 256);  // assignment mode: the upper warps' part
  float* am_second = am_best + TT_M;
  int* am_bj = (int*)(am_second + TT_M);
  __shared__ int abort_flag, acc_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const CUtensorMap* maps[3] = {&map0, &map1, &map2};
  int tcols = 32;
  while (tcols < p.nn) tcols <<= 1;
  auto a_big = [&](int s) { return base + (size_t)s * sb; };
  auto a_sml = [&](int s) { return base + (size_t)s * sb + TT_ATILE; };
  auto w_big = [&](int s) { return base + (size_t)s * sb + 2 * TT_ATILE; };

  if (tid == 0) {
    abort_flag = 0;
    am_chg = 0;
    for (int q = 0; q < 2 * TT_MAXSTG + 1; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int q = 0; q < p.nseg; ++q)
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)maps[q]) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(p.nn >> 3) << 17) |
                         ((uint32_t)(TT_M >> 4) << 24);

  // the CTA's sequence of loads: index i -> tile blockIdx.x + (i / nchunks) gridDim.x, chunk
  // i % nchunks, stage i % nstg
  const int my_tiles = blockIdx.x < p.ntiles ? (p.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long total = (long long)my_tiles * p.nchunks;
  // thread 0's next load (stage, chunk, tile), advanced without divisions
  int is_s = 0, is_ch = 0, is_tile = blockIdx.x;
  auto issue = [&]() {
    int q = 0, cc = is_ch;
    while (q + 1 < p.nseg && cc >= p.nch[q]) cc -= p.nch[q++];
    mbar_expect_tx(&full[is_s], TT_ATILE + 2 * wbytes);
    tma_load_2d(a_big(is_s), maps[q], cc * TT_K, is_tile * TT_M, &full[is_s]);
    bulk_load(w_big(is_s), p.wimg + (size_t)is_ch * 2 * wbytes, 2 * wbytes, &full[is_s]);
    if (++is_s == nstg) is_s = 0;
    if (++is_ch == p.nchunks) {
      is_ch = 0;
      is_tile += gridDim.x;
    }
  };
  long long issued = 0, acc_commits = 0;
  // per stage: bit s of mpar = parity of the commits to mdone[s] so far, of many = any commit
  uint32_t mpar = 0, many = 0;
  if (tid == 0)
    for (; issued < total && issued < nstg; ++issued) issue();

#ifdef SC_TT_PHASES
  long long tt_acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  long long tt_t0 = clock64();
  const long long tt_start = tt_t0;
#endif
  // chunk i: stage s = i % nstg (full-barrier parity fpar = (i / nstg) & 1), chunk ch of
  // tile `tile`
  int s = 0, ch = 0, tile = blockIdx.x;
  uint32_t fpar = 0;
  auto advance = [&]() {
    if (++s == nstg) {
      s = 0;
      fpar ^= 1u;
    }
    if (++ch == p.nchunks) {
      ch = 0;
      tile += gridDim.x;
    }
  };
  for (long long i = 0; i < total; ++i, advance()) {
    if (!mbar_wait(&full[s], fpar)) atomicExch(&abort_flag, 1);
    __syncthreads();
    if (abort_flag) break;
    TT_T(0);
    // split the staged FP32 A chunk in place: big over the FP32 values, small beside it
    {
      uint4* sbg = reinterpret_cast<uint4*>(a_big(s));
      uint4* ssm = reinterpret_cast<uint4*>(a_sml(s));
#pragma unroll
      for (int v = tid; v < TT_ATILE / 16; v += TT_NTH) {
        const uint4 x = sbg[v];
        uint4 bg, sm;
        bg.x = to_tf32(__uint_as_float(x.x));
        bg.y = to_tf32(__uint_as_float(x.y));
        bg.z = to_tf32(__uint_as_float(x.z));
        bg.w = to_tf32(__uint_as_float(x.w));
        sm.x = to_tf32(__uint_as_float(x.x) - __uint_as_float(bg.x));
        sm.y = to_tf32(__uint_as_float(x.y) - __uint_as_float(bg.y));
        sm.z = to_tf32(__uint_as_float(x.z) - __uint_as_float(bg.z));
        sm.w = to_tf32(__uint_as_float(x.w) - __uint_as_float(bg.w));
        sbg[v] = bg;
        ssm[v] = sm;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    TT_T(1);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ab = smem_u32(a_big(s)), as_ = smem_u32(a_sml(s));
      const uint32_t wb = smem_u32(w_big(s)), ws = wb + wbytes;
#pragma unroll
      for (int ks = 0; ks < TT_K / 8; ++ks) {
        const uint32_t ko = ks * 32;
        const uint32_t acc0 = (ch > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(tmem, sw128_desc(as_ + ko), sw128_desc(wb + ko), idesc, acc0);
        mma_tf32(tmem, sw128_desc(ab + ko), sw128_desc(ws + ko), idesc, 1u);
        mma_tf32(tmem, sw128_desc(ab + ko), sw128_desc(wb + ko), idesc, 1u);
      }
      mma_commit(&mdone[s]);
      mpar ^= 1u << s;
      many |= 1u << s;
      if (ch == p.nchunks - 1) {
        mma_commit(accd);
        acc_commits += 1;
      }
      TT_T(2);
      // refill the previous chunk's stage (its MMAs were issued one chunk ago): load
      // i + nstg - 1 goes where load i - 1 was
      if (i >= 1 && issued < total) {
        const int sp = s == 0 ? nstg - 1 : s - 1;
        const bool okw = mbar_wait(&mdone[sp], ((mpar >> sp) & 1u) ^ 1u);
        TT_T(8);
        if (!okw) {
          atomicExch(&abort_flag, 1);
        } else {
          issue();
          ++issued;
        }
        TT_T(9);
      }
    }
    if (ch == p.nchunks - 1) {
      // epilogue of the tile: all threads wait for the accumulator
      if (tid == 0) acc_ok = mbar_wait(accd, (uint32_t)((acc_commits - 1) & 1)) ? 1 : 0;
      __syncthreads();
      if (!acc_ok) {
        if (tid == 0) atomicExch(&abort_flag, 1);
        break;
      }
      TT_T(3);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const long long row = (long long)tile * TT_M + 32 * (warp & 3) + lane;
      if (p.amode) {
        assign_epilogue(p, tmem, warp, lane, row, am_best, am_second, am_bj, &am_chg);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        continue;
      }
      for (int c0 = 32 * (warp >> 2); c0 < p.b; c0 += 64) {  // uniform in the warp
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
              "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tt_store32(p, v, row, c0);
      }
      // the accumulator is read: the next tile's first MMA may overwrite it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      TT_T(4);
    }
  }
#ifdef SC_TT_PHASES
  if (tid == 0) {
    tt_acc[5] = clock64() - tt_start;
    for (int q = 0; q < 10; ++q)
      if (q != 6 && q != 7) atomicAdd((unsigned long long*)&g_tt_phase[q], (unsigned long long)tt_acc[q]);
    atomicAdd((unsigned long long*)&g_tt_phase[6], 1ull);
    atomicAdd((unsigned long long*)&g_tt_phase[7], (unsigned long long)total);
  }
#endif
  // drain: wait (bounded) for this CTA's MMAs, and after a time-out for its copies in flight
  if (tid == 0) {
    bool ok = !abort_flag;
    for (int q = 0; q < nstg; ++q)
      if ((many >> q) & 1u) ok = mbar_wait(&mdone[q], ((mpar >> q) & 1u) ^ 1u) && ok;
    if (acc_commits > 0) ok = mbar_wait(accd, (uint32_t)((acc_commits - 1) & 1)) && ok;
    if (!ok) {
      // the latest load into each stage (a load into a stage is issued only after the one
      // before it was consumed, so waiting for the latest covers them all)
      for (long long j = std::max(0LL, issued - nstg); j < issued; ++j)
        mbar_wait(&full[j % nstg], (uint32_t)((j / nstg) & 1));
      atomicOr(status, ST_TIMEOUT);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (p.amode && tid == 0 && am_chg) atomicAdd(p.changes, am_chg);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tcols)
                 : "memory");
  }
}

// The update (not the assignment mode) with the roles of a CTA on separate warps, so that the
// copies, the TF32 split, the MMA issue and the epilogue of consecutive chunks and tiles
// overlap instead of taking turns behind CTA-wide barriers:
//   warp 0, lane 0: copies (A chunk + W^T chunk per stage; a stage is refilled once the MMAs
//     that read it have completed, mbarrier `empty`);
//   warps 2, 3, 8 .. 11: the in-place split of each landed A chunk (mbarrier `splitd`, one
//     arrival per warp);
//   warp 1, lane 0: the MMAs of each split chunk into one of two tensor-memory accumulators
//     (alternating by tile), committing `empty` per chunk and `accf` per tile;
//   warps 4 .. 7: the epilogue of each finished accumulator (lane quarter = warp % 4, every
//     column), then `acce` frees it for the tile after next.
// The arithmetic (products, their order, the accumulation) is that of k_tall_tc.  Every wait
// is bounded; after a time-out the CTA records ST_TIMEOUT, waits (bounded) for its own copies
// and MMAs in flight, frees its tensor memory and returns.
constexpr int TW_NTH = 384;
constexpr int TW_NSPLIT = 6;  // splitter warps

__device__ __forceinline__ int tw_splitter(int warp) {
  return warp >= 8 ? warp - 6 : ((warp == 2 || warp == 3) ? warp - 2 : -1);
}

__global__ void __launch_bounds__(TW_NTH, 1)
    k_tall_ws(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
              const __grid_constant__ CUtensorMap map2, const __grid_constant__ TcTall p,
              int* status) {
  extern __shared__ __align__(1024) uint8_t tw_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)tw_raw + 1023) & ~(uintptr_t)1023);
  const int nstg = p.nstg, sb = p.stage, wbytes = p.nn * 128;
  uint64_t* bars = (uint64_t*)(base + (size_t)nstg * sb);
  uint64_t* full = bars;                       // [nstg] A chunk and W^T chunk landed
  uint64_t* splitd = bars + TT_MAXSTG;         // [nstg] A chunk split (one arrival per warp)
  uint64_t* empty = bars + 2 * TT_MAXSTG;      // [nstg] MMAs reading the stage finished
  uint64_t* accf = bars + 3 * TT_MAXSTG;       // [2] accumulator of a tile complete
  uint64_t* acce = accf + 2;                   // [2] accumulator read by the epilogue
  uint32_t* tmem_slot = (uint32_t*)(acce + 2);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const CUtensorMap* maps[3] = {&map0, &map1, &map2};
  int tcols = 32;
  while (tcols < p.nn) tcols <<= 1;
  auto a_big = [&](int st) { return base + (size_t)st * sb; };
  auto a_sml = [&](int st) { return base + (size_t)st * sb + TT_ATILE; };
  auto w_big = [&](int st) { return base + (size_t)st * sb + 2 * TT_ATILE; };

  if (tid == 0) {
    abort_flag = 0;
    for (int q = 0; q < TT_MAXSTG; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&splitd[q], TW_NSPLIT);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&accf[q], 1);
      mbar_init(&acce[q], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int q = 0; q < p.nseg; ++q)
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)maps[q]) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(p.nn >> 3) << 17) |
                         ((uint32_t)(TT_M >> 4) << 24);
  const int my_tiles = blockIdx.x < p.ntiles ? (p.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long total = (long long)my_tiles * p.nchunks;
  volatile int* vabort = &abort_flag;

#ifdef SC_TT_PHASES
  long long tw_acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const bool tw_me = lane == 0 && (warp == 0 || warp == 1 || warp == 2 || warp == 4);
  long long tw_t0 = clock64();
  const long long tw_start = tw_t0;
#endif
  // thread-local records for the drain after a time-out
  long long issued = 0;           // copies issued (warp 0, lane 0)
  uint32_t mpar = 0, many = 0;    // per stage: parity of the commits to empty[s], any commit
  int acnt[2] = {0, 0};           // commits to accf[0 / 1]

  if (warp == 0) {
    if (lane == 0) {
      int st = 0, ch = 0, tile = blockIdx.x;
      uint32_t rpar = 0;  // parity of the stage round (issue index / nstg)
      for (long long i = 0; i < total; ++i) {
        if (*vabort) break;
        if (i >= nstg && !mbar_wait(&empty[st], rpar ^ 1u)) {  // the round before, consumed
          atomicExch(&abort_flag, 1);
          break;
        }
        TW_T(0);
        int q = 0, cc = ch;
        while (q + 1 < p.nseg && cc >= p.nch[q]) cc -= p.nch[q++];
        mbar_expect_tx(&full[st], TT_ATILE + 2 * wbytes);
        tma_load_2d(a_big(st), maps[q], cc * TT_K, tile * TT_M, &full[st]);
        bulk_load(w_big(st), p.wimg + (size_t)ch * 2 * wbytes, 2 * wbytes, &full[st]);
        ++issued;
        TW_T(1);
        if (++st == nstg) {
          st = 0;
          rpar ^= 1u;
        }
        if (++ch == p.nchunks) {
          ch = 0;
          tile += gridDim.x;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int st = 0, ch = 0, tl = 0;
      uint32_t rpar = 0;
      for (long long i = 0; i < total; ++i) {
        if (*vabort) break;
        if (!mbar_wait(&splitd[st], rpar)) {
          atomicExch(&abort_flag, 1);
          break;
        }
        TW_T(4);
        const int ab = tl & 1;
        if (ch == 0 && tl >= 2 && !mbar_wait(&acce[ab], (uint32_t)(((tl >> 1) - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        TW_T(5);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(ab * tcols);
        const uint32_t abg = smem_u32(a_big(st)), asm_ = smem_u32(a_sml(st));
        const uint32_t wb = smem_u32(w_big(st)), ws = wb + wbytes;
#pragma unroll
        for (int ks = 0; ks < TT_K / 8; ++ks) {
          const uint32_t ko = ks * 32;
          const uint32_t acc0 = (ch > 0 || ks > 0) ? 1u : 0u;
          mma_tf32(acc, sw128_desc(asm_ + ko), sw128_desc(wb + ko), idesc, acc0);
          mma_tf32(acc, sw128_desc(abg + ko), sw128_desc(ws + ko), idesc, 1u);
          mma_tf32(acc, sw128_desc(abg + ko), sw128_desc(wb + ko), idesc, 1u);
        }
        mma_commit(&empty[st]);
        mpar ^= 1u << st;
        many |= 1u << st;
        if (ch == p.nchunks - 1) {
          mma_commit(&accf[ab]);
          acnt[ab] += 1;
        }
        TW_T(6);
        if (++st == nstg) {
          st = 0;
          rpar ^= 1u;
        }
        if (++ch == p.nchunks) {
          ch = 0;
          ++tl;
        }
      }
    }
  } else if (warp >= 4 && warp < 8) {
    // epilogue: lane quarter warp % 4 (rows 32 (warp % 4) + lane of the tile), every column
    for (int tl = 0; tl < my_tiles; ++tl) {
      if (*vabort) break;
      const int ab = tl & 1;
      if (!mbar_wait(&accf[ab], (uint32_t)((tl >> 1) & 1))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      TW_T(7);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const long long row =
          (long long)(blockIdx.x + tl * gridDim.x) * TT_M + 32 * (warp & 3) + lane;
      for (int c0 = 0; c0 < p.b; c0 += 32) {  // uniform in the warp
        uint32_t v[32];
        tt_ld32(tmem + (uint32_t)(ab * tcols), warp, c0, v);
        tt_store32(p, v, row, c0);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[ab]);
      TW_T(8);
    }
  } else {
    const int sw = tw_splitter(warp);  // 0 .. TW_NSPLIT - 1
    int st = 0;
    uint32_t rpar = 0;
    for (long long i = 0; i < total; ++i) {
      if (*vabort) break;
      if (!mbar_wait(&full[st], rpar)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      TW_T(2);
      // big over the FP32 values, small beside them (the arithmetic of k_tall_tc's split)
      uint4* sbg = reinterpret_cast<uint4*>(a_big(st));
      uint4* ssm = reinterpret_cast<uint4*>(a_sml(st));
      for (int v = sw * 32 + lane; v < TT_ATILE / 16; v += TW_NSPLIT * 32) {
        const uint4 x = sbg[v];
        uint4 bg, sm;
        bg.x = to_tf32(__uint_as_float(x.x));
        bg.y = to_tf32(__uint_as_float(x.y));
        bg.z = to_tf32(__uint_as_float(x.z));
        bg.w = to_tf32(__uint_as_float(x.w));
        sm.x = to_tf32(__uint_as_float(x.x) - __uint_as_float(bg.x));
        sm.y = to_tf32(__uint_as_float(x.y) - __uint_as_float(bg.y));
        sm.z = to_tf32(__uint_as_float(x.z) - __uint_as_float(bg.z));
        sm.w = to_tf32(__uint_as_float(x.w) - __uint_as_float(bg.w));
        sbg[v] = bg;
        ssm[v] = sm;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&splitd[st]);
      TW_T(3);
      if (++st == nstg) {
        st = 0;
        rpar ^= 1u;
      }
    }
  }

  __syncthreads();
#ifdef SC_TT_PHASES
  if (tw_me) {
    tw_acc[9] = clock64() - tw_start;
    for (int q = 0; q < 10; ++q)
      if (tw_acc[q]) atomicAdd((unsigned long long*)&g_tw_phase[q], (unsigned long long)tw_acc[q]);
  }
  if (tid == 0) {
    atomicAdd((unsigned long long*)&g_tw_phase[10], 1ull);
    atomicAdd((unsigned long long*)&g_tw_phase[11], (unsigned long long)total);
  }
#endif
  if (*vabort) {
    // drain: this CTA's MMAs, then its copies in flight (the latest load into each stage
    // covers the ones before it)
    if (warp == 1 && lane == 0) {
      for (int q = 0; q < nstg; ++q)
        if ((many >> q) & 1u) mbar_wait(&empty[q], ((mpar >> q) & 1u) ^ 1u);
      for (int q = 0; q < 2; ++q)
        if (acnt[q] > 0) mbar_wait(&accf[q], (uint32_t)((acnt[q] - 1) & 1));
    }
    if (warp == 0 && lane == 0)
      for (long long j = issued > nstg ? issued - nstg : 0; j < issued; ++j)
        mbar_wait(&full[j % nstg], (uint32_t)((j / nstg) & 1));
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * tcols)
                 : "memory");
  }
}

}  // namespace

// out = beta Cin + A W on tensor cores when the shape fits (A segments 16-byte aligned with
// strides a multiple of 4 floats, N <= 256 output columns); otherwise cudaErrorNotSupported and
// the caller uses the CUDA-core kernels.  The W^T image (2 x chunks x N x 128 bytes, at most
// 1 MB) is a stream-ordered allocation of the call, freed behind the launch.
static cudaError_t tall_gemm_tc_one(cudaStream_t st, long long n, const Cat3<float>& A,
                                    const TallSeg<float>& s0, const TallSeg<float>& s1,
                                    float beta, int* d_status, const TcTall* am = nullptr);

// Outputs wider than one MMA (N > 256) run as column pieces of at most 256 (multiples of 16),
// each its own pass over A.
cudaError_t tall_gemm_tc(cudaStream_t st, long long n, const Cat3<float>& A,
                         const TallSeg<float>& s0, const TallSeg<float>& s1, float beta,
                         int* d_status) {
  const int b = s0.b + s1.b;
  if (n <= 0 || b <= 0) return cudaErrorNotSupported;
  if (((b + 15) & ~15) <= 256) return tall_gemm_tc_one(st, n, A, s0, s1, beta, d_status);
  const TallSeg<float>* sg[2] = {&s0, &s1};
  for (int q = 0; q < 2; ++q) {
    const TallSeg<float>& g = *sg[q];
    if (g.b == 0) continue;
    const int pieces = (g.b + 255) / 256;
    const int width = ((g.b + pieces - 1) / pieces + 15) & ~15;
    for (int c0 = 0; c0 < g.b; c0 += width) {
      TallSeg<float> part = g;
      part.b = std::min(width, g.b - c0);
      part.out = g.out + c0;
      part.Cin = g.Cin ? g.Cin + c0 : nullptr;
      part.W = g.W + c0;
      const TallSeg<float> none{};
      const cudaError_t e = tall_gemm_tc_one(st, n, A, part, none, beta, d_status);
      if (e != cudaSuccess) return e;  // (a piece that is not supported aborts the call)
    }
  }
  return cudaSuccess;
}

static cudaError_t tall_gemm_tc_one(cudaStream_t st, long long n, const Cat3<float>& A,
                                    const TallSeg<float>& s0, const TallSeg<float>& s1,
                                    float beta, int* d_status, const TcTall* am) {
  const int b = s0.b + s1.b;
  if (n <= 0 || b <= 0) return cudaErrorNotSupported;
  TcTall p{};
  if (am) {  // the k-means assignment mode (assign_tc)
    p.wt = am->wt;
    p.amode = am->amode;
    p.first = am->first;
    p.d = am->d;
    p.tie = am->tie;
    p.cn = am->cn;
    p.C64 = am->C64;
    p.E = am->E;
    p.lde = am->lde;
    p.labels = am->labels;
    p.changes = am->changes;
    p.ctl = am->ctl;
  }
  p.nseg = A.nblk;
  p.n = n;
  int ch = 0, wr = 0;
  for (int q = 0; q < A.nblk; ++q) {
    if (((uintptr_t)A.p[q] & 15) || (A.ld[q] & 3) || A.c[q] <= 0) return cudaErrorNotSupported;
    p.cseg[q] = A.c[q];
    p.nch[q] = (A.c[q] + TT_K - 1) / TT_K;
    p.wrow[q] = wr;
    ch += p.nch[q];
    wr += A.c[q];
  }
  p.nchunks = ch;
  p.nn = (b + 15) & ~15;
  if (p.nn > 256) return cudaErrorNotSupported;
  p.stage = 2 * TT_ATILE + 2 * p.nn * 128;
  p.nstg = std::min(TT_MAXSTG, TT_SMEM_USE / p.stage);
  if (p.nstg < 2) return cudaErrorNotSupported;
  const TallSeg<float>* sg[2] = {&s0, &s1};
  for (int q = 0; q < 2; ++q) {
    const TallSeg<float>& g = *sg[q];
    p.out[q] = g.out;
    p.ldo[q] = g.ldo;
    p.cin[q] = g.Cin;
    p.ldc[q] = g.ldc;
    p.w[q] = g.W;
    p.ldw[q] = g.ldw;
    p.wskip[q] = g.wskip;
    p.vec[q] = g.b > 0 && ((uintptr_t)g.out & 15) == 0 && (g.ldo & 3) == 0 &&
               (!g.Cin || (((uintptr_t)g.Cin & 15) == 0 && (g.ldc & 3) == 0)) &&
               (q == 0 || (s0.b & 3) == 0);
  }
  p.b0 = s0.b;
  p.b = b;
  p.beta = beta;
  p.ntiles = (int)((n + TT_M - 1) / TT_M);
  CUtensorMap m[3];
  for (int q = 0; q < 3; ++q) {
    const int qq = q < A.nblk ? q : 0;
    if (!make_map_fp32(&m[q], A.p[qq], n, A.c[qq], A.ld[qq], TT_K, TT_M,
                       CU_TENSOR_MAP_SWIZZLE_128B))
      return cudaErrorNotSupported;
  }
  const size_t img_bytes = (size_t)2 * ch * p.nn * 128;
  uint8_t* img = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&img, img_bytes, st);
  if (e != cudaSuccess) return e;
  p.wimg = img;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(k_tall_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TT_SMEM);
    cudaFuncSetAttribute(k_tall_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, TT_SMEM);
  });
  {
    ProfScope ps(st, am ? "kmeans_assign" : "tall_gemm");
    const long long tot = (long long)ch * p.nn * TT_K;
    k_tall_wsplit<<<(unsigned)std::min<long long>((tot + 255) / 256, 1024), 256, 0, st>>>(p, img);
    note_launch();
    const int grid = std::min(p.ntiles, 152);
    if (am)
      k_tall_tc<<<grid, TT_NTH, TT_SMEM, st>>>(m[0], m[1], m[2], p, d_status);
    else
      k_tall_ws<<<grid, TW_NTH, TT_SMEM, st>>>(m[0], m[1], m[2], p, d_status);
    note_launch();
  }
  e = cudaGetLastError();
  cudaFreeAsync(img, st);
  return e;
}

#ifdef SC_TT_PHASES
}  // namespace sc
// Debug builds only: the k_tall_tc phase sums (out[0..9], see g_tt_phase) and the k_tall_ws
// ones (out[10..21], see g_tw_phase) since the previous call, which clears them.
extern "C" int sc_debug_tt_phases(long long* out) {
  if (cudaDeviceSynchronize() != cudaSuccess) return -6;
  if (cudaMemcpyFromSymbol(out, sc::g_tt_phase, sizeof(long long) * 10) != cudaSuccess) return -6;
  if (cudaMemcpyFromSymbol(out + 10, sc::g_tw_phase, sizeof(long long) * 12) != cudaSuccess)
    return -6;
  long long z[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (cudaMemcpyToSymbol(sc::g_tw_phase, z, sizeof(z)) != cudaSuccess) return -6;
  return cudaMemcpyToSymbol(sc::g_tt_phase, z, sizeof(long long) * 10) == cudaSuccess ? 0 : -6;
}
namespace sc {
#endif

// k-means assignment on tensor cores: the update kernel with A = E (n x d rows) and W = C^T (the
// k x d FP32 centroids read transposed), its epilogue turning e_i . c_j into labels (k <= 256;
// near ties re-decided in FP64).  cudaErrorNotSupported when the shape does not fit the tensor
// map rules (E 16-byte aligned, lde a multiple of 4); the caller then uses the CUDA-core kernel.
cudaError_t assign_tc(cudaStream_t st, long long n, int d, int k, const float* E, long long lde,
                      const float* C32, const float* cn, const double* C64, int* labels,
                      int* changes, int first, float tie, const int* ctl, int* d_status) {
  if (n <= 0 || d < 1 || k < 1 || k > 256) return cudaErrorNotSupported;
  TcTall am{};
  am.wt = 1;
  am.amode = 1;
  am.first = first;
  am.d = d;
  am.tie = 4.f * tie;
  am.cn = cn;
  am.C64 = C64;
  am.E = E;
  am.lde = lde;
  am.labels = labels;
  am.changes = changes;
  am.ctl = ctl;
  const TallSeg<float> s0{nullptr, 0, nullptr, 0, C32, d, 0, k};
  const TallSeg<float> s1{};
  return tall_gemm_tc_one(st, n, cat<float>(E, lde, d), s0, s1, 0.f, d_status, &am);
}

}  // namespace sc
