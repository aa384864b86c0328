// Tensor-core Gram matrices on sm_103a: C = A' B for tall FP32 blocks A (n x a), B (n x b)
// (Sec. IV: Gram products of the n x l multi-vectors, O(n l^2)).
//
// 3-term split TF32 (Markidis et al. 2018 style error-free splitting): x = x_big + x_small
// with x_big = tf32(x) and x_small = tf32(x - x_big); A'B ~ Ab'Bb + Ab'Bs + As'Bb, products on
// tcgen05 (kind::tf32, FP32 accumulation in tensor memory), ~2^-21 relative per product.
//
// CTA = one 128 x 128 output tile over one chunk of rows.  Per stage of 32 rows:
//   TMA (cp.async.bulk.tensor.2d) brings the FP32 row blocks of A and B into shared memory
//   (three staging slots, mbarrier complete_tx); all 256 threads split them into big/small TF32
//   operands written in the K-major 128-byte-swizzled layout the MMA reads (the transpose
//   from row-major to K-major happens here, for free); one thread issues 4 K-steps x 3
//   products of tcgen05.mma 128x128x8 into a TMEM accumulator and commits to an mbarrier
//   that frees the operand buffer.  The epilogue reads TMEM with tcgen05.ld and writes the
//   tile's FP64 partial; a second kernel sums the partials over chunks in fixed order.
// Every wait is bounded: on a timeout the CTA records ST_TIMEOUT, waits (bounded) for its
// own outstanding copies and MMAs, frees its tensor memory and returns.  If that draining wait
// gives up as well, the CTA still frees its tensor memory and returns, with an MMA or a copy
// possibly still running; the launch has then already failed with ST_TIMEOUT, and the
// context's status word reports it.
// Test hook (probe_spins > 0): after every copy and MMA of the CTA has completed, thread 0
// waits on an mbarrier phase that nothing completes, for at most probe_spins polls; the wait
// gives up and records ST_TIMEOUT with nothing in flight, which exercises the time-out
// reporting without a fault.
#include <algorithm>
#include <cstring>

#include "tc.cuh"

namespace sc {
namespace {

constexpr int TM = 128, TN = 128, BK = 32, NTH = 256;
constexpr int STAGE_BYTES = BK * TM * 4;     // 16 KB: FP32 rows of one operand
constexpr int OP_BYTES = TM * BK * 4;        // 16 KB: one TF32 operand tile
constexpr int NSTG = 3;                      // FP32 staging slots (copies in flight)
constexpr int SMEM_BYTES = NSTG * 2 * STAGE_BYTES + 2 * 4 * OP_BYTES + 1024 + 256;
struct SegMap {
  int start[3];
  int count[3];
  int nseg;
};

__device__ inline int seg_index(const SegMap& s, int c) {
  int off = 0;
  for (int q = 0; q < s.nseg; ++q) {
    if (c >= s.start[q] && c < s.start[q] + s.count[q]) return off + c - s.start[q];
    off += s.count[q];
  }
  return -1;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_tf32() {
  return (1u << 4)                 // c_format F32
         | (2u << 7)               // a_format TF32
         | (2u << 10)              // b_format TF32
         | ((uint32_t)(TN >> 3) << 17)
         | ((uint32_t)(TM >> 4) << 24);
}

// Split one FP32 stage (BK rows x TM columns, row-major) into big/small K-major operands;
// only the first ncols columns (operand rows) are needed.
__device__ inline void convert_stage(const float* stage, uint8_t* big, uint8_t* small,
                                     int ncols) {
  const int r = threadIdx.x & (TM - 1);  // operand row = column of the block
  if (r >= ncols) return;
  for (int kc = threadIdx.x >> 7; kc < BK / 4; kc += NTH / TM) {
    uint32_t bg[4], sm[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float x = stage[(kc * 4 + q) * TM + r];
      uint32_t b = to_tf32(x);
      bg[q] = b;
      sm[q] = to_tf32(x - __uint_as_float(b));
    }
    uint32_t off = sw128_off(r, kc * 4);
    *reinterpret_cast<uint4*>(big + off) = make_uint4(bg[0], bg[1], bg[2], bg[3]);
    *reinterpret_cast<uint4*>(small + off) = make_uint4(sm[0], sm[1], sm[2], sm[3]);
  }
}

__global__ void __launch_bounds__(NTH, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              long long n, int nbt, int sym, int nch, int ntiles, long long rows_per_chunk,
              int a, int b, double* __restrict__ part, int* status, long long probe_spins) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte aligned base for the swizzled operands
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* opA = base;                           // [buf][big/small] 16 KB each
  uint8_t* opB = opA + 4 * OP_BYTES;
  float* stA = (float*)(opB + 4 * OP_BYTES);     // [slot] 16 KB
  float* stB = stA + NSTG * (STAGE_BYTES / 4);
  uint64_t* bars = (uint64_t*)(stB + NSTG * (STAGE_BYTES / 4));
  uint64_t* full = bars;            // [NSTG] TMA landed
  uint64_t* mdone = bars + NSTG;    // [2] MMAs of an operand buffer finished
  uint64_t* probe = bars + NSTG + 2; // test hook: a phase nothing completes
  uint32_t* tmem_slot = (uint32_t*)(bars + NSTG + 3);
  __shared__ int abort_flag;

  const int tile = blockIdx.x / nch, chunk = blockIdx.x % nch;
  const int2 tl = tile_coord(tile, nbt, sym);
  const int ca = tl.x * TM, cb = tl.y * TN;
  // The MMA's M side is always 128 wide; its N side is trimmed to the valid width of the
  // narrower block (rounded up to 16).  When A's side of the tile is the narrower one the
  // tile is computed transposed (B columns as M); the reduction maps it back.
  const int va = min(TM, a - ca), vb = min(TN, b - cb);
  const bool swp = !sym && va < vb;
  const int nn = ((swp ? va : vb) + 15) & ~15;
  const CUtensorMap* mapM = swp ? &mapB : &mapA;
  const CUtensorMap* mapN = swp ? &mapA : &mapB;
  const int xm = swp ? cb : ca, xn = swp ? ca : cb;
  const long long r0 = (long long)chunk * rows_per_chunk;
  long long r1 = r0 + rows_per_chunk;
  if (r1 > n) r1 = n;
  const int nst = (int)((r1 - r0 + BK - 1) / BK);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int q = 0; q < NSTG + 3; ++q) mbar_init(&bars[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapB) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t IDESC = (idesc_tf32() & ~(0x3Fu << 17)) | ((uint32_t)(nn >> 3) << 17);

  // prologue: stages 0 .. NSTG - 1 in flight
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTG && s < nst; ++s) {
      mbar_expect_tx(&full[s], 2 * STAGE_BYTES);
      int y = (int)(r0 + (long long)s * BK);
      tma_load_2d(stA + s * (STAGE_BYTES / 4), mapM, xm, y, &full[s]);
      tma_load_2d(stB + s * (STAGE_BYTES / 4), mapN, xn, y, &full[s]);
    }
  }
  int issued_commits[2] = {0, 0};
  int loads_issued[NSTG], loads_done[NSTG];  // thread 0's bookkeeping
  for (int q = 0; q < NSTG; ++q) {
    loads_issued[q] = q < nst ? 1 : 0;
    loads_done[q] = 0;
  }
  for (int s = 0; s < nst; ++s) {
    const int ss = s % NSTG;  // staging slot
    const int slot = s & 1;   // operand buffer
    bool ok = mbar_wait(&full[ss], (uint32_t)((s / NSTG) & 1));
    if (ok) loads_done[ss] += 1;
    if (ok && s >= 2) ok = mbar_wait(&mdone[slot], (uint32_t)(((s - 2) >> 1) & 1));
    if (!ok) atomicExch(&abort_flag, 1);
    __syncthreads();
    if (abort_flag) break;
    uint8_t* aB = opA + (slot * 2) * OP_BYTES;
    uint8_t* aS = aB + OP_BYTES;
    uint8_t* bB = opB + (slot * 2) * OP_BYTES;
    uint8_t* bS = bB + OP_BYTES;
    convert_stage(stA + ss * (STAGE_BYTES / 4), aB, aS, TM);
    convert_stage(stB + ss * (STAGE_BYTES / 4), bB, bS, nn);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ab = smem_u32(aB), as_ = smem_u32(aS), bb = smem_u32(bB), bs = smem_u32(bS);
#pragma unroll
      for (int ks = 0; ks < BK / 8; ++ks) {
        const uint32_t ko = ks * 32;  // 8 TF32 values along K
        uint32_t acc0 = (s > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(tmem, sw128_desc(as_ + ko), sw128_desc(bb + ko), IDESC, acc0);
        mma_tf32(tmem, sw128_desc(ab + ko), sw128_desc(bs + ko), IDESC, 1u);
        mma_tf32(tmem, sw128_desc(ab + ko), sw128_desc(bb + ko), IDESC, 1u);
      }
      mma_commit(&mdone[slot]);
      issued_commits[slot] += 1;
      // the staging slot was consumed by the conversion above: refill it with stage s + NSTG
      if (s + NSTG < nst) {
        loads_issued[ss] += 1;
        mbar_expect_tx(&full[ss], 2 * STAGE_BYTES);
        int y = (int)(r0 + (long long)(s + NSTG) * BK);
        tma_load_2d(stA + ss * (STAGE_BYTES / 4), mapM, xm, y, &full[ss]);
        tma_load_2d(stB + ss * (STAGE_BYTES / 4), mapN, xn, y, &full[ss]);
      }
    }
  }
  // wait for the last MMAs (both buffers' latest commits); thread 0 knows the counts
  __shared__ int last_ok;
  if (threadIdx.x == 0) {
    bool ok = !abort_flag;
    for (int q = 0; q < 2; ++q)
      if (issued_commits[q] > 0)
        ok = mbar_wait(&mdone[q], (uint32_t)((issued_commits[q] - 1) & 1)) && ok;
    // after an abort, copies may still be in flight: wait (bounded) for the latest one
    for (int q = 0; q < NSTG; ++q)
      if (loads_issued[q] > loads_done[q])
        ok = mbar_wait(&full[q], (uint32_t)((loads_issued[q] - 1) & 1)) && ok;
    last_ok = ok ? 1 : 0;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (last_ok && nst > 0) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +32 (M index), columns 64 (w / 4) ..
    // +64 (N index, up to nn); element (M, N) is tile entry (M, N), or (N, M) when swapped
    const int lrow = 32 * (warp & 3) + lane;
    const int cbase = 64 * (warp >> 2);
    double* dst = part + ((long long)chunk * ntiles + tile) * TM * TN;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (cbase + 32 * h >= nn) break;  // uniform in the warp
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cbase + 32 * h);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // partials are stored N-major (element (M, N) at N * TM + M), so the 32 lanes (32
      // consecutive M) of each store write one contiguous 256-byte run
      const int mcount = swp ? vb : va, ncount = swp ? va : vb;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int jn = cbase + 32 * h + q;  // N index
        if (lrow < mcount && jn < ncount)
          dst[(long long)jn * TM + lrow] = (double)__uint_as_float(v[q]);
      }
    }
  } else if (!last_ok && threadIdx.x == 0) {
    atomicOr(status, ST_TIMEOUT);
  }
  if (probe_spins > 0 && threadIdx.x == 0 && last_ok) {
    // every copy and MMA of this CTA has completed (waited above): nothing is in flight
    if (!mbar_wait(probe, 0u, probe_spins)) atomicOr(status, ST_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN)
                 : "memory");
  }
}

// C = the sum of the chunk partials of each tile, in a fixed order.  One CTA per N index of a
// tile (the partials are N-major) and one thread per M index and chunk group: thread (M, h)
// sums chunks h, h + RH, h + 2 RH, ... into four accumulators (chunk h + RH (4q + u) goes to
// accumulator u), which are added pairwise; the RH group sums are added in order h = 0 .. RH-1.
// Element (M, N) is tile entry (M, N), or (N, M) when the kernel swapped the operand roles.
// Entries past the output are skipped.
static_assert(TM == 128 && TN == 128, "the reduction maps one thread to each of 128 M indices");
constexpr int RH = 8;  // chunk groups of the reduction: thread (mi, h) sums chunks c = h (mod RH)
__global__ void __launch_bounds__(TM * RH)
    k_gram_tc_reduce(const double* __restrict__ part, int nch, int ntiles, int nbt, int a, int b,
                     SegMap ma, SegMap mb, double* C, int ldc, int sym) {
  __shared__ double hs[RH][TM];
  const int tile = blockIdx.x / TN, jn = blockIdx.x % TN;
  const int2 tl = tile_coord(tile, nbt, sym);
  const int ca = tl.x * TM, cb = tl.y * TN;
  const int va = min(TM, a - ca), vb = min(TN, b - cb);
  const bool swp = !sym && va < vb;  // the same choice as the Gram kernel
  const int mcount = swp ? vb : va, ncount = swp ? va : vb;
  if (jn >= ncount) return;  // uniform in the CTA
  const int mi = threadIdx.x & (TM - 1), h = threadIdx.x / TM;
  const double* src = part + (long long)tile * TM * TN + (long long)jn * TM;
  const long long cstride = (long long)ntiles * TM * TN;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (mi < mcount) {
    int c = h;
    for (; c + 3 * RH < nch; c += 4 * RH) {
      s0 += src[(long long)c * cstride + mi];
      s1 += src[(long long)(c + RH) * cstride + mi];
      s2 += src[(long long)(c + 2 * RH) * cstride + mi];
      s3 += src[(long long)(c + 3 * RH) * cstride + mi];
    }
    for (; c < nch; c += RH) s0 += src[(long long)c * cstride + mi];
  }
  hs[h][mi] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (h == 0 && mi < mcount) {
    double t = hs[0][mi];
#pragma unroll
    for (int q = 1; q < RH; ++q) t += hs[q][mi];
    const int ti = swp ? jn : mi, tj = swp ? mi : jn;
    const int oi = seg_index(ma, ca + ti), oj = seg_index(mb, cb + tj);
    if (oi >= 0 && oj >= 0) {
      C[(long long)oi * ldc + oj] = t;
      if (sym && tl.x != tl.y) C[(long long)oj * ldc + oi] = t;
    }
  }
}

bool make_map(CUtensorMap* m, const float* ptr, long long rows, int cols, long long ld,
              int box_cols) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)BK};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

int gram_tc_smem_bytes() { return SMEM_BYTES; }

// C (compact, FP64) = A' B with A = columns [0, a) of a row-major FP32 block (stride lda) and
// B = columns [0, b) of another; the segment maps drop padding columns from the output.
cudaError_t gram_tc(cudaStream_t st, Alloc& al, long long n, const float* A, long long lda,
                    int a, const int* segA, int nsegA, const float* B, long long ldb, int b,
                    const int* segB, int nsegB, double* C, int ldc, bool sym, int* d_status,
                    long long probe_spins) {
  if (a == 0 || b == 0) return cudaSuccess;
  SegMap ma{}, mb{};
  ma.nseg = nsegA;
  mb.nseg = nsegB;
  for (int q = 0; q < nsegA; ++q) { ma.start[q] = segA[2 * q]; ma.count[q] = segA[2 * q + 1]; }
  for (int q = 0; q < nsegB; ++q) { mb.start[q] = segB[2 * q]; mb.count[q] = segB[2 * q + 1]; }
  int oa = 0, ob = 0;
  for (int q = 0; q < nsegA; ++q) oa += ma.count[q];
  for (int q = 0; q < nsegB; ++q) ob += mb.count[q];
  if (n == 0) return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * ob, oa, st);
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (lda & 3) || (ldb & 3))
    return cudaErrorInvalidValue;
  CUtensorMap mapA, mapB;
  if (!make_map(&mapA, A, n, a, lda, TM) || !make_map(&mapB, B, n, b, ldb, TN))
    return cudaErrorNotSupported;
  const int na = (a + TM - 1) / TM, nb = (b + TN - 1) / TN;
  if (sym && na != nb) return cudaErrorInvalidValue;
  const int nt = sym ? na * (na + 1) / 2 : na * nb;
  long long nch = std::max<long long>(1, (152 + nt - 1) / nt);
  long long maxch = (n + 4 * BK - 1) / (4 * BK);  // at least 4 stages per CTA
  if (nch > maxch) nch = maxch;
  long long rpc = (n + nch - 1) / nch;
  rpc = (rpc + BK - 1) / BK * BK;
  nch = (n + rpc - 1) / rpc;
  double* part = al.get<double>((size_t)nt * nch * TM * TN);
  cudaError_t e = cudaSuccess;
  if (!part) {
    e = cudaErrorMemoryAllocation;
  } else {
    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
      cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    });
    {
      ProfScope ps(st, "gram_tc");
      k_gram_tc<<<(unsigned)(nt * nch), NTH, SMEM_BYTES, st>>>(mapA, mapB, n, nb, sym ? 1 : 0,
                                                               (int)nch, nt, rpc, a, b, part,
                                                               d_status, probe_spins);
      note_launch();
      k_gram_tc_reduce<<<(unsigned)(nt * TN), TM * RH, 0, st>>>(part, (int)nch, nt, nb, a, b, ma, mb,
                                                            C, ldc, sym ? 1 : 0);
      note_launch();
    }
    e = cudaGetLastError();
  }
  al.put(part);
  return e;
}

}  // namespace sc
