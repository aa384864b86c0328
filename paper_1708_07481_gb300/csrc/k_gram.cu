// Tall-skinny Gram matrices C = A' B (Sec. IV: the Gram products of the n x l multi-vectors
// cost O(n l^2) and take over from the O(n l) vector work as the block widens).
//
// CUDA-core form (SC_PREC_FP32 / SC_PREC_FP64).  Split-K over row chunks: CTA (tile,
// chunk) forms a 64 x 64 tile of A'B over its rows with a 4 x 4 register micro-tile per
// thread (FP32 accumulation for float blocks, FP64 for double), writes the tile as FP64
// partials; a second kernel sums the chunks in fixed chunk order, one thread per output
// element.  The result is deterministic and independent of scheduling.
// The tensor-core form lives in k_gram_tc.cu.
#include <algorithm>

#include "common.cuh"

namespace sc {
namespace {

constexpr int TB = 64;   // output tile
constexpr int RB = 16;   // rows per smem stage
constexpr int NT = 256;  // threads

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

struct ColMap {
  int blk;
  int lc;
};

template <typename T>
__device__ inline void map_cols(const Cat3<T>& M, int c0, ColMap* cm) {
  for (int t = threadIdx.x; t < TB; t += blockDim.x) {
    int c = c0 + t;
    int b = -1, lc = 0;
    int acc = 0;
    for (int q = 0; q < M.nblk; ++q) {
      if (c >= acc && c < acc + M.c[q]) {
        b = q;
        lc = c - acc;
      }
      acc += M.c[q];
    }
    cm[t].blk = b;
    cm[t].lc = lc;
  }
}

template <typename T>
__global__ void __launch_bounds__(NT)
    k_gram(long long n, Cat3<T> A, Cat3<T> B, int nb, int sym, int nch, int ntiles,
           long long rows_per_chunk, double* __restrict__ part) {
  using AT = typename Acc<T>::type;
  __shared__ __align__(16) T As[RB][TB];
  __shared__ __align__(16) T Bs[RB][TB];
  __shared__ ColMap cma[TB], cmb[TB];
  const int tile = blockIdx.x / nch;
  const int chunk = blockIdx.x % nch;
  const int2 tl = tile_coord(tile, nb, sym);
  const int ti = tl.x, tj = tl.y;
  map_cols(A, ti * TB, cma);
  map_cols(B, tj * TB, cmb);
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  AT acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  long long r0 = (long long)chunk * rows_per_chunk;
  long long r1 = r0 + rows_per_chunk;
  if (r1 > n) r1 = n;
  const int lr = threadIdx.x / 16;        // row within the stage
  const int lc = (threadIdx.x % 16) * 4;  // first of 4 columns
  for (long long r = r0; r < r1; r += RB) {
    long long row = r + lr;
    bool ok = row < r1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ColMap ma = cma[lc + q], mb = cmb[lc + q];
      T va = 0, vb = 0;
      if (ok && ma.blk >= 0) va = A.p[ma.blk][row * A.ld[ma.blk] + ma.lc];
      if (ok && mb.blk >= 0) vb = B.p[mb.blk][row * B.ld[mb.blk] + mb.lc];
      As[lr][lc + q] = va;
      Bs[lr][lc + q] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RB; ++k) {
      AT av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = (AT)As[k][ty * 4 + i];
        bv[i] = (AT)Bs[k][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* mine = part + ((long long)chunk * ntiles + tile) * TB * TB;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) mine[(ty * 4 + i) * TB + tx * 4 + j] = (double)acc[i][j];
}

// C[tile element] = sum over chunks in chunk order; one thread per tile element, so the
// chunk loop reads consecutive addresses across a warp.
__global__ void k_gram_reduce(const double* __restrict__ part, int nch, int ntiles, int nb,
                              int a, int b, double* C, int ldc, int sym) {
  long long tot = (long long)ntiles * TB * TB;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < tot;
       g += (long long)gridDim.x * blockDim.x) {
    int tile = (int)(g / (TB * TB));
    int e = (int)(g % (TB * TB));
    int2 tl = tile_coord(tile, nb, sym);
    int gi = tl.x * TB + e / TB, gj = tl.y * TB + e % TB;
    if (gi >= a || gj >= b) continue;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[((long long)c * ntiles + tile) * TB * TB + e];
    C[(long long)gi * ldc + gj] = s;
    if (sym && tl.x != tl.y) C[(long long)gj * ldc + gi] = s;
  }
}

}  // namespace

template <typename T>
cudaError_t gram(cudaStream_t st, Alloc& al, long long n, const Cat3<T>& A, const Cat3<T>& B,
                 double* C, int ldc, bool sym, int use_tc) {
  (void)use_tc;
  int a = A.cols(), b = B.cols();
  if (a == 0 || b == 0) return cudaSuccess;
  if (n == 0) return cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * b, a, st);
  int na = (a + TB - 1) / TB, nb = (b + TB - 1) / TB;
  if (sym && na != nb) return cudaErrorInvalidValue;
  const int nt = sym ? na * (na + 1) / 2 : na * nb;
  // Row chunks: enough CTAs to fill the GPU twice, but at least 512 rows per chunk so the
  // FP64 partial tiles stay small next to the rows they summarise.
  long long target = 152LL * 2;
  long long nch = (target + nt - 1) / nt;
  long long maxch = (n + 511) / 512;
  if (nch > maxch) nch = maxch;
  if (nch < 1) nch = 1;
  long long rpc = (n + nch - 1) / nch;
  rpc = (rpc + RB - 1) / RB * RB;
  nch = (n + rpc - 1) / rpc;
  if (nch < 1) nch = 1;
  double* part = al.get<double>((size_t)nt * nch * TB * TB);
  cudaError_t e = cudaSuccess;
  if (!part) {
    e = cudaErrorMemoryAllocation;
  } else {
    ProfScope ps(st, "gram");
    k_gram<T><<<(unsigned)(nt * nch), NT, 0, st>>>(n, A, B, nb, sym ? 1 : 0, (int)nch, nt, rpc,
                                                   part);
    note_launch();
    long long tot = (long long)nt * TB * TB;
    unsigned rb = (unsigned)std::min<long long>((tot + 255) / 256, 152LL * 8);
    k_gram_reduce<<<rb, 256, 0, st>>>(part, (int)nch, nt, nb, a, b, C, ldc, sym ? 1 : 0);
    note_launch();
    e = cudaGetLastError();
  }
  al.put(part);
  return e;
}

template cudaError_t gram<float>(cudaStream_t, Alloc&, long long, const Cat3<float>&,
                                 const Cat3<float>&, double*, int, bool, int);
template cudaError_t gram<double>(cudaStream_t, Alloc&, long long, const Cat3<double>&,
                                  const Cat3<double>&, double*, int, bool, int);

}  // namespace sc

// ---- Gram without allocation --------------------------------------------------------------
// The split-K partials of sc_gram_static live in this fixed device array instead of memory
// allocated per call.  8 MiB: 64 x 64-tile partials for up to 256 tile-chunk pairs.  Every
// GPU that loads the library keeps it until exit.
#include <mutex>

#include "../../include/sc.h"

namespace sc {
namespace {
constexpr size_t GRAM_STATIC_DOUBLES = (size_t)1 << 20;  // 8 MiB
static __device__ __align__(256) double g_gram_static[GRAM_STATIC_DOUBLES];
// the largest block pair (1024 x 1024 columns: 16 x 16 tiles) still gets one row chunk per
// tile, which the chunk clamp below relies on
static_assert((size_t)((SC_GRAM_STATIC_MAX_COLS + TB - 1) / TB) *
                      ((SC_GRAM_STATIC_MAX_COLS + TB - 1) / TB) * TB * TB <=
                  GRAM_STATIC_DOUBLES,
              "static Gram scratch too small for one chunk per tile");

// Device address of g_gram_static for the current device, looked up once per device (the
// host-side name of the array is only a stand-in, never a device address).
double* gram_static_addr(int dev) {
  static std::mutex mu;
  static double* addr[64] = {nullptr};
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gram_static) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    addr[dev] = (double*)p;
  }
  return addr[dev];
}
}  // namespace
}  // namespace sc

extern "C" int sc_gram_static(int64_t n, int a, int b, const float* A, int64_t lda,
                              const float* B, int64_t ldb, double* C, void* cuda_stream) {
  using namespace sc;
  if (n < 0 || a < 1 || b < 1 || a > SC_GRAM_STATIC_MAX_COLS || b > SC_GRAM_STATIC_MAX_COLS ||
      lda < a || ldb < b || !A || !B || !C)
    return SC_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SC_ECUDA;
  double* scratch = gram_static_addr(dev);
  if (!scratch) return SC_ECUDA;
  if (n == 0) {
    return cudaMemset2DAsync(C, sizeof(double) * b, 0, sizeof(double) * b, a, st) == cudaSuccess
               ? SC_OK
               : SC_ECUDA;
  }
  const int na = (a + TB - 1) / TB, nb = (b + TB - 1) / TB;
  const int nt = na * nb;  // <= 16 x 16 = 256 tiles
  // chunks: fill the GPU, at least 512 rows each, and fit the partials in the array
  const long long cap_pairs = (long long)GRAM_STATIC_DOUBLES / (TB * TB);
  long long nch = (152LL * 2 + nt - 1) / nt;
  long long maxch = (n + 511) / 512;
  if (nch > maxch) nch = maxch;
  if (nch * nt > cap_pairs) nch = cap_pairs / nt;
  if (nch < 1) nch = 1;
  long long rpc = (n + nch - 1) / nch;
  rpc = (rpc + RB - 1) / RB * RB;
  nch = (n + rpc - 1) / rpc;
  double* part = scratch;
  // the partials need no clearing (the array keeps the previous call's contents): every entry
  // the reduction reads is written by this call
  Cat3<float> ca = cat<float>(A, lda, a), cb = cat<float>(B, ldb, b);
  k_gram<float><<<(unsigned)(nt * nch), NT, 0, st>>>(n, ca, cb, nb, 0, (int)nch, nt, rpc, part);
  note_launch();
  long long tot = (long long)nt * TB * TB;
  unsigned rb = (unsigned)std::min<long long>((tot + 255) / 256, 152LL * 8);
  k_gram_reduce<<<rb, 256, 0, st>>>(part, (int)nch, nt, nb, a, b, C, b, 0);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SC_OK : SC_ECUDA;
}
