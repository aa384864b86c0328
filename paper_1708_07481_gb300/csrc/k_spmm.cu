// SpMM with the graph Laplacian: Y = D V - W V for a row-major n x k block V (Sec. III:
// LOBPCG needs one multiplication of the graph matrix by a multi-vector per iteration).
//
// A team of TL lanes owns one row; each lane owns 16-byte column chunks (float4 / double2)
// c = lane, lane + TL, ...  The team loads TL neighbour indices at once (one per lane) and
// broadcasts them with shuffles, so every gathered neighbour row is read as consecutive
// 16-byte vectors.  TL is picked from the block width so idle lanes stay few.
// HBM/L2-bound: per row, 4 bytes of index per neighbour plus k * sizeof(T) bytes of the
// neighbour's row (served from L2 when the block fits there), and the row's own V/Y rows.
#include <algorithm>

#include "common.cuh"

namespace sc {
namespace {

template <typename T> struct Vec;
template <> struct Vec<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static void fma(float4& a, float w, const float4& x) {
    a.x = fmaf(w, x.x, a.x); a.y = fmaf(w, x.y, a.y); a.z = fmaf(w, x.z, a.z); a.w = fmaf(w, x.w, a.w);
  }
  __device__ static void add(float4& a, const float4& x) {
    a.x += x.x; a.y += x.y; a.z += x.z; a.w += x.w;
  }
  __device__ static float4 lap(float d, const float4& v, const float4& s) {
    return make_float4(fmaf(d, v.x, -s.x), fmaf(d, v.y, -s.y), fmaf(d, v.z, -s.z), fmaf(d, v.w, -s.w));
  }
};
template <> struct Vec<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static void fma(double2& a, double w, const double2& x) {
    a.x = fma_(w, x.x, a.x); a.y = fma_(w, x.y, a.y);
  }
  __device__ static double fma_(double a, double b, double c) { return ::fma(a, b, c); }
  __device__ static void add(double2& a, const double2& x) { a.x += x.x; a.y += x.y; }
  __device__ static double2 lap(double d, const double2& v, const double2& s) {
    return make_double2(::fma(d, v.x, -s.x), ::fma(d, v.y, -s.y));
  }
};

constexpr int MAXC = 4;  // chunks per lane: TL=32 x 4 chunks x 4 floats = 512 columns

// NC = 16-byte chunks per lane (compile time).  Neighbours are processed four at a time with
// all of their row loads issued before the first accumulation, so each lane keeps 4 * NC
// gathers in flight instead of one.  The neighbours of a row are summed in CSR order whatever
// TL and NC are, so every kernel shape gives the same bits.
template <typename T, int TL, int NC>
__device__ __forceinline__ void spmm_row(long long row, int lane, unsigned gmask,
                                         const int* __restrict__ rp, const int* __restrict__ ci,
                                         const float* __restrict__ val, const T* __restrict__ deg,
                                         const T* __restrict__ V, long long ldv,
                                         T* __restrict__ Y, long long ldy, int nvec) {
  using V4 = typename Vec<T>::type;
  bool act[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) act[c] = lane + c * TL < nvec;
  V4 acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = Vec<T>::zero();
  const int s = rp[row], e = rp[row + 1];
  for (int base = s; base < e; base += TL) {
    const int my = base + lane < e ? ci[base + lane] : 0;
    const float mw = (val && base + lane < e) ? val[base + lane] : 1.0f;
    const int cnt = min(TL, e - base);
    int t = 0;
    for (; t + 4 <= cnt; t += 4) {
      int j[4];
      T w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        j[u] = __shfl_sync(gmask, my, t + u, TL);
        w[u] = (T)__shfl_sync(gmask, mw, t + u, TL);
      }
      V4 x[4][NC];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const V4* vr = reinterpret_cast<const V4*>(V + (long long)j[u] * ldv);
#pragma unroll
        for (int c = 0; c < NC; ++c) x[u][c] = act[c] ? __ldg(vr + lane + c * TL) : Vec<T>::zero();
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (val) Vec<T>::fma(acc[c], w[u], x[u][c]);
          else Vec<T>::add(acc[c], x[u][c]);
        }
    }
    for (; t < cnt; ++t) {
      const int jj = __shfl_sync(gmask, my, t, TL);
      const T ww = (T)__shfl_sync(gmask, mw, t, TL);
      const V4* vr = reinterpret_cast<const V4*>(V + (long long)jj * ldv);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (act[c]) {
          V4 x = __ldg(vr + lane + c * TL);
          if (val) Vec<T>::fma(acc[c], ww, x);
          else Vec<T>::add(acc[c], x);
        }
      }
    }
  }
  const T d = deg[row];
  const V4* vi = reinterpret_cast<const V4*>(V + row * ldv);
  V4* yo = reinterpret_cast<V4*>(Y + row * ldy);
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (act[c]) yo[lane + c * TL] = Vec<T>::lap(d, vi[lane + c * TL], acc[c]);
}

template <int TL>
__device__ __forceinline__ unsigned team_mask() {
  return (TL == 32) ? 0xffffffffu : (((1u << TL) - 1u) << ((threadIdx.x & 31) / TL * TL));
}

template <typename T, int TL, int NC>
__global__ void __launch_bounds__(256)
    k_spmm(int n, const int* __restrict__ rp, const int* __restrict__ ci,
           const float* __restrict__ val, const T* __restrict__ deg, const T* __restrict__ V,
           long long ldv, T* __restrict__ Y, long long ldy, int nvec) {
  const int lane = threadIdx.x % TL;
  const unsigned gmask = team_mask<TL>();
  long long team = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / TL;
  long long nteams = ((long long)gridDim.x * blockDim.x) / TL;
  for (long long row = team; row < n; row += nteams)
    spmm_row<T, TL, NC>(row, lane, gmask, rp, ci, val, deg, V, ldv, Y, ldy, nvec);
}

// Lockstep batch (FP32): the rows of every graph of the descriptor table form one range that
// the teams stride through; a team's rows only grow, so it finds each row's graph by moving
// forward through the table (descriptors in row0 order).
template <int TL, int NC>
__global__ void __launch_bounds__(256)
    k_spmm_b(const SpmmDesc* __restrict__ tab, int count, long long rows) {
  const int lane = threadIdx.x % TL;
  const unsigned gmask = team_mask<TL>();
  long long team = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / TL;
  long long nteams = ((long long)gridDim.x * blockDim.x) / TL;
  int q = 0;
  for (long long grow = team; grow < rows; grow += nteams) {
    while (q + 1 < count && tab[q + 1].row0 <= grow) ++q;
    const SpmmDesc& a = tab[q];
    spmm_row<float, TL, NC>(grow - a.row0, lane, gmask, a.rp, a.ci, a.val, a.deg, a.V, a.ldv,
                            a.Y, a.ldy, a.nvec);
  }
}

template <typename T, int TL, int NC>
cudaError_t launch(cudaStream_t st, const CsrDev& g, const T* deg, const T* V, long long ldv,
                   T* Y, long long ldy, int nvec) {
  long long teams = g.n;
  long long threads = teams * TL;
  long long blocks = (threads + 255) / 256;
  long long cap = 152LL * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ProfScope ps(st, "spmm");
  k_spmm<T, TL, NC><<<(unsigned)blocks, 256, 0, st>>>(g.n, g.row_ptr, g.col_idx, g.val, deg, V,
                                                     ldv, Y, ldy, nvec);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

// Kernel shapes the autotuner chooses among: (lanes per row, 16-byte chunks per lane).
struct SpmmShape {
  int tl, nc;
};
constexpr SpmmShape kSpmmShapes[] = {{4, 1},  {8, 1},  {16, 1}, {32, 1}, {8, 2},
                                     {16, 2}, {32, 2}, {8, 3},  {16, 3}, {32, 3},
                                     {8, 4},  {16, 4}, {32, 4}};
constexpr int kNumSpmmShapes = sizeof(kSpmmShapes) / sizeof(kSpmmShapes[0]);

template <typename T>
cudaError_t launch_shape(int v, cudaStream_t st, const CsrDev& g, const T* deg, const T* V,
                         long long ldv, T* Y, long long ldy, int nvec) {
  switch (v) {
    case 0: return launch<T, 4, 1>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 1: return launch<T, 8, 1>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 2: return launch<T, 16, 1>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 3: return launch<T, 32, 1>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 4: return launch<T, 8, 2>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 5: return launch<T, 16, 2>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 6: return launch<T, 32, 2>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 7: return launch<T, 8, 3>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 8: return launch<T, 16, 3>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 9: return launch<T, 32, 3>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 10: return launch<T, 8, 4>(st, g, deg, V, ldv, Y, ldy, nvec);
    case 11: return launch<T, 16, 4>(st, g, deg, V, ldv, Y, ldy, nvec);
    default: return launch<T, 32, 4>(st, g, deg, V, ldv, Y, ldy, nvec);
  }
}

// The kernel shapes that fit nvec 16-byte column chunks with no wholly idle chunk per lane;
// out[0] is the built-in default (the smallest team that covers the row with one chunk, then
// 32 lanes with as many chunks as needed).
int spmm_shapes(int nvec, int* out) {
  int cnt = 0, def = -1;
  if (nvec <= 4) def = 0;
  else if (nvec <= 8) def = 1;
  else if (nvec <= 16) def = 2;
  else if (nvec <= 32) def = 3;
  else if (nvec <= 64) def = 6;
  else if (nvec <= 96) def = 9;
  else def = 12;
  out[cnt++] = def;
  for (int v = 0; v < kNumSpmmShapes; ++v) {
    const SpmmShape sh = kSpmmShapes[v];
    if (v == def || sh.tl * sh.nc < nvec || sh.tl * (sh.nc - 1) >= nvec) continue;
    out[cnt++] = v;
  }
  return cnt;
}

template <typename T>
cudaError_t spmm_lap(cudaStream_t st, const CsrDev& g, const T* V, long long ldv, T* Y,
                     long long ldy, int k, int shape) {
  constexpr int W = Vec<T>::W;
  if (ldv % W || ldy % W) return cudaErrorInvalidValue;
  int nvec = (k + W - 1) / W;
  if (nvec > 32 * MAXC) {  // wider blocks: column chunks of the widest kernel shape
    const int kc = 32 * MAXC * W;
    for (int c0 = 0; c0 < k; c0 += kc) {
      cudaError_t e = spmm_lap<T>(st, g, V + c0, ldv, Y + c0, ldy, std::min(kc, k - c0), -1);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const T* deg;
  if constexpr (sizeof(T) == 4) deg = (const T*)g.degf;
  else deg = (const T*)g.degd;
  if (g.n == 0) return cudaSuccess;
  if (shape < 0 || shape >= kNumSpmmShapes ||
      kSpmmShapes[shape].tl * kSpmmShapes[shape].nc < nvec) {
    int list[kNumSpmmShapes];
    spmm_shapes(nvec, list);
    shape = list[0];
  }
  return launch_shape<T>(shape, st, g, deg, V, ldv, Y, ldy, nvec);
}

template <int TL, int NC>
static cudaError_t launch_b(cudaStream_t st, const SpmmDesc* dtab, int count, long long rows) {
  long long blocks = (rows * TL + 255) / 256;
  const long long cap = 152LL * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  ProfScope ps(st, "spmm");
  k_spmm_b<TL, NC><<<(unsigned)blocks, 256, 0, st>>>(dtab, count, rows);
  note_launch();
  return cudaGetLastError();
}

// One launch for the SpMM of every graph of a lockstep batch, with the default kernel shape
// of the widest block (nvec_max <= 128 chunks).
cudaError_t spmm_batch_launch(cudaStream_t st, const SpmmDesc* dtab, int count, long long rows,
                              int nvec_max) {
  if (count <= 0 || rows <= 0) return cudaSuccess;
  if (nvec_max > 32 * MAXC) return cudaErrorInvalidValue;
  if (nvec_max <= 4) return launch_b<4, 1>(st, dtab, count, rows);
  if (nvec_max <= 8) return launch_b<8, 1>(st, dtab, count, rows);
  if (nvec_max <= 16) return launch_b<16, 1>(st, dtab, count, rows);
  if (nvec_max <= 32) return launch_b<32, 1>(st, dtab, count, rows);
  if (nvec_max <= 64) return launch_b<32, 2>(st, dtab, count, rows);
  if (nvec_max <= 96) return launch_b<32, 3>(st, dtab, count, rows);
  return launch_b<32, 4>(st, dtab, count, rows);
}

template cudaError_t spmm_lap<float>(cudaStream_t, const CsrDev&, const float*, long long,
                                     float*, long long, int, int);
template cudaError_t spmm_lap<double>(cudaStream_t, const CsrDev&, const double*, long long,
                                      double*, long long, int, int);

}  // namespace sc
