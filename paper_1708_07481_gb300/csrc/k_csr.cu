// Laplacian build (Sec. II.A symmetrization W <- W + W', Sec. III sparse adjacency): a directed
// edge list becomes the CSR of the symmetrized adjacency W plus the degrees D of L = D - W.
//
// Pipeline (all on the device, integer-exact and deterministic):
//   1. count both directions of every non-loop edge per row (atomics on row counters);
//   2. exclusive scan -> per-row slots; scatter 64-bit keys (col << 32 | weight bits);
//   3. sort every row's keys (bitonic in shared memory; rows longer than the shared
//      capacity are merge-sorted by one CTA through a global ping-pong buffer);
//   4. merge equal columns (logical: one entry of weight 1; algebraic: FP64 sum of the
//      weights in sorted order) into a unique list per row;
//   5. scan the unique counts -> row_ptr; compact; deg = FP64 row sums.
// Because duplicate weights are summed in key order, the result does not depend on the
// order in which atomics placed them.
#include <cfloat>
#include <climits>

#include "common.cuh"

namespace sc {
namespace {

constexpr int SORT_CAP = 2048;  // keys per row sorted in shared memory by one CTA
constexpr int SORT_THREADS = 256;
constexpr unsigned long long KEY_MAX = ~0ull;

__global__ void k_count(long long m, int n, const int* __restrict__ src,
                        const int* __restrict__ dst, int* cnt, int* status) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x) {
    int u = src[e], v = dst[e];
    if ((unsigned)u >= (unsigned)n || (unsigned)v >= (unsigned)n) {
      atomicOr(status, ST_EDGE_RANGE);
      continue;
    }
    if (u == v) continue;
    atomicAdd(&cnt[u], 1);
    atomicAdd(&cnt[v], 1);
  }
}

__global__ void k_scatter(long long m, int n, const int* __restrict__ src,
                          const int* __restrict__ dst, const float* __restrict__ w,
                          const long long* __restrict__ tptr, int* fill,
                          unsigned long long* tkey) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m;
       e += (long long)gridDim.x * blockDim.x) {
    int u = src[e], v = dst[e];
    if ((unsigned)u >= (unsigned)n || (unsigned)v >= (unsigned)n || u == v) continue;
    unsigned long long wb = w ? (unsigned long long)__float_as_uint(w[e]) : 0ull;
    long long pu = tptr[u] + atomicAdd(&fill[u], 1);
    tkey[pu] = ((unsigned long long)(unsigned)v << 32) | wb;
    long long pv = tptr[v] + atomicAdd(&fill[v], 1);
    tkey[pv] = ((unsigned long long)(unsigned)u << 32) | wb;
  }
}

// ---- device-wide exclusive scan of int counts into long long offsets (out[n] = total) ----
constexpr int SCAN_BLOCK = 1024;

__device__ long long block_excl_scan(long long v, long long* sh, long long* total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long s = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  long long base = wid > 0 ? sh[wid - 1] : 0;
  long long incl = x + base;
  if (total) *total = sh[nw - 1];
  __syncthreads();
  return incl - v;
}

template <typename Tin>
__global__ void k_scan_local(long long n, const Tin* __restrict__ in, long long* out,
                             long long* bsum) {
  __shared__ long long sh[32];
  long long i = blockIdx.x * (long long)SCAN_BLOCK + threadIdx.x;
  long long v = i < n ? (long long)in[i] : 0;
  long long tot;
  long long ex = block_excl_scan(v, sh, &tot);
  if (i < n) out[i] = ex;
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_bsum(long long nb, long long* bsum, long long* total) {
  __shared__ long long sh[32];
  long long carry = 0;
  for (long long base = 0; base < nb; base += SCAN_BLOCK) {
    long long i = base + threadIdx.x;
    long long v = i < nb ? bsum[i] : 0;
    long long tot;
    long long ex = block_excl_scan(v, sh, &tot);
    if (i < nb) bsum[i] = ex + carry;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(long long n, long long* out, const long long* bsum,
                           const long long* total) {
  long long i = blockIdx.x * (long long)SCAN_BLOCK + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
  if (i == 0) out[n] = *total;
}

template <typename Tin>
cudaError_t scan_excl(cudaStream_t st, Alloc& al, long long n, const Tin* in, long long* out) {
  long long nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  if (nb == 0) nb = 1;
  long long* bsum = al.get<long long>(nb + 1);
  if (!bsum) return cudaErrorMemoryAllocation;
  k_scan_local<Tin><<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(n, in, out, bsum);
  note_launch();
  k_scan_bsum<<<1, SCAN_BLOCK, 0, st>>>(nb, bsum, bsum + nb);
  note_launch();
  k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(n, out, bsum, bsum + nb);
  note_launch();
  cudaError_t e = cudaGetLastError();
  al.put(bsum);
  return e;
}

// ---- per-row sort + merge of duplicate columns ---------------------------------------------

__device__ void bitonic_sort(unsigned long long* a, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long x = a[i], y = a[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Merge runs of equal column in sorted keys a[0..len) into out (unique, summed weights).
// Returns the unique count (valid in every thread).  `flags` is shared scratch of >= len+1
// ints when `flags_shared`, else a global region of the same size.
__device__ int dedup_sorted(const unsigned long long* a, int len, unsigned long long* out,
                            int algebraic, int* pos, long long* sh) {
  int base = 0;
  int chunk = blockDim.x;
  for (int s = 0; s < len; s += chunk) {
    int i = s + threadIdx.x;
    int head = 0;
    if (i < len) head = (i == 0) || ((a[i] >> 32) != (a[i - 1] >> 32));
    long long tot;
    long long ex = block_excl_scan(head, sh, &tot);
    if (i < len && head) pos[i] = base + (int)ex;
    base += (int)tot;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    bool head = (i == 0) || ((a[i] >> 32) != (a[i - 1] >> 32));
    if (!head) continue;
    unsigned long long col = a[i] >> 32;
    float wv = 1.0f;
    if (algebraic) {
      double s = 0.0;
      for (int j = i; j < len && (a[j] >> 32) == col; ++j)
        s += (double)__uint_as_float((unsigned)(a[j] & 0xffffffffull));
      wv = (float)s;
    }
    out[pos[i]] = (col << 32) | (unsigned long long)__float_as_uint(wv);
  }
  __syncthreads();
  return base;
}

__global__ void __launch_bounds__(SORT_THREADS)
    k_sort_rows(int n, const long long* __restrict__ tptr, const unsigned long long* tkey,
                unsigned long long* ukey, int* ucnt, int* longrows, int* nlong, int algebraic) {
  __shared__ unsigned long long a[SORT_CAP];
  __shared__ unsigned long long o[SORT_CAP];
  __shared__ int pos[SORT_CAP];
  __shared__ long long sh[32];
  for (int row = blockIdx.x; row < n; row += gridDim.x) {
    long long s0 = tptr[row];
    int len = (int)(tptr[row + 1] - s0);
    if (len > SORT_CAP) {
      if (threadIdx.x == 0) longrows[atomicAdd(nlong, 1)] = row;
      continue;
    }
    if (len == 0) {
      if (threadIdx.x == 0) ucnt[row] = 0;
      continue;
    }
    int P = 1;
    while (P < len) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) a[i] = i < len ? tkey[s0 + i] : KEY_MAX;
    __syncthreads();
    bitonic_sort(a, P);
    int u = dedup_sorted(a, len, o, algebraic, pos, sh);
    for (int i = threadIdx.x; i < u; i += blockDim.x) ukey[s0 + i] = o[i];
    if (threadIdx.x == 0) ucnt[row] = u;
    __syncthreads();
  }
}

// One CTA per long row: bitonic-sort chunks of SORT_CAP in shared memory, then merge runs
// pairwise through the row's own region of `scr` (same indexing as tkey), then dedup.
__global__ void __launch_bounds__(SORT_THREADS)
    k_sort_long(const int* longrows, const long long* __restrict__ tptr,
                unsigned long long* tkey, unsigned long long* scr, unsigned long long* ukey,
                int* ucnt, int* posbuf, int algebraic) {
  __shared__ unsigned long long a[SORT_CAP];
  __shared__ long long sh[32];
  int row = longrows[blockIdx.x];
  long long s0 = tptr[row];
  int len = (int)(tptr[row + 1] - s0);
  unsigned long long* src = tkey + s0;
  unsigned long long* dst = scr + s0;
  for (int c = 0; c < len; c += SORT_CAP) {
    int cl = min(SORT_CAP, len - c);
    for (int i = threadIdx.x; i < SORT_CAP; i += blockDim.x) a[i] = i < cl ? src[c + i] : KEY_MAX;
    __syncthreads();
    bitonic_sort(a, SORT_CAP);
    for (int i = threadIdx.x; i < cl; i += blockDim.x) src[c + i] = a[i];
    __syncthreads();
  }
  for (int w = SORT_CAP; w < len; w <<= 1) {
    for (int s = 0; s < len; s += 2 * w) {
      int la = min(w, len - s);
      int lb = max(0, min(w, len - s - w));
      const unsigned long long* A = src + s;
      const unsigned long long* B = src + s + la;
      for (int p = threadIdx.x; p < la + lb; p += blockDim.x) {
        // co-rank: i elements of A and p - i of B precede output p
        int lo = max(0, p - lb), hi = min(p, la);
        while (lo < hi) {
          int i = (lo + hi) >> 1;
          if (A[i] <= B[p - i - 1]) lo = i + 1;
          else hi = i;
        }
        int i = lo, j = p - lo;
        unsigned long long v;
        if (i < la && (j >= lb || A[i] <= B[j])) v = A[i];
        else v = B[j];
        dst[s + p] = v;
      }
    }
    __syncthreads();
    unsigned long long* t = src;
    src = dst;
    dst = t;
  }
  // src holds the sorted row; dedup into ukey (positions scratch in posbuf at s0)
  int base = 0;
  for (int s = 0; s < len; s += blockDim.x) {
    int i = s + threadIdx.x;
    int head = 0;
    if (i < len) head = (i == 0) || ((src[i] >> 32) != (src[i - 1] >> 32));
    long long tot;
    long long ex = block_excl_scan(head, sh, &tot);
    if (i < len && head) posbuf[s0 + i] = base + (int)ex;
    base += (int)tot;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    bool head = (i == 0) || ((src[i] >> 32) != (src[i - 1] >> 32));
    if (!head) continue;
    unsigned long long col = src[i] >> 32;
    float wv = 1.0f;
    if (algebraic) {
      double s = 0.0;
      for (int j = i; j < len && (src[j] >> 32) == col; ++j)
        s += (double)__uint_as_float((unsigned)(src[j] & 0xffffffffull));
      wv = (float)s;
    }
    ukey[s0 + posbuf[s0 + i]] = (col << 32) | (unsigned long long)__float_as_uint(wv);
  }
  if (threadIdx.x == 0) ucnt[row] = base;
}

__global__ void k_rowptr32(int n, const long long* __restrict__ rp64, int* rp, int* status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= n;
       i += (long long)gridDim.x * blockDim.x) {
    long long v = rp64[i];
    if (v > INT_MAX) {
      atomicOr(status, ST_NNZ_OVERFLOW);
      v = INT_MAX;
    }
    rp[i] = (int)v;
  }
}

// Warp per row: copy the unique keys to col_idx/val and sum the row (deg, FP64).
__global__ void k_compact(int n, const long long* __restrict__ tptr,
                          const unsigned long long* __restrict__ ukey,
                          const int* __restrict__ rp, int* col, float* val, float* degf,
                          double* degd, int algebraic) {
  int lane = threadIdx.x & 31;
  long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long row = wid; row < n; row += nwarps) {
    long long s0 = tptr[row];
    int o = rp[row];
    int len = rp[row + 1] - o;
    double s = 0.0;
    for (int i = lane; i < len; i += 32) {
      unsigned long long k = ukey[s0 + i];
      col[o + i] = (int)(k >> 32);
      float wv = __uint_as_float((unsigned)(k & 0xffffffffull));
      if (algebraic) {
        val[o + i] = wv;
        s += (double)wv;
      } else {
        s += 1.0;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
      degd[row] = s;
      degf[row] = (float)s;
    }
  }
}

__global__ void k_max(int n, const double* __restrict__ x, double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) v = fmax(v, x[i]);
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) *out = v;
  }
}

// ---- merge of two CSRs (streaming update) -------------------------------------------------

__device__ inline int row_len(const CsrDev& g, int r) {
  return r < g.n ? g.row_ptr[r + 1] - g.row_ptr[r] : 0;
}

__global__ void k_merge_count(int n, CsrDev a, CsrDev b, int* cnt) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    int la = row_len(a, (int)r), lb = row_len(b, (int)r);
    const int* A = la ? a.col_idx + a.row_ptr[r] : nullptr;
    const int* B = lb ? b.col_idx + b.row_ptr[r] : nullptr;
    int i = 0, j = 0, c = 0;
    while (i < la || j < lb) {
      if (j >= lb || (i < la && A[i] < B[j])) ++i;
      else if (i >= la || B[j] < A[i]) ++j;
      else { ++i; ++j; }
      ++c;
    }
    cnt[r] = c;
  }
}

__global__ void k_merge_fill(int n, CsrDev a, CsrDev b, const long long* __restrict__ rp,
                             int* col, float* val, float* degf, double* degd, int algebraic) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    int la = row_len(a, (int)r), lb = row_len(b, (int)r);
    const int* A = la ? a.col_idx + a.row_ptr[r] : nullptr;
    const int* B = lb ? b.col_idx + b.row_ptr[r] : nullptr;
    const float* Av = (la && a.val) ? a.val + a.row_ptr[r] : nullptr;
    const float* Bv = (lb && b.val) ? b.val + b.row_ptr[r] : nullptr;
    long long o = rp[r];
    int i = 0, j = 0;
    double s = 0.0;
    while (i < la || j < lb) {
      int c;
      double wv;
      if (j >= lb || (i < la && A[i] < B[j])) {
        c = A[i]; wv = Av ? (double)Av[i] : 1.0; ++i;
      } else if (i >= la || B[j] < A[i]) {
        c = B[j]; wv = Bv ? (double)Bv[j] : 1.0; ++j;
      } else {
        c = A[i];
        wv = algebraic ? (double)(Av ? Av[i] : 1.0f) + (double)(Bv ? Bv[j] : 1.0f) : 1.0;
        ++i; ++j;
      }
      col[o] = c;
      float wf = algebraic ? (float)wv : 1.0f;
      if (algebraic) val[o] = wf;
      s += algebraic ? (double)wf : 1.0;
      ++o;
    }
    degd[r] = s;
    degf[r] = (float)s;
  }
}

inline unsigned grid_for(long long work, int threads, int cap = 152 * 32) {
  long long g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

cudaError_t build_csr(cudaStream_t st, Alloc& al, int n, long long m, const int* d_src,
                      const int* d_dst, const float* d_w, int algebraic, int* d_status,
                      CsrDev* out, int* host_status) {
  cudaError_t e = cudaSuccess;
  *out = CsrDev{};
  out->n = n;
  int* cnt = al.get<int>((size_t)n * 2 + 2);
  long long* tptr = al.get<long long>((size_t)n + 1);
  long long* rp64 = al.get<long long>((size_t)n + 1);
  long long tot2 = 2 * (m > 0 ? m : 1);
  unsigned long long* tkey = al.get<unsigned long long>((size_t)tot2);
  unsigned long long* ukey = al.get<unsigned long long>((size_t)tot2);
  int* longrows = al.get<int>((size_t)n + 1);
  int* misc = al.get<int>(8);
  double* dmax = al.get<double>(1);
  int* ucnt = cnt + n + 1;
  int* fill = cnt;
  if (!cnt || !tptr || !rp64 || !tkey || !ukey || !longrows || !misc || !dmax) {
    e = cudaErrorMemoryAllocation;
    goto done;
  }
  cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)n * 2 + 2), st);
  cudaMemsetAsync(misc, 0, sizeof(int) * 8, st);
  if (m > 0) {
    k_count<<<grid_for(m, 256), 256, 0, st>>>(m, n, d_src, d_dst, cnt, d_status);
    note_launch();
  }
  if ((e = scan_excl<int>(st, al, n, cnt, tptr)) != cudaSuccess) goto done;
  cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)n, st);
  if (m > 0) {
    k_scatter<<<grid_for(m, 256), 256, 0, st>>>(m, n, d_src, d_dst, algebraic ? d_w : nullptr,
                                                  tptr, fill, tkey);
    note_launch();
  }
  k_sort_rows<<<grid_for(n, 1, 152 * 8), SORT_THREADS, 0, st>>>(n, tptr, tkey, ukey, ucnt,
                                                                 longrows, misc, algebraic);
  note_launch();
  {
    int nlong = 0;
    cudaMemcpyAsync(&nlong, misc, sizeof(int), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto done;
    if (nlong > 0) {
      unsigned long long* scr = al.get<unsigned long long>((size_t)tot2);
      int* posbuf = al.get<int>((size_t)tot2);
      if (!scr || !posbuf) {
        al.put(scr);
        al.put(posbuf);
        e = cudaErrorMemoryAllocation;
        goto done;
      }
      k_sort_long<<<nlong, SORT_THREADS, 0, st>>>(longrows, tptr, tkey, scr, ukey, ucnt,
                                                   posbuf, algebraic);
      note_launch();
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto done;
      al.put(scr);
      al.put(posbuf);
    }
  }
  if ((e = scan_excl<int>(st, al, n, ucnt, rp64)) != cudaSuccess) goto done;
  {
    long long nnz = 0;
    cudaMemcpyAsync(&nnz, rp64 + n, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto done;
    if (nnz > INT_MAX) {
      *host_status |= ST_NNZ_OVERFLOW;
      goto done;
    }
    out->nnz = nnz;
    out->row_ptr = al.get<int>((size_t)n + 1);
    out->col_idx = al.get<int>((size_t)(nnz > 0 ? nnz : 1));
    out->val = algebraic ? al.get<float>((size_t)(nnz > 0 ? nnz : 1)) : nullptr;
    out->degf = al.get<float>((size_t)n);
    out->degd = al.get<double>((size_t)n);
    if (!out->row_ptr || !out->col_idx || (algebraic && !out->val) || !out->degf || !out->degd) {
      e = cudaErrorMemoryAllocation;
      goto done;
    }
    k_rowptr32<<<grid_for(n + 1, 256), 256, 0, st>>>(n, rp64, out->row_ptr, d_status);
    note_launch();
    k_compact<<<grid_for((long long)n * 32, 256), 256, 0, st>>>(
        n, tptr, ukey, out->row_ptr, out->col_idx, out->val, out->degf, out->degd, algebraic);
    note_launch();
    k_max<<<1, 1024, 0, st>>>(n, out->degd, dmax);
    note_launch();
    int hs = 0;
    cudaMemcpyAsync(&out->deg_max, dmax, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&hs, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto done;
    *host_status |= hs;
  }
done:
  al.put(cnt);
  al.put(tptr);
  al.put(rp64);
  al.put(tkey);
  al.put(ukey);
  al.put(longrows);
  al.put(misc);
  al.put(dmax);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

cudaError_t merge_csr(cudaStream_t st, Alloc& al, const CsrDev& a, const CsrDev& b,
                      int algebraic, int* d_status, CsrDev* out, int* host_status) {
  (void)d_status;
  cudaError_t e = cudaSuccess;
  int n = b.n;
  *out = CsrDev{};
  out->n = n;
  int* cnt = al.get<int>((size_t)n + 1);
  long long* rp64 = al.get<long long>((size_t)n + 1);
  double* dmax = al.get<double>(1);
  if (!cnt || !rp64 || !dmax) {
    e = cudaErrorMemoryAllocation;
    goto done;
  }
  k_merge_count<<<grid_for(n, 128), 128, 0, st>>>(n, a, b, cnt);
  note_launch();
  if ((e = scan_excl<int>(st, al, n, cnt, rp64)) != cudaSuccess) goto done;
  {
    long long nnz = 0;
    cudaMemcpyAsync(&nnz, rp64 + n, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto done;
    if (nnz > INT_MAX) {
      *host_status |= ST_NNZ_OVERFLOW;
      goto done;
    }
    out->nnz = nnz;
    out->row_ptr = al.get<int>((size_t)n + 1);
    out->col_idx = al.get<int>((size_t)(nnz > 0 ? nnz : 1));
    out->val = algebraic ? al.get<float>((size_t)(nnz > 0 ? nnz : 1)) : nullptr;
    out->degf = al.get<float>((size_t)n);
    out->degd = al.get<double>((size_t)n);
    if (!out->row_ptr || !out->col_idx || (algebraic && !out->val) || !out->degf || !out->degd) {
      e = cudaErrorMemoryAllocation;
      goto done;
    }
    k_rowptr32<<<grid_for(n + 1, 256), 256, 0, st>>>(n, rp64, out->row_ptr, d_status);
    note_launch();
    k_merge_fill<<<grid_for(n, 128), 128, 0, st>>>(n, a, b, rp64, out->col_idx, out->val,
                                                    out->degf, out->degd, algebraic);
    note_launch();
    k_max<<<1, 1024, 0, st>>>(n, out->degd, dmax);
    note_launch();
    cudaMemcpyAsync(&out->deg_max, dmax, sizeof(double), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto done;
  }
done:
  al.put(cnt);
  al.put(rp64);
  al.put(dmax);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace sc
