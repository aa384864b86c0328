// C ABI of the library (include/sc.h): contexts, graphs, the LOBPCG driver, k-means,
// the end-to-end partition and streaming updates.  Host code only orchestrates: every
// arithmetic step runs in the kernels of k_*.cu on the context stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/sc.h"
#include "common.cuh"

// ---------------------------------------------------------------------------------------
namespace sc {
static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// Event-pair profiler (process-wide): the kernels named in the filter ("*" = all) get an
// event pair around every launch; sc_profile_end sums the pairs per kernel name.
struct ProfState {
  std::mutex mu;
  bool on = false;
  std::string filter;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> recs;
  std::unordered_map<std::string, cudaEvent_t> pending;
};
static ProfState g_prof;
static cudaEvent_t prof_event() {
  if (g_prof.used == g_prof.pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g_prof.pool.push_back(e);
  }
  return g_prof.pool[g_prof.used++];
}
static bool prof_match(const char* name) {
  if (!g_prof.on) return false;
  if (g_prof.filter == "*") return true;
  std::string f = "," + g_prof.filter + ",";
  return f.find("," + std::string(name) + ",") != std::string::npos;
}
void prof_begin(cudaStream_t st, const char* name) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!prof_match(name)) return;
  cudaEvent_t e = prof_event();
  cudaEventRecord(e, st);
  g_prof.pending[name] = e;
}
void prof_end(cudaStream_t st, const char* name) {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  if (!prof_match(name)) return;
  auto it = g_prof.pending.find(name);
  if (it == g_prof.pending.end() || !it->second) return;
  cudaEvent_t e = prof_event();
  cudaEventRecord(e, st);
  g_prof.recs.push_back({name, {it->second, e}});
  it->second = nullptr;
}
}  // namespace sc

using namespace sc;

struct sc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  size_t in_use = 0;
  std::unordered_map<void*, size_t> sizes;
  std::string err;
  int* d_status = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

struct sc_graph {
  sc_ctx* ctx = nullptr;
  int sym = 0;
  CsrDev csr;
  int K = 0;              // width of the resident block (0 = none)
  float* X = nullptr;     // resident eigenvector block, n x K, row-major
};

// ---- allocation with budget accounting ---------------------------------------------------
static void* ctx_alloc(void* self, size_t bytes) {
  sc_ctx* c = (sc_ctx*)self;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (c->budget && c->in_use + bytes > c->budget) return nullptr;
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c->sizes[p] = bytes;
  c->in_use += bytes;
  return p;
}
static void ctx_free(void* self, void* p) {
  sc_ctx* c = (sc_ctx*)self;
  if (!p) return;
  auto it = c->sizes.find(p);
  if (it != c->sizes.end()) {
    c->in_use -= it->second;
    c->sizes.erase(it);
  }
  cudaFreeAsync(p, c->stream);
}
static Alloc alloc_of(sc_ctx* c) { return Alloc{ctx_alloc, ctx_free, c}; }

static int fail(sc_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}
static int cuda_fail(sc_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return fail(c, SC_ENOMEM, std::string(where) + ": out of device memory or HBM budget");
  return fail(c, SC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(expr, where)                                   \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
  } while (0)

// ---- SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator ---------------------
static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline uint64_t sm64(uint64_t state, uint64_t i) {
  return mix64(state + (i + 1) * 0x9E3779B97F4A7C15ull);
}
static uint64_t stream_key(uint64_t seed, uint64_t purpose, uint64_t sub) {
  uint64_t k = sm64(seed ^ purpose, 0);
  if (sub) k = sm64(k, sub);
  return k;
}
static inline double uniform_at(uint64_t k, uint64_t i) {
  return (double)(sm64(k, i) >> 11) * (1.0 / 9007199254740992.0);
}
// purpose ids of the streams: 1 = Gaussian start block (generated on the device by
// gauss_block), 2 = k-means++ uniforms.
static void kmeans_uniforms(uint64_t seed, int k, std::vector<double>& u) {
  uint64_t key = stream_key(seed, 2, 0);
  u.resize(k);
  for (int t = 0; t < k; ++t) u[t] = uniform_at(key, (uint64_t)t);
}

// ---------------------------------------------------------------------------------------
// The entry points below were declared extern "C" in sc.h and keep that linkage.

int sc_ctx_create(sc_ctx** out, int device, void* cuda_stream, size_t hbm_budget) {
  if (!out) return SC_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SC_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return SC_ECUDA;
  sc_ctx* c = new sc_ctx();
  c->device = device;
  c->budget = hbm_budget;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return SC_ECUDA;
    }
    c->own_stream = true;
  }
  // keep freed blocks in the pool: later calls reuse them without new allocations
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  c->d_status = (int*)ctx_alloc(c, sizeof(int));
  if (!c->d_status) {
    sc_ctx_destroy(c);
    return SC_ENOMEM;
  }
  cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    sc_ctx_destroy(c);
    return SC_ECUDA;
  }
  *out = c;
  return SC_OK;
}

void sc_ctx_destroy(sc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->d_status) ctx_free(c, c->d_status);
  cudaStreamSynchronize(c->stream);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* sc_last_error(const sc_ctx* c) { return c ? c->err.c_str() : "null context"; }

size_t sc_ctx_bytes_in_use(const sc_ctx* c) { return c ? c->in_use : 0; }
uint64_t sc_ctx_kernel_launches(const sc_ctx*) { return launches_total(); }

int sc_profile_begin(sc_ctx* c, const char* kernels) {
  if (!c || !kernels) return SC_EINVAL;
  std::lock_guard<std::mutex> lk(g_prof.mu);
  g_prof.on = true;
  g_prof.filter = kernels;
  g_prof.recs.clear();
  g_prof.pending.clear();
  g_prof.used = 0;
  return SC_OK;
}

int sc_profile_end(sc_ctx* c, char* report, size_t len) {
  if (!c) return SC_EINVAL;
  cudaSetDevice(c->device);
  CK(cudaStreamSynchronize(c->stream), "profile");
  std::lock_guard<std::mutex> lk(g_prof.mu);
  std::vector<std::string> order;
  std::unordered_map<std::string, std::pair<long long, double>> acc;
  for (auto& r : g_prof.recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.second.first, r.second.second) != cudaSuccess) ms = 0.f;
    auto it = acc.find(r.first);
    if (it == acc.end()) {
      order.push_back(r.first);
      acc[r.first] = {1, ms};
    } else {
      it->second.first += 1;
      it->second.second += ms;
    }
  }
  std::string out;
  char line[160];
  for (auto& k : order) {
    snprintf(line, sizeof(line), "%s %lld %.6f\n", k.c_str(), acc[k].first, acc[k].second);
    out += line;
  }
  if (report && len) {
    size_t nb = std::min(len - 1, out.size());
    memcpy(report, out.data(), nb);
    report[nb] = 0;
  }
  g_prof.on = false;
  g_prof.recs.clear();
  g_prof.pending.clear();
  g_prof.used = 0;
  return SC_OK;
}

// ---- graphs ------------------------------------------------------------------------------

static void free_csr(sc_ctx* c, CsrDev& g) {
  ctx_free(c, g.row_ptr);
  ctx_free(c, g.col_idx);
  ctx_free(c, g.val);
  ctx_free(c, g.degf);
  ctx_free(c, g.degd);
  g = CsrDev{};
}

static int read_status(sc_ctx* c, int* out) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status");
  CK(cudaStreamSynchronize(c->stream), "status");
  CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "status");
  *out = h;
  return SC_OK;
}

// Copy an edge list to the device (or use it in place) and build a CSR.
static int edges_to_csr(sc_ctx* c, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                        const float* w, int algebraic, int on_device, CsrDev* out) {
  Alloc al = alloc_of(c);
  const int32_t *ds = src, *dd = dst;
  const float* dw = w;
  int32_t *ts = nullptr, *td = nullptr;
  float* tw = nullptr;
  if (!on_device && m > 0) {
    ts = al.get<int32_t>((size_t)m);
    td = al.get<int32_t>((size_t)m);
    if (algebraic && w) tw = al.get<float>((size_t)m);
    if (!ts || !td || (algebraic && w && !tw)) {
      al.put(ts); al.put(td); al.put(tw);
      return fail(c, SC_ENOMEM, "edge staging: out of device memory or HBM budget");
    }
    cudaMemcpyAsync(ts, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(td, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, c->stream);
    if (tw) cudaMemcpyAsync(tw, w, sizeof(float) * m, cudaMemcpyHostToDevice, c->stream);
    ds = ts; dd = td; dw = tw;
  }
  int hs = 0;
  cudaError_t e = build_csr(c->stream, al, n, m, ds, dd, algebraic ? dw : nullptr, algebraic,
                            c->d_status, out, &hs);
  cudaStreamSynchronize(c->stream);
  al.put(ts); al.put(td); al.put(tw);
  int st = 0;
  int rc = read_status(c, &st);
  if (rc != SC_OK) return rc;
  hs |= st;
  if (e != cudaSuccess) {
    free_csr(c, *out);
    return cuda_fail(c, e, "sc_build_laplacian");
  }
  if (hs & ST_EDGE_RANGE) {
    free_csr(c, *out);
    return fail(c, SC_EINVAL, "edge endpoint outside [0, n)");
  }
  if (hs & ST_NNZ_OVERFLOW) {
    free_csr(c, *out);
    return fail(c, SC_EINVAL, "symmetrized graph has more than 2^31-1 stored entries");
  }
  return SC_OK;
}

int sc_build_laplacian(sc_ctx* c, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                       const float* w, int sym, int on_device, sc_graph** out) {
  if (!c || !out) return SC_EINVAL;
  *out = nullptr;
  if (n < 1 || m < 0 || (m > 0 && (!src || !dst)) || (sym != SC_SYM_LOGICAL && sym != SC_SYM_ALGEBRAIC))
    return fail(c, SC_EINVAL, "sc_build_laplacian: bad arguments");
  cudaSetDevice(c->device);
  sc_graph* g = new sc_graph();
  g->ctx = c;
  g->sym = sym;
  int rc = edges_to_csr(c, n, m, src, dst, w, sym == SC_SYM_ALGEBRAIC, on_device, &g->csr);
  if (rc != SC_OK) {
    delete g;
    return rc;
  }
  *out = g;
  return SC_OK;
}

int sc_graph_info(const sc_graph* g, int32_t* n, int64_t* nnz, double* deg_max) {
  if (!g) return SC_EINVAL;
  if (n) *n = g->csr.n;
  if (nnz) *nnz = g->csr.nnz;
  if (deg_max) *deg_max = g->csr.deg_max;
  return SC_OK;
}

int sc_graph_copy_csr(const sc_graph* g, int32_t* row_ptr, int32_t* col_idx, float* val,
                      double* deg) {
  if (!g) return SC_EINVAL;
  sc_ctx* c = g->ctx;
  cudaSetDevice(c->device);
  const CsrDev& a = g->csr;
  if (row_ptr) CK(cudaMemcpyAsync(row_ptr, a.row_ptr, sizeof(int) * (a.n + 1), cudaMemcpyDeviceToHost, c->stream), "copy_csr");
  if (col_idx && a.nnz) CK(cudaMemcpyAsync(col_idx, a.col_idx, sizeof(int) * a.nnz, cudaMemcpyDeviceToHost, c->stream), "copy_csr");
  if (val && a.nnz) {
    if (a.val) {
      CK(cudaMemcpyAsync(val, a.val, sizeof(float) * a.nnz, cudaMemcpyDeviceToHost, c->stream), "copy_csr");
    } else {
      CK(cudaStreamSynchronize(c->stream), "copy_csr");
      for (int64_t i = 0; i < a.nnz; ++i) val[i] = 1.0f;
    }
  }
  if (deg) CK(cudaMemcpyAsync(deg, a.degd, sizeof(double) * a.n, cudaMemcpyDeviceToHost, c->stream), "copy_csr");
  CK(cudaStreamSynchronize(c->stream), "copy_csr");
  return SC_OK;
}

void sc_graph_destroy(sc_graph* g) {
  if (!g) return;
  sc_ctx* c = g->ctx;
  cudaSetDevice(c->device);
  free_csr(c, g->csr);
  ctx_free(c, g->X);
  cudaStreamSynchronize(c->stream);
  delete g;
}

// ---- SpMM entry point --------------------------------------------------------------------

template <typename T>
static int lap_apply_t(sc_ctx* c, sc_graph* g, int k, const T* V, T* Y, int on_device) {
  Alloc al = alloc_of(c);
  const int W = 16 / sizeof(T);
  const int n = g->csr.n;
  const int kp = (k + W - 1) / W * W;
  T* dv = al.get<T>((size_t)n * kp);
  T* dy = al.get<T>((size_t)n * kp);
  if (!dv || !dy) {
    al.put(dv); al.put(dy);
    return fail(c, SC_ENOMEM, "sc_lap_apply: out of device memory");
  }
  cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaMemsetAsync(dv, 0, sizeof(T) * (size_t)n * kp, c->stream);
  CK(cudaMemcpy2DAsync(dv, sizeof(T) * kp, V, sizeof(T) * k, sizeof(T) * k, n, kin, c->stream), "lap_apply");
  CK(spmm_lap<T>(c->stream, g->csr, dv, kp, dy, kp, k), "lap_apply");
  CK(cudaMemcpy2DAsync(Y, sizeof(T) * k, dy, sizeof(T) * kp, sizeof(T) * k, n, kout, c->stream), "lap_apply");
  CK(cudaStreamSynchronize(c->stream), "lap_apply");
  al.put(dv);
  al.put(dy);
  return SC_OK;
}

int sc_lap_apply(sc_ctx* c, sc_graph* g, int k, int prec, const void* V, void* Y, int on_device) {
  if (!c || !g || !V || !Y || k < 1 || k > SC_MAX_K) return SC_EINVAL;
  cudaSetDevice(c->device);
  if (prec == SC_PREC_FP64) return lap_apply_t<double>(c, g, k, (const double*)V, (double*)Y, on_device);
  return lap_apply_t<float>(c, g, k, (const float*)V, (float*)Y, on_device);
}

// ---- LOBPCG --------------------------------------------------------------------------------

namespace {

template <typename T>
struct Lob {
  sc_ctx* c;
  Alloc al;
  sc_graph* g;
  int n, K, kp;  // kp: padded row stride of every block
  int use_tc;
  double pivot_tol;
  std::vector<T*> pool;
  std::vector<void*> misc;
  T* get_block() {
    T* p = al.get<T>((size_t)n * kp);
    if (p) {
      pool.push_back(p);
      cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n * kp, c->stream);
    }
    return p;
  }
  template <typename U>
  U* get_small(size_t count) {
    U* p = al.get<U>(count);
    if (p) misc.push_back(p);
    return p;
  }
  ~Lob() {
    for (T* p : pool) al.put(p);
    for (void* p : misc) al.put(p);
  }
};

struct Seg {
  int start, count;
};

// C (compact FP64) = A' B over the listed column segments of two strided blocks.  FP32 with
// tensor cores selected -> tcgen05 kernel; otherwise the CUDA-core kernel.
template <typename T>
cudaError_t gram_seg(Lob<T>& L, const T* A, long long lda, std::initializer_list<Seg> sa,
                     const T* B, long long ldb, std::initializer_list<Seg> sb, double* C,
                     int ldc, bool sym) {
  std::vector<Seg> va(sa), vb(sb);
  if constexpr (sizeof(T) == 4) {
    if (L.use_tc) {
      int pa[6], pb[6], spa = 0, spb = 0;
      for (size_t q = 0; q < va.size(); ++q) {
        pa[2 * q] = va[q].start;
        pa[2 * q + 1] = va[q].count;
        spa = std::max(spa, va[q].start + va[q].count);
      }
      for (size_t q = 0; q < vb.size(); ++q) {
        pb[2 * q] = vb[q].start;
        pb[2 * q + 1] = vb[q].count;
        spb = std::max(spb, vb[q].start + vb[q].count);
      }
      return gram_tc(L.c->stream, L.al, L.n, (const float*)A, lda, spa, pa, (int)va.size(),
                     (const float*)B, ldb, spb, pb, (int)vb.size(), C, ldc, sym, L.c->d_status);
    }
  }
  Cat3<T> ca{}, cb{};
  ca.nblk = (int)va.size();
  cb.nblk = (int)vb.size();
  for (size_t q = 0; q < va.size(); ++q) {
    ca.p[q] = A + va[q].start;
    ca.ld[q] = lda;
    ca.c[q] = va[q].count;
  }
  for (size_t q = 0; q < vb.size(); ++q) {
    cb.p[q] = B + vb[q].start;
    cb.ld[q] = ldb;
    cb.c[q] = vb[q].count;
  }
  return gram<T>(L.c->stream, L.al, L.n, ca, cb, C, ldc, sym, 0);
}

// Cholesky-QR of block V (n x kc, stride ldv) into out (stride ldo); optionally applies the
// same transform to LV (into lout).  Reports ST_CHOL_FAIL in *status_out (nothing written).
template <typename T>
int cholqr_step(Lob<T>& L, const T* V, long long ldv, int kc, T* out, long long ldo, double* G,
                T* Tm, const T* LV, long long ldlv, T* lout, long long ldlo, int* status_out) {
  sc_ctx* c = L.c;
  cudaStream_t st = c->stream;
  CK(gram_seg<T>(L, V, ldv, {{0, kc}}, V, ldv, {{0, kc}}, G, kc, true), "gram");
  CK(chol_inv<T>(st, L.al, kc, G, kc, Tm, c->d_status, L.pivot_tol), "chol");
  int hs = 0;
  int rc = read_status(c, &hs);
  if (rc != SC_OK) return rc;
  *status_out = hs;
  if (hs & 32) return fail(c, SC_ETIMEOUT, "a bounded device wait gave up");
  if (hs & (ST_CHOL_FAIL | ST_NONFINITE)) return SC_OK;
  CK(tall_gemm<T>(st, L.n, cat<T>(V, ldv, kc), Tm, kc, kc, out, ldo, nullptr, 0, (T)0), "tall");
  if (LV) CK(tall_gemm<T>(st, L.n, cat<T>(LV, ldlv, kc), Tm, kc, kc, lout, ldlo, nullptr, 0, (T)0), "tall");
  return SC_OK;
}

// Block layout: S = [X | R | P] and LS = [LX | LR | LP], each n x 3kp row-major (column slots
// of kp = K rounded up to 16 bytes), so every Gram operand is one strided matrix.
template <typename T>
int run_lobpcg(sc_ctx* c, sc_graph* g, int K, const sc_lobpcg_opts* o, const float* X0,
               int32_t x0_rows, float* X_out, sc_eig_info* info) {
  const int n = g->csr.n;
  const int W = 16 / sizeof(T);
  const int kp = (K + W - 1) / W * W;
  const long long ld3 = 3LL * kp;
  Lob<T> L{c, alloc_of(c), g, n, K, kp, (sizeof(T) == 4 && o->prec == SC_PREC_MIXED) ? 1 : 0,
           sizeof(T) == 4 ? 1e-8 : 1e-14, {}, {}};
  cudaStream_t st = c->stream;
  const int mmax = 3 * K;
  auto big = [&]() {
    T* p = L.al.template get<T>((size_t)n * ld3);
    if (p) {
      L.pool.push_back(p);
      cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n * ld3, st);
    }
    return p;
  };
  T* S = big();
  T* LS = big();
  T* S2 = big();
  T* LS2 = big();
  T* T1 = L.get_block();
  auto wide = [&]() {
    T* p = L.al.template get<T>((size_t)n * 2 * kp);
    if (p) {
      L.pool.push_back(p);
      cudaMemsetAsync(p, 0, sizeof(T) * (size_t)n * 2 * kp, st);
    }
    return p;
  };
  T* W1 = wide();
  T* W2 = wide();
  T* Q1 = wide();
  T* LQ1 = wide();
  double* G = L.template get_small<double>((size_t)mmax * mmax);
  T* Tm = L.template get_small<T>((size_t)mmax * mmax);
  T* Y = L.template get_small<T>((size_t)mmax * K);
  double* theta = L.template get_small<double>(K);
  double* rho2 = L.template get_small<double>(K);
  int* dcols = L.template get_small<int>(K);
  int* dfail = L.template get_small<int>(1);
  int* dP = L.template get_small<int>(1);   // 1 = direction block in use this pass
  int* dfb = L.template get_small<int>(1);  // passes that dropped it
  if (!S || !LS || !S2 || !LS2 || !T1 || !W1 || !W2 || !Q1 || !LQ1 || !G || !Tm || !Y || !theta ||
      !rho2 || !dcols || !dfail || !dP || !dfb)
    return fail(c, SC_ENOMEM, "sc_lobpcg: out of device memory or HBM budget");
  auto X = [&]() { return S; };
  auto LX = [&]() { return LS; };

  // ---- start block --------------------------------------------------------------------
  {
    const float* src = nullptr;
    int rows = 0;
    bool dev_src = false;
    if (X0) {
      src = X0;
      rows = x0_rows > 0 ? std::min(x0_rows, n) : n;
    } else if (g->X && g->K == K && !o->cold) {
      src = g->X;
      rows = n;
      dev_src = true;
    }
    if (!src) {
      CK(gauss_block<T>(st, n, K, stream_key(o->seed, 1, 0), S, ld3), "x0");
    } else if (sizeof(T) == 4) {
      CK(cudaMemcpy2DAsync(S, sizeof(T) * ld3, src, sizeof(float) * K, sizeof(float) * K, rows,
                           dev_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st), "x0");
    } else {
      std::vector<float> hf((size_t)rows * K);
      if (dev_src) {
        CK(cudaMemcpyAsync(hf.data(), src, sizeof(float) * hf.size(), cudaMemcpyDeviceToHost, st), "x0");
        CK(cudaStreamSynchronize(st), "x0");
      } else {
        std::memcpy(hf.data(), src, sizeof(float) * hf.size());
      }
      std::vector<double> hd(hf.begin(), hf.end());
      CK(cudaMemcpy2DAsync(S, sizeof(T) * ld3, hd.data(), sizeof(double) * K, sizeof(double) * K,
                           rows, cudaMemcpyHostToDevice, st), "x0");
    }
    CK(cudaStreamSynchronize(st), "x0");
  }
  {
    int one = 1, zero = 0;
    CK(cudaMemcpyAsync(dP, &one, sizeof(int), cudaMemcpyHostToDevice, st), "flags");
    CK(cudaMemcpyAsync(dfb, &zero, sizeof(int), cudaMemcpyHostToDevice, st), "flags");
    CK(cudaStreamSynchronize(st), "flags");
  }
  CK(cudaEventRecord(c->ev0, st), "event");
  const uint64_t l0 = launches_total();
  int hs = 0;
  // X <- CholQR(CholQR(X0)):  X slot -> T1 -> X slot
  {
    int rc = cholqr_step<T>(L, S, ld3, K, T1, kp, G, Tm, nullptr, 0, nullptr, 0, &hs);
    if (rc != SC_OK) return rc;
    if (hs & (ST_CHOL_FAIL | ST_NONFINITE)) return fail(c, SC_EBREAKDOWN, "start block is rank deficient");
    rc = cholqr_step<T>(L, T1, kp, K, S, ld3, G, Tm, nullptr, 0, nullptr, 0, &hs);
    if (rc != SC_OK) return rc;
    if (hs & (ST_CHOL_FAIL | ST_NONFINITE)) return fail(c, SC_EBREAKDOWN, "start block is rank deficient");
  }
  CK(spmm_lap<T>(st, g->csr, S, ld3, LS, ld3, K), "spmm");
  CK(gram_seg<T>(L, S, ld3, {{0, K}}, LS, ld3, {{0, K}}, G, K, false), "gram");
  CK(rr_eig<T>(st, L.al, K, K, G, K, theta, Y, c->d_status), "rr");
  CK(tall_gemm<T>(st, n, cat<T>(S, ld3, K), Y, K, K, S2, ld3, nullptr, 0, (T)0), "tall");
  CK(tall_gemm<T>(st, n, cat<T>(LS, ld3, K), Y, K, K, LS2, ld3, nullptr, 0, (T)0), "tall");
  std::swap(S, S2);
  std::swap(LS, LS2);
  CK(residual<T>(st, L.al, n, K, S, LS, ld3, theta, S + kp, rho2), "residual");
  (void)X;
  (void)LX;

  std::vector<double> hrho(K), hth(K);
  bool haveP = false;
  int done = 0, fallbacks = 0, converged = 0;
  // The host reads the residual norms between passes only when it has to decide something
  // (a stopping tolerance or soft locking); otherwise the passes are issued back to back.
  const bool watch = o->tol_abs > 0 || o->tol_lock > 0;
  std::vector<int> all_cols(K);
  for (int j = 0; j < K; ++j) all_cols[j] = j;
  for (int it = 0; it < o->iters; ++it) {
    std::vector<int> act;
    double mx = 0.0;
    if (watch) {
      CK(cudaMemcpyAsync(hrho.data(), rho2, sizeof(double) * K, cudaMemcpyDeviceToHost, st), "rho");
      CK(cudaStreamSynchronize(st), "rho");
      for (int j = 0; j < K; ++j) {
        double r = std::sqrt(std::max(hrho[j], 0.0));
        mx = std::max(mx, r);
        if (r > o->tol_lock) act.push_back(j);
      }
    } else {
      act = all_cols;
    }
    if (o->tol_abs > 0 && mx <= o->tol_abs) {
      converged = 1;
      break;
    }
    if (act.empty()) {
      converged = o->tol_abs > 0 ? 1 : 0;
      break;
    }
    const int ka = (int)act.size();
    const bool all = ka == K;
    T* Rslot = S + kp;
    T* LRslot = LS + kp;
    T* Pslot = S + 2 * kp;
    T* LPslot = LS + 2 * kp;
    // Working copies of the active R and P columns.  With every column active they are the
    // S slots themselves ([R P] = columns kp.. and 2kp.. of S); otherwise the active columns
    // are gathered into W1 = [R_a | P_a] (n x 2kp) and W2 = [. | LP_a].
    T* WR = Rslot;
    T* WP = Pslot;
    T* WLP = LPslot;
    long long ldw = ld3;
    int offP = kp;  // column offset of P in the working block (relative to WR)
    if (!all) {
      CK(cudaMemcpyAsync(dcols, act.data(), sizeof(int) * ka, cudaMemcpyHostToDevice, st), "cols");
      CK(gather_cols<T>(st, n, Rslot, ld3, W1, 2 * kp, dcols, ka), "gather");
      WR = W1;
      WP = W1 + kp;
      ldw = 2 * kp;
      if (haveP) {
        CK(gather_cols<T>(st, n, Pslot, ld3, WP, ldw, dcols, ka), "gather");
        CK(gather_cols<T>(st, n, LPslot, ld3, W2 + kp, ldw, dcols, ka), "gather");
        WLP = W2 + kp;
      }
    }
    const int w = haveP ? 2 * ka : ka;
    // (1) project [R_a P_a] against X: F = X' [R_a P_a]; R_a -= X F_R, P_a -= X F_P, LP_a -= LX F_P
    if (haveP)
      CK(gram_seg<T>(L, S, ld3, {{0, K}}, WR, ldw, {{0, ka}, {offP, ka}}, G, w, false), "gram");
    else
      CK(gram_seg<T>(L, S, ld3, {{0, K}}, WR, ldw, {{0, ka}}, G, w, false), "gram");
    CK(cast_mat<T>(st, K, w, G, w, Tm, w, -1.0), "cast");
    CK(tall_gemm<T>(st, n, cat<T>(S, ld3, K), Tm, w, ka, WR, ldw, WR, ldw, (T)1), "tall");
    if (haveP) {
      CK(tall_gemm<T>(st, n, cat<T>(S, ld3, K), Tm + ka, w, ka, WP, ldw, WP, ldw, (T)1), "tall");
      CK(tall_gemm<T>(st, n, cat<T>(LS, ld3, K), Tm + ka, w, ka, WLP, ldw, WLP, ldw, (T)1), "tall");
    }
    // (2) LR_a = L R_a (the one SpMM of the pass), into the LR slot / working block
    T* WLR = all ? LRslot : W2;
    CK(spmm_lap<T>(st, g->csr, WR, ldw, WLR, ldw, ka), "spmm");
    // (3) Cholesky-QR twice of [R_a P_a] (R first, so P is orthogonalized against R as well),
    //     with [LR_a LP_a] transformed alike.  A breakdown inside the P columns is handled on
    //     the device: the kernel keeps the R transform, zeroes P's, and clears *dP, which the
    //     Rayleigh-Ritz step reads to solve without P (a fallback).  A breakdown inside R is
    //     reported through the status word.
    {
      const int wq = w;
      int* pf = haveP ? dP : nullptr;
      Cat3<T> Vw = haveP ? cat<T>(WR, ldw, ka, WP, ldw, ka) : cat<T>(WR, ldw, ka);
      Cat3<T> LVw = haveP ? cat<T>(WLR, ldw, ka, WLP, ldw, ka) : cat<T>(WLR, ldw, ka);
      if (haveP)
        CK(gram_seg<T>(L, WR, ldw, {{0, ka}, {offP, ka}}, WR, ldw, {{0, ka}, {offP, ka}}, G, wq, true), "gram");
      else
        CK(gram_seg<T>(L, WR, ldw, {{0, ka}}, WR, ldw, {{0, ka}}, G, wq, true), "gram");
      CK(chol_inv<T>(st, L.al, wq, G, wq, Tm, c->d_status, L.pivot_tol, dfail, ka, pf), "chol");
      CK(tall_gemm<T>(st, n, Vw, Tm, wq, wq, Q1, 2 * kp, nullptr, 0, (T)0), "tall");
      CK(tall_gemm<T>(st, n, LVw, Tm, wq, wq, LQ1, 2 * kp, nullptr, 0, (T)0), "tall");
      CK(gram_seg<T>(L, Q1, 2 * kp, {{0, wq}}, Q1, 2 * kp, {{0, wq}}, G, wq, true), "gram");
      CK(chol_inv<T>(st, L.al, wq, G, wq, Tm, c->d_status, L.pivot_tol, dfail, ka, pf), "chol");
      CK(tall_gemm<T>(st, n, cat<T>(Q1, 2 * kp, ka), Tm, wq, ka, Rslot, ld3, nullptr, 0, (T)0), "tall");
      CK(tall_gemm<T>(st, n, cat<T>(LQ1, 2 * kp, ka), Tm, wq, ka, LRslot, ld3, nullptr, 0, (T)0), "tall");
      if (haveP) {
        CK(tall_gemm<T>(st, n, cat<T>(Q1, 2 * kp, wq), Tm + ka, wq, ka, Pslot, ld3, nullptr, 0, (T)0), "tall");
        CK(tall_gemm<T>(st, n, cat<T>(LQ1, 2 * kp, wq), Tm + ka, wq, ka, LPslot, ld3, nullptr, 0, (T)0), "tall");
      }
    }
    const bool useP = haveP;
    // Rayleigh-Ritz on S = [X R_a P_a]
    const int m = K + ka + (useP ? ka : 0);
    if (useP)
      CK(gram_seg<T>(L, S, ld3, {{0, K}, {kp, ka}, {2 * kp, ka}}, LS, ld3, {{0, K}, {kp, ka}, {2 * kp, ka}}, G, m, false), "gram");
    else
      CK(gram_seg<T>(L, S, ld3, {{0, K}, {kp, ka}}, LS, ld3, {{0, K}, {kp, ka}}, G, m, false), "gram");
    CK(rr_eig<T>(st, L.al, m, K, G, m, theta, Y, c->d_status, useP ? dP : nullptr, ka, dfb), "rr");
    // update into S2 / LS2: P = [R_a P_a] Y_RP, X = X Y_X + P (L-images alike), R = LX - X theta
    const T* Yrp = Y + (size_t)K * K;
    Cat3<T> RP = useP ? cat<T>(Rslot, ld3, ka, Pslot, ld3, ka) : cat<T>(Rslot, ld3, ka);
    Cat3<T> LRP = useP ? cat<T>(LRslot, ld3, ka, LPslot, ld3, ka) : cat<T>(LRslot, ld3, ka);
    CK(tall_gemm<T>(st, n, RP, Yrp, K, K, S2 + 2 * kp, ld3, nullptr, 0, (T)0), "tall");
    CK(tall_gemm<T>(st, n, cat<T>(S, ld3, K), Y, K, K, S2, ld3, S2 + 2 * kp, ld3, (T)1), "tall");
    CK(tall_gemm<T>(st, n, LRP, Yrp, K, K, LS2 + 2 * kp, ld3, nullptr, 0, (T)0), "tall");
    CK(tall_gemm<T>(st, n, cat<T>(LS, ld3, K), Y, K, K, LS2, ld3, LS2 + 2 * kp, ld3, (T)1), "tall");
    std::swap(S, S2);
    std::swap(LS, LS2);
    haveP = true;
    CK(residual<T>(st, L.al, n, K, S, LS, ld3, theta, S + kp, rho2), "residual");
    ++done;
  }
  CK(cudaEventRecord(c->ev1, st), "event");
  CK(cudaStreamSynchronize(st), "sync");
  int st_final = 0;
  int rc = read_status(c, &st_final);
  if (rc != SC_OK) return rc;
  if (st_final & 32) return fail(c, SC_ETIMEOUT, "a bounded device wait gave up");
  if (st_final & ST_NONFINITE) return fail(c, SC_EBREAKDOWN, "non-finite values in Rayleigh-Ritz");
  if (st_final & ST_CHOL_FAIL) return fail(c, SC_EBREAKDOWN, "residual block lost rank");
  CK(cudaMemcpyAsync(&fallbacks, dfb, sizeof(int), cudaMemcpyDeviceToHost, st), "out");
  CK(cudaMemcpyAsync(hrho.data(), rho2, sizeof(double) * K, cudaMemcpyDeviceToHost, st), "out");
  CK(cudaMemcpyAsync(hth.data(), theta, sizeof(double) * K, cudaMemcpyDeviceToHost, st), "out");
  // resident block (float, n x K) for warm starts and the embedding
  if (!g->X || g->K != K) {
    ctx_free(c, g->X);
    g->X = (float*)ctx_alloc(c, sizeof(float) * (size_t)n * K);
    g->K = g->X ? K : 0;
  }
  if (g->X) {
    if (sizeof(T) == 4) {
      CK(cudaMemcpy2DAsync(g->X, sizeof(float) * K, S, sizeof(T) * ld3, sizeof(float) * K, n,
                           cudaMemcpyDeviceToDevice, st), "resident");
    } else {
      std::vector<double> hd((size_t)n * K);
      CK(cudaMemcpy2DAsync(hd.data(), sizeof(double) * K, S, sizeof(T) * ld3, sizeof(double) * K, n,
                           cudaMemcpyDeviceToHost, st), "resident");
      CK(cudaStreamSynchronize(st), "resident");
      std::vector<float> hf(hd.begin(), hd.end());
      CK(cudaMemcpyAsync(g->X, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice, st), "resident");
      if (X_out) std::memcpy(X_out, hf.data(), sizeof(float) * hf.size());
      CK(cudaStreamSynchronize(st), "resident");
    }
  }
  if (X_out && sizeof(T) == 4) {
    CK(cudaMemcpy2DAsync(X_out, sizeof(float) * K, S, sizeof(T) * ld3, sizeof(float) * K, n,
                         cudaMemcpyDeviceToHost, st), "xout");
  }
  CK(cudaStreamSynchronize(st), "sync");
  if (info) {
    info->K = K;
    info->iters_done = done;
    info->fallbacks = fallbacks;
    info->converged = converged;
    for (int j = 0; j < K; ++j) {
      info->lambda[j] = hth[j];
      info->resid[j] = std::sqrt(std::max(hrho[j], 0.0));
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    info->ms = ms;
    info->kernels = launches_total() - l0;
  }
  if (o->tol_abs > 0 && !converged) return fail(c, SC_ENOTCONV, "tolerance not reached");
  return SC_OK;
}

}  // namespace

// FP64 copies of the double-precision resident block go through the host (the library keeps
// one float block per graph); the FP64 path writes X_out from that copy.
int sc_lobpcg(sc_ctx* c, sc_graph* g, int K, const sc_lobpcg_opts* o, const float* X0,
              int32_t x0_rows, float* X_out, sc_eig_info* info) {
  if (!c || !g || !o || K < 1 || K > SC_MAX_K || o->iters < 0) return SC_EINVAL;
  if ((int64_t)3 * K > g->csr.n) return fail(c, SC_EINVAL, "sc_lobpcg: need 3K <= n");
  if (o->prec < SC_PREC_MIXED || o->prec > SC_PREC_FP64) return fail(c, SC_EINVAL, "bad precision");
  cudaSetDevice(c->device);
  if (o->prec == SC_PREC_FP64) return run_lobpcg<double>(c, g, K, o, X0, x0_rows, X_out, info);
  return run_lobpcg<float>(c, g, K, o, X0, x0_rows, X_out, info);
}

int sc_embed_rows(sc_ctx* c, const float* X, int32_t n, int K, float* E, int on_device) {
  if (!c || !X || !E || n < 1 || K < 1) return SC_EINVAL;
  cudaSetDevice(c->device);
  Alloc al = alloc_of(c);
  const float* dx = X;
  float* de = E;
  float *tx = nullptr, *te = nullptr;
  if (!on_device) {
    tx = al.get<float>((size_t)n * K);
    te = al.get<float>((size_t)n * K);
    if (!tx || !te) {
      al.put(tx); al.put(te);
      return fail(c, SC_ENOMEM, "sc_embed_rows");
    }
    CK(cudaMemcpyAsync(tx, X, sizeof(float) * (size_t)n * K, cudaMemcpyHostToDevice, c->stream), "embed");
    dx = tx;
    de = te;
  }
  CK(rownorm<float>(c->stream, n, K, dx, K, de, K), "embed");
  if (!on_device)
    CK(cudaMemcpyAsync(E, te, sizeof(float) * (size_t)n * K, cudaMemcpyDeviceToHost, c->stream), "embed");
  CK(cudaStreamSynchronize(c->stream), "embed");
  al.put(tx);
  al.put(te);
  return SC_OK;
}

// ---- k-means -------------------------------------------------------------------------------

static int kmeans_dev(sc_ctx* c, const float* dE, int32_t n, int d, int k, int iters, uint64_t seed,
                      const int32_t* init_idx, int32_t* labels_out, float* centroids_out,
                      int32_t* seeds_out, double* inertia, int* iters_run) {
  Alloc al = alloc_of(c);
  int* seeds = al.get<int>(k);
  int* labels = al.get<int>(n);
  double* C64 = al.get<double>((size_t)k * d);
  if (!seeds || !labels || !C64) {
    al.put(seeds); al.put(labels); al.put(C64);
    return fail(c, SC_ENOMEM, "sc_kmeans");
  }
  cudaStream_t st = c->stream;
  if (init_idx) {
    for (int j = 0; j < k; ++j)
      if (init_idx[j] < 0 || init_idx[j] >= n) return fail(c, SC_EINVAL, "init_idx out of range");
    CK(cudaMemcpyAsync(seeds, init_idx, sizeof(int) * k, cudaMemcpyHostToDevice, st), "kmeans");
    CK(cudaStreamSynchronize(st), "kmeans");
  } else {
    std::vector<double> u;
    kmeans_uniforms(seed, k, u);
    CK(kmeanspp(st, al, n, d, k, dE, d, u.data(), seeds), "kmeans++");
  }
  double inert = 0.0;
  int ran = 0;
  CK(lloyd(st, al, n, d, k, dE, d, seeds, iters, labels, C64, &ran, &inert), "lloyd");
  if (labels_out) CK(cudaMemcpyAsync(labels_out, labels, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "kmeans");
  if (seeds_out) CK(cudaMemcpyAsync(seeds_out, seeds, sizeof(int) * k, cudaMemcpyDeviceToHost, st), "kmeans");
  std::vector<double> hc;
  if (centroids_out) {
    hc.resize((size_t)k * d);
    CK(cudaMemcpyAsync(hc.data(), C64, sizeof(double) * hc.size(), cudaMemcpyDeviceToHost, st), "kmeans");
  }
  CK(cudaStreamSynchronize(st), "kmeans");
  for (size_t q = 0; q < hc.size(); ++q) centroids_out[q] = (float)hc[q];
  if (inertia) *inertia = inert;
  if (iters_run) *iters_run = ran;
  al.put(seeds);
  al.put(labels);
  al.put(C64);
  return SC_OK;
}

int sc_kmeans(sc_ctx* c, const float* E, int32_t n, int d, int k, int iters, uint64_t seed,
              const int32_t* init_idx, int on_device, int32_t* labels_out, float* centroids_out,
              int32_t* seeds_out, double* inertia, int* iters_run) {
  if (!c || !E || !labels_out || n < 1 || d < 1 || k < 1 || k > n || iters < 0) return SC_EINVAL;
  cudaSetDevice(c->device);
  Alloc al = alloc_of(c);
  const float* dE = E;
  float* tE = nullptr;
  if (!on_device) {
    tE = al.get<float>((size_t)n * d);
    if (!tE) return fail(c, SC_ENOMEM, "sc_kmeans");
    CK(cudaMemcpyAsync(tE, E, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice, c->stream), "kmeans");
    dE = tE;
  }
  int rc = kmeans_dev(c, dE, n, d, k, iters, seed, init_idx, labels_out, centroids_out, seeds_out,
                      inertia, iters_run);
  cudaStreamSynchronize(c->stream);
  al.put(tE);
  return rc;
}

int sc_partition(sc_ctx* c, sc_graph* g, int K, int k, const sc_lobpcg_opts* o, int kmeans_iters,
                 int32_t* labels_out, sc_eig_info* info) {
  if (!c || !g || !o || !labels_out || k < 1 || k > g->csr.n) return SC_EINVAL;
  int rc = sc_lobpcg(c, g, K, o, nullptr, 0, nullptr, info);
  if (rc != SC_OK) return rc;
  Alloc al = alloc_of(c);
  const int n = g->csr.n;
  float* E = al.get<float>((size_t)n * K);
  if (!E) return fail(c, SC_ENOMEM, "sc_partition");
  CK(rownorm<float>(c->stream, n, K, g->X, K, E, K), "embed");
  rc = kmeans_dev(c, E, n, K, k, kmeans_iters, o->seed, nullptr, labels_out, nullptr, nullptr,
                  nullptr, nullptr);
  cudaStreamSynchronize(c->stream);
  al.put(E);
  return rc;
}

// ---- streaming ----------------------------------------------------------------------------

int sc_stream_update(sc_ctx* c, sc_graph* g, int32_t n_new, int64_t m_delta, const int32_t* src,
                     const int32_t* dst, const float* w, int on_device) {
  if (!c || !g || n_new < g->csr.n || m_delta < 0 || (m_delta > 0 && (!src || !dst)))
    return fail(c, SC_EINVAL, "sc_stream_update: bad arguments");
  cudaSetDevice(c->device);
  const int alg = g->sym == SC_SYM_ALGEBRAIC;
  CsrDev delta;
  int rc = edges_to_csr(c, n_new, m_delta, src, dst, w, alg, on_device, &delta);
  if (rc != SC_OK) return rc;
  Alloc al = alloc_of(c);
  CsrDev merged;
  int hs = 0;
  cudaError_t e = merge_csr(c->stream, al, g->csr, delta, alg, c->d_status, &merged, &hs);
  free_csr(c, delta);
  if (e != cudaSuccess) return cuda_fail(c, e, "sc_stream_update");
  if (hs & ST_NNZ_OVERFLOW) {
    free_csr(c, merged);
    return fail(c, SC_EINVAL, "merged graph too large");
  }
  const int n_old = g->csr.n;
  free_csr(c, g->csr);
  g->csr = merged;
  if (g->X && n_new > n_old) {
    float* nx = (float*)ctx_alloc(c, sizeof(float) * (size_t)n_new * g->K);
    if (!nx) return fail(c, SC_ENOMEM, "sc_stream_update: block");
    CK(cudaMemsetAsync(nx, 0, sizeof(float) * (size_t)n_new * g->K, c->stream), "stream");
    CK(cudaMemcpyAsync(nx, g->X, sizeof(float) * (size_t)n_old * g->K, cudaMemcpyDeviceToDevice, c->stream), "stream");
    ctx_free(c, g->X);
    g->X = nx;
  }
  CK(cudaStreamSynchronize(c->stream), "stream");
  return SC_OK;
}

// ---- component entry points -----------------------------------------------------------

template <typename T>
static int gram_t(sc_ctx* c, int prec, int64_t n, int a, int b, const T* A, int64_t lda,
                  const T* B, int64_t ldb, double* C, int on_device) {
  Alloc al = alloc_of(c);
  const int W = 16 / sizeof(T);
  const int ap = (a + W - 1) / W * W, bp = (b + W - 1) / W * W;
  T* dA = al.get<T>((size_t)n * ap + 1);
  T* dB = al.get<T>((size_t)n * bp + 1);
  double* dC = al.get<double>((size_t)a * b);
  if (!dA || !dB || !dC) {
    al.put(dA); al.put(dB); al.put(dC);
    return fail(c, SC_ENOMEM, "sc_gram");
  }
  cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemsetAsync(dA, 0, sizeof(T) * (size_t)n * ap, c->stream), "gram");
  CK(cudaMemsetAsync(dB, 0, sizeof(T) * (size_t)n * bp, c->stream), "gram");
  if (n > 0) {
    CK(cudaMemcpy2DAsync(dA, sizeof(T) * ap, A, sizeof(T) * lda, sizeof(T) * a, n, kin, c->stream), "gram");
    CK(cudaMemcpy2DAsync(dB, sizeof(T) * bp, B, sizeof(T) * ldb, sizeof(T) * b, n, kin, c->stream), "gram");
  }
  if constexpr (sizeof(T) == 4) {
    if (prec == SC_PREC_MIXED) {
      int sa[2] = {0, a}, sb[2] = {0, b};
      CK(gram_tc(c->stream, al, n, (const float*)dA, ap, a, sa, 1, (const float*)dB, bp, b, sb, 1,
                 dC, b, false, c->d_status), "gram_tc");
    } else {
      CK(gram<T>(c->stream, al, n, cat<T>(dA, ap, a), cat<T>(dB, bp, b), dC, b, false, 0), "gram");
    }
  } else {
    CK(gram<T>(c->stream, al, n, cat<T>(dA, ap, a), cat<T>(dB, bp, b), dC, b, false, 0), "gram");
  }
  CK(cudaMemcpyAsync(C, dC, sizeof(double) * (size_t)a * b, cudaMemcpyDeviceToHost, c->stream), "gram");
  CK(cudaStreamSynchronize(c->stream), "gram");
  al.put(dA);
  al.put(dB);
  al.put(dC);
  int hs = 0;
  int rc = read_status(c, &hs);
  if (rc != SC_OK) return rc;
  if (hs & 32) return fail(c, SC_ETIMEOUT, "sc_gram: a bounded device wait gave up");
  return SC_OK;
}

int sc_gram(sc_ctx* c, int prec, int64_t n, int a, int b, const void* A, int64_t lda,
            const void* B, int64_t ldb, double* C, int on_device) {
  if (!c || !A || !B || !C || n < 0 || a < 1 || b < 1 || a > 3 * SC_MAX_K || b > 3 * SC_MAX_K ||
      lda < a || ldb < b)
    return SC_EINVAL;
  cudaSetDevice(c->device);
  if (prec == SC_PREC_FP64)
    return gram_t<double>(c, prec, n, a, b, (const double*)A, lda, (const double*)B, ldb, C, on_device);
  return gram_t<float>(c, prec, n, a, b, (const float*)A, lda, (const float*)B, ldb, C, on_device);
}

template <typename T>
static int rr_t(sc_ctx* c, int m, int K, const double* G, double* theta, double* Y) {
  Alloc al = alloc_of(c);
  double* dG = al.get<double>((size_t)m * m);
  double* dth = al.get<double>(K);
  T* dY = al.get<T>((size_t)m * K);
  if (!dG || !dth || !dY) {
    al.put(dG); al.put(dth); al.put(dY);
    return fail(c, SC_ENOMEM, "sc_rr_solve");
  }
  CK(cudaMemcpyAsync(dG, G, sizeof(double) * (size_t)m * m, cudaMemcpyHostToDevice, c->stream), "rr");
  CK(rr_eig<T>(c->stream, al, m, K, dG, m, dth, dY, c->d_status), "rr");
  std::vector<T> hy((size_t)m * K);
  CK(cudaMemcpyAsync(theta, dth, sizeof(double) * K, cudaMemcpyDeviceToHost, c->stream), "rr");
  CK(cudaMemcpyAsync(hy.data(), dY, sizeof(T) * hy.size(), cudaMemcpyDeviceToHost, c->stream), "rr");
  CK(cudaStreamSynchronize(c->stream), "rr");
  for (size_t q = 0; q < hy.size(); ++q) Y[q] = (double)hy[q];
  al.put(dG);
  al.put(dth);
  al.put(dY);
  int hs = 0;
  int rc = read_status(c, &hs);
  if (rc != SC_OK) return rc;
  if (hs & ST_NONFINITE) return fail(c, SC_EBREAKDOWN, "non-finite input");
  return SC_OK;
}

int sc_rr_solve(sc_ctx* c, int prec, int m, int K, const double* G, double* theta, double* Y) {
  if (!c || !G || !theta || !Y || m < 1 || K < 1 || K > m || m > 3 * SC_MAX_K) return SC_EINVAL;
  cudaSetDevice(c->device);
  if (prec == SC_PREC_FP64) return rr_t<double>(c, m, K, G, theta, Y);
  return rr_t<float>(c, m, K, G, theta, Y);
}
