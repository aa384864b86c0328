// C ABI of the library (include/sc.h): contexts, graphs, the LOBPCG driver, k-means,
// the end-to-end partition and streaming updates.  Host code only orchestrates: every
// arithmetic step runs in the kernels of k_*.cu on the context stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/sc.h"
#include "common.cuh"

// ---------------------------------------------------------------------------------------
namespace sc {
static std::atomic<uint64_t> g_launches{0};
static thread_local uint64_t t_launches = 0;  // this thread's launches (graph capture counts)
void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void note_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
// launches noted while a pass was only being recorded into a graph are taken back
static void unnote_launches(uint64_t k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }
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
bool prof_active() {
  std::lock_guard<std::mutex> lk(g_prof.mu);
  return g_prof.on;
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
  size_t peak = 0;  // high-water mark of in_use
  std::unordered_map<void*, size_t> sizes;
  std::string err;
  int* d_status = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // test hook (sc_debug_inject): the armed failure and its argument
  int inject_kind = 0;
  long long inject_arg = 0;
  long long probe_spins() const { return inject_kind == SC_INJECT_WAIT_TIMEOUT ? inject_arg : 0; }
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
  if (c->in_use > c->peak) c->peak = c->in_use;
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
size_t sc_ctx_bytes_peak(sc_ctx* c) {
  if (!c) return 0;
  const size_t p = c->peak;
  c->peak = c->in_use;
  return p;
}
uint64_t sc_ctx_kernel_launches(const sc_ctx*) { return launches_total(); }
static std::atomic<uint64_t> g_graph_replays{0};
uint64_t sc_ctx_graph_replays(const sc_ctx*) { return g_graph_replays.load(); }

int sc_debug_inject(sc_ctx* c, int kind, long long arg) {
  if (!c) return SC_EINVAL;
  if (kind != SC_INJECT_NONE && kind != SC_INJECT_WAIT_TIMEOUT && kind != SC_INJECT_P_BREAKDOWN)
    return fail(c, SC_EINVAL, "sc_debug_inject: unknown kind");
  if (kind == SC_INJECT_WAIT_TIMEOUT && arg < 1)
    return fail(c, SC_EINVAL, "sc_debug_inject: the wait limit must be >= 1");
  c->inject_kind = kind;
  c->inject_arg = arg;
  return SC_OK;
}

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
  if (!c) return SC_EINVAL;
  if (!g || !V || !Y || k < 1 || k > SC_MAX_K)
    return fail(c, SC_EINVAL, "sc_lap_apply: invalid argument (null pointer or size out of range)");
  cudaSetDevice(c->device);
  if (prec == SC_PREC_FP64) return lap_apply_t<double>(c, g, k, (const double*)V, (double*)Y, on_device);
  return lap_apply_t<float>(c, g, k, (const float*)V, (float*)Y, on_device);
}

// ---- LOBPCG --------------------------------------------------------------------------------

namespace {

// Stream-bound allocator of one LOBPCG run: stream-ordered allocations on the run's stream,
// counted against the context budget.
// A run's allocator: stream-ordered allocations on the run's stream.  With `cache` set, a
// freed block is kept for the next request of the same size instead of being returned to the
// pool, so that after one pass of each shape the passes allocate nothing (the condition for
// capturing them into a CUDA graph).  Every user of a cached block is ordered on the run's
// stream, which makes the reuse safe.  While `capturing`, a request the cache cannot serve
// fails (and sets `miss`) instead of allocating inside the capture.
struct RunAlloc {
  sc_ctx* c;
  cudaStream_t st;
  bool cache = false, capturing = false, miss = false;
  std::multimap<size_t, void*> kept;
};
void* run_alloc(void* self, size_t bytes) {
  RunAlloc* r = (RunAlloc*)self;
  sc_ctx* c = r->c;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (r->cache) {
    auto it = r->kept.find(bytes);
    if (it != r->kept.end()) {
      void* p = it->second;
      r->kept.erase(it);
      return p;
    }
    if (r->capturing) {
      r->miss = true;
      return nullptr;
    }
  }
  if (c->budget && c->in_use + bytes > c->budget) return nullptr;
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, r->st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c->sizes[p] = bytes;
  c->in_use += bytes;
  if (c->in_use > c->peak) c->peak = c->in_use;
  return p;
}
void run_free(void* self, void* p) {
  RunAlloc* r = (RunAlloc*)self;
  if (!p) return;
  auto it = r->c->sizes.find(p);
  if (r->cache && it != r->c->sizes.end()) {
    r->kept.emplace(it->second, p);
    return;
  }
  if (it != r->c->sizes.end()) {
    r->c->in_use -= it->second;
    r->c->sizes.erase(it);
  }
  cudaFreeAsync(p, r->st);
}

// Returns the cached blocks to the pool (the run's stream orders the frees after their uses).
void run_release(RunAlloc* r) {
  r->cache = false;
  for (auto& kv : r->kept) run_free(r, kv.second);
  r->kept.clear();
}

struct Seg {
  int start, count;
};

// One LOBPCG solve as a state machine: setup() (start block and initial Rayleigh-Ritz),
// pass() (one LOBPCG iteration, issued asynchronously), finish() (outputs).  Every run owns
// its stream, allocator and device status word, so several runs can be interleaved pass by
// pass and their kernels overlap on the device (batched solves, the serving loop).
// Block layout: S = [X | R | P] and LS = [LX | LR | LP], each n x 3kp row-major (column slots
// of kp = K rounded up to 16 bytes), so every Gram operand is one strided matrix.
struct RunBase {
  virtual ~RunBase() {}
  virtual int setup(const float* X0, int32_t x0_rows) = 0;
  virtual int pass() = 0;
  virtual int finish(float* X_out, sc_eig_info* info) = 0;
  virtual bool finished() const = 0;
  virtual cudaStream_t stream() const = 0;
};

template <typename T>
struct LobRun : RunBase {
  sc_ctx* c;
  sc_graph* g;
  int n, K, kp;
  long long ld3;
  sc_lobpcg_opts o;
  cudaStream_t st;
  RunAlloc ra;
  Alloc al;
  int use_tc;
  bool dense64 = false;      // small dense solves in FP64, results cast to T
  double *Gd = nullptr, *Yd = nullptr;  // FP64 results of those solves
  double pivot_tol;
  // Rounding floors of the arithmetic T.  A residual column at or below res_floor (64 ulps of
  // the Gershgorin bound 2 max_i d_i on ||L||) cannot improve its Ritz pair any further: it is
  // left out of the pass, which soft-locks that pair on the device.  A direction column whose
  // norm (X unit) has sunk to dir_floor carries no step, only rounding noise: it is left out
  // too.
  double res_floor, dir_floor;
  const T* pdeg = nullptr;  // degrees for the Jacobi preconditioner, or null
  // Hard locking (Sec. IV): an orthonormal constraint block Yc (n x kc, stride ldyc) whose
  // complement the iteration runs in; x0_pitch = row stride (floats) of a host start block.
  const T* Yc = nullptr;
  int kc = 0;
  long long ldyc = 0, x0_pitch = 0;
  // FP64 host start block (used instead of an FP32 one when set) and FP64 host result block
  const double* X0d = nullptr;
  double* Xout64 = nullptr;
  double* Gy = nullptr;
  T* Ty = nullptr;
  static constexpr int kReorth = 16;
  std::vector<void*> bufs;
  T *S = nullptr, *LS = nullptr, *S2 = nullptr, *LS2 = nullptr, *T1 = nullptr, *W1 = nullptr,
    *Q1 = nullptr, *Tm = nullptr, *TmA = nullptr, *TmB = nullptr,
    *Y = nullptr;
  double *G = nullptr, *theta = nullptr, *rho2 = nullptr;
  int *dcols = nullptr, *dfail = nullptr, *dP = nullptr, *dfb = nullptr, *ddrop = nullptr,
      *dstatus = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // second stream for the L-image updates, which overlap the X/R/P side of the pass
  cudaStream_t st2 = nullptr;
  cudaEvent_t evf = nullptr, evj = nullptr;
  uint64_t l0 = 0;
  int it = 0, done_passes = 0, converged = 0;
  bool haveP = false, over = false;
  std::vector<double> hrho, hth;
  // CUDA graphs of the pass (fixed-pass solves): one executable graph per buffer parity
  bool graphs = false;
  T* Sa = nullptr;  // the X/R/P block at the first pass: parity 0
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  uint64_t glaunch[2] = {0, 0};
  int eager_p = 0;  // passes with P run eagerly

  LobRun(sc_ctx* c_, sc_graph* g_, int K_, const sc_lobpcg_opts* o_, cudaStream_t st_)
      : c(c_), g(g_), n(g_->csr.n), K(K_), o(*o_), st(st_) {
    const int W = 16 / sizeof(T);
    kp = (K + W - 1) / W * W;
    ld3 = 3LL * kp;
    ra = RunAlloc{c, st};
    al = Alloc{run_alloc, run_free, &ra};
    use_tc = (sizeof(T) == 4 && (o.prec == SC_PREC_MIXED || o.prec == SC_PREC_MIXED_DD)) ? 1 : 0;
    dense64 = sizeof(T) == 4 && o.prec == SC_PREC_MIXED_DD;
    pivot_tol = sizeof(T) == 4 ? 1e-8 : 1e-10;
    dir_floor = 64.0 * (sizeof(T) == 4 ? 0x1p-24 : 0x1p-53);
    res_floor = dir_floor * 2.0 * g->csr.deg_max;
    if (o.precond == SC_PRECOND_JACOBI) {
      // the residual slot holds D^-1 R: a column with ||r|| above the floor keeps
      // ||D^-1 r|| >= ||r|| / max_i d_i above res_floor / max_i d_i
      pdeg = sizeof(T) == 4 ? (const T*)g->csr.degf : (const T*)g->csr.degd;
      if (g->csr.deg_max > 0) res_floor /= g->csr.deg_max;
    }
    hrho.assign(K, 0.0);
    hth.assign(K, 0.0);
    const char* ge = std::getenv("SC_CUDA_GRAPHS");
    graphs = !(ge && std::strcmp(ge, "0") == 0) && o.tol_abs <= 0 && o.tol_lock <= 0;
    ra.cache = graphs;
  }
  ~LobRun() override {
    if (st2) cudaStreamSynchronize(st2);
    for (cudaGraphExec_t& x : gexec)
      if (x) cudaGraphExecDestroy(x);
    for (void* p : bufs) al.put(p);
    run_release(&ra);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (evf) cudaEventDestroy(evf);
    if (evj) cudaEventDestroy(evj);
    cudaStreamSynchronize(st);
    if (st2) cudaStreamDestroy(st2);
  }
  // st2 continues from everything issued on st so far / st waits for everything on st2
  void fork() {
    cudaEventRecord(evf, st);
    cudaStreamWaitEvent(st2, evf, 0);
  }
  void join() {
    cudaEventRecord(evj, st2);
    cudaStreamWaitEvent(st, evj, 0);
  }
  bool finished() const override { return over; }
  cudaStream_t stream() const override { return st; }

  template <typename U>
  U* get(size_t count, bool zero = false) {
    U* p = al.template get<U>(count);
    if (p) {
      bufs.push_back(p);
      if (zero) cudaMemsetAsync(p, 0, sizeof(U) * count, st);
    }
    return p;
  }
  int read_status(int* out) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    CK(cudaStreamSynchronize(st), "status");
    CK(cudaMemsetAsync(dstatus, 0, sizeof(int), st), "status");
    *out = h;
    return SC_OK;
  }

  // C (compact FP64) = A' B over column segments of two strided blocks.  FP32 with tensor
  // cores selected -> tcgen05 kernel; otherwise the CUDA-core kernel.
  cudaError_t gram_seg(const T* A, long long lda, std::initializer_list<Seg> sa, const T* B,
                       long long ldb, std::initializer_list<Seg> sb, double* C, int ldc,
                       bool sym) {
    std::vector<Seg> va(sa), vb(sb);
    if constexpr (sizeof(T) == 4) {
      if (use_tc) {
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
        return gram_tc(st, al, n, (const float*)A, lda, spa, pa, (int)va.size(), (const float*)B,
                       ldb, spb, pb, (int)vb.size(), C, ldc, sym, dstatus, c->probe_spins());
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
    return gram<T>(st, al, n, ca, cb, C, ldc, sym, 0);
  }

  // The small dense solves, in T or (dense64) in FP64 with the result cast to T.
  cudaError_t chol(int ka, const double* Gm, T* out, int* fail_col = nullptr, int keep = 0,
                   int* pflag = nullptr, int ndrop = 0, int* ndropped = nullptr,
                   double rfloor = 0.0, double pfloor = 0.0) {
    if (!dense64)
      return chol_inv<T>(st, al, ka, Gm, ka, out, dstatus, pivot_tol, fail_col, keep, pflag, ndrop,
                         ndropped, rfloor, pfloor);
    cudaError_t e = chol_inv<double>(st, al, ka, Gm, ka, Gd, dstatus, pivot_tol, fail_col, keep,
                                     pflag, ndrop, ndropped, rfloor, pfloor);
    if (e == cudaSuccess) e = cast_mat<T>(st, ka, ka, Gd, ka, out, ka, 1.0);
    return e;
  }
  cudaError_t rr(int m, const double* Gm, int* pflag = nullptr, int mP = 0,
                 int* nfallback = nullptr) {
    if (!dense64) return rr_eig<T>(st, al, m, K, Gm, m, theta, Y, dstatus, pflag, mP, nfallback);
    cudaError_t e = rr_eig<double>(st, al, m, K, Gm, m, theta, Yd, dstatus, pflag, mP, nfallback);
    if (e == cudaSuccess) e = cast_mat<T>(st, m, K, Yd, K, Y, K, 1.0);
    return e;
  }

  // V (n x cols, stride ldv) <- V - Yc (Yc' V): the part of V in the complement of Yc.
  cudaError_t project_off(T* V, long long ldv, int cols) {
    cudaError_t e = gram_seg(Yc, ldyc, {{0, kc}}, V, ldv, {{0, cols}}, Gy, cols, false);
    if (e == cudaSuccess) e = cast_mat<T>(st, kc, cols, Gy, cols, Ty, cols, -1.0);
    if (e == cudaSuccess)
      e = tall(st, n, cat<T>(Yc, ldyc, kc), Ty, cols, cols, V, ldv, V, ldv, (T)1);
    return e;
  }

  // ---- autotuned kernel choices (tune.cu) --------------------------------------------------
  static int log2ceil(long long x) {
    int l = 0;
    while ((1LL << l) < x) ++l;
    return l;
  }
  T* tune_scratch = nullptr;  // n x (2 kp + 8): outputs of the update variants being timed
  // The tall update on CUDA cores (variant 0) or tensor cores (variant 1, FP32 mixed only),
  // whichever the autotuner measured faster for this (n bucket, columns, segments); without a
  // measurement, tensor cores from n = 250,000 on.
  int tall_variant(cudaStream_t s, const Cat3<T>& A, const TallSeg<T>& s0, const TallSeg<T>& s1,
                   T beta) {
    if constexpr (sizeof(T) != 4) {
      return 0;
    } else {
      if (!use_tc) return 0;
      const int fallback = n >= 250000 ? 1 : 0;
      char key[128];
      snprintf(key, sizeof(key), "tall/f32/n2=%d/a=%d/b=%d/seg=%d", log2ceil(n), A.cols(),
               s0.b + s1.b, A.nblk);
      return tune_pick(key, "tall", s, 2, fallback, [&](int v) -> cudaError_t {
        if (!tune_scratch) {
          tune_scratch = get<T>((size_t)n * (2 * kp + 8));
          if (!tune_scratch) return cudaErrorMemoryAllocation;
          // allocated in the order of the run's stream; the second stream may use it next
          cudaStreamSynchronize(st);
        }
        const long long b0 = (s0.b + 3) & ~3, lds = b0 + ((s1.b + 3) & ~3);
        TallSeg<T> a0 = s0, a1 = s1;
        a0.out = tune_scratch;
        a0.ldo = lds;
        a1.out = tune_scratch + b0;
        a1.ldo = lds;
        return tall_gemm2<T>(s, n, A, a0, a1, beta, dstatus, v == 1);
      });
    }
  }
  cudaError_t tall2(cudaStream_t s, long long nn, const Cat3<T>& A, const TallSeg<T>& s0,
                    const TallSeg<T>& s1, T beta) {
    return tall_gemm2<T>(s, nn, A, s0, s1, beta, dstatus, tall_variant(s, A, s0, s1, beta) == 1);
  }
  cudaError_t tall(cudaStream_t s, long long nn, const Cat3<T>& A, const T* W, int ldw, int b,
                   T* out, long long ldo, const T* Cin, long long ldc, T beta) {
    TallSeg<T> s0{out, ldo, Cin, ldc, W, ldw, 0, b};
    TallSeg<T> s1{};
    return tall2(s, nn, A, s0, s1, beta);
  }
  // SpMM with the kernel shape (lanes per row x chunks per lane) the autotuner measured fastest
  // for this (n bucket, average degree bucket, columns).
  cudaError_t spmm(const T* V, long long ldv, T* Yo, long long ldy, int k) {
    const int Wd = 16 / sizeof(T);
    const int nvec = (k + Wd - 1) / Wd;
    int list[16];
    const int cnt = nvec <= 128 ? spmm_shapes(nvec, list) : 0;
    if (cnt <= 1) return spmm_lap<T>(st, g->csr, V, ldv, Yo, ldy, k, -1);
    char key[128];
    snprintf(key, sizeof(key), "spmm/%s/n2=%d/deg2=%d/k=%d", sizeof(T) == 4 ? "f32" : "f64",
             log2ceil(n), log2ceil(std::max<long long>(1, g->csr.nnz / std::max(1, n))), k);
    const int v = tune_pick(key, "spmm", st, cnt, 0, [&](int i) {
      return spmm_lap<T>(st, g->csr, V, ldv, Yo, ldy, k, list[i]);
    });
    return spmm_lap<T>(st, g->csr, V, ldv, Yo, ldy, k, list[v]);
  }

  // Cholesky-QR of V (n x kc, stride ldv) into out (stride ldo); failure -> *failed.
  int cholqr_step(const T* V, long long ldv, int kc, T* out, long long ldo, bool* failed) {
    CK(gram_seg(V, ldv, {{0, kc}}, V, ldv, {{0, kc}}, G, kc, true), "gram");
    CK(chol(kc, G, Tm), "chol");
    int hs = 0;
    int rc = read_status(&hs);
    if (rc != SC_OK) return rc;
    if (hs & 32) return fail(c, SC_ETIMEOUT, "a bounded device wait gave up");
    *failed = (hs & (ST_CHOL_FAIL | ST_NONFINITE)) != 0;
    if (*failed) return SC_OK;
    CK(tall(st, n, cat<T>(V, ldv, kc), Tm, kc, kc, out, ldo, nullptr, 0, (T)0), "tall");
    return SC_OK;
  }

  int setup(const float* X0, int32_t x0_rows) override {
    if (!ev0) {
      cudaEventCreate(&ev0);
      cudaEventCreate(&ev1);
      cudaEventCreateWithFlags(&evf, cudaEventDisableTiming);
      cudaEventCreateWithFlags(&evj, cudaEventDisableTiming);
      CK(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking), "stream");
    }
    const int mmax = 3 * K;
    S = get<T>((size_t)n * ld3, true);
    LS = get<T>((size_t)n * ld3, true);
    S2 = get<T>((size_t)n * ld3, true);
    LS2 = get<T>((size_t)n * ld3, true);
    T1 = get<T>((size_t)n * kp, true);
    W1 = get<T>((size_t)n * 2 * kp, true);
    Q1 = get<T>((size_t)n * 2 * kp, true);
    G = get<double>((size_t)mmax * mmax);
    if (dense64) {
      Gd = get<double>((size_t)mmax * mmax);
      Yd = get<double>((size_t)mmax * K);
      if (!Gd || !Yd) return fail(c, SC_ENOMEM, "sc_lobpcg: out of device memory or HBM budget");
    }
    Tm = get<T>((size_t)mmax * mmax);
    TmA = get<T>((size_t)mmax * mmax);
    TmB = get<T>((size_t)mmax * mmax);
    Y = get<T>((size_t)mmax * K);
    theta = get<double>(K);
    rho2 = get<double>(K);
    dcols = get<int>(K);
    dfail = get<int>(1);
    dP = get<int>(1);
    dfb = get<int>(1);
    ddrop = get<int>(1);
    dstatus = get<int>(1, true);
    if (!S || !LS || !S2 || !LS2 || !T1 || !W1 || !Q1 || !G || !Tm || !TmA ||
        !TmB || !Y ||
        !theta || !rho2 || !dcols || !dfail || !dP || !dfb || !ddrop || !dstatus)
      return fail(c, SC_ENOMEM, "sc_lobpcg: out of device memory or HBM budget");
    {
      int one = 1, zero = 0;
      CK(cudaMemcpyAsync(dP, &one, sizeof(int), cudaMemcpyHostToDevice, st), "flags");
      CK(cudaMemcpyAsync(dfb, &zero, sizeof(int), cudaMemcpyHostToDevice, st), "flags");
      CK(cudaMemcpyAsync(ddrop, &zero, sizeof(int), cudaMemcpyHostToDevice, st), "flags");
    }
    // ---- start block: given X0 (top x0_rows rows, zero fill below), the resident block of
    //      the previous call (warm start), or a seeded Gaussian block generated on the device
    const float* src = nullptr;
    int rows = 0;
    bool dev_src = false;
    if (X0d) {
      // an FP64 host start block: staged on the device, then narrowed to T (or copied)
      rows = x0_rows > 0 ? std::min(x0_rows, n) : n;
      double* tmp = get<double>((size_t)rows * K);
      if (!tmp) return fail(c, SC_ENOMEM, "sc_lobpcg: start block");
      const long long sp = x0_pitch > 0 ? x0_pitch : K;
      CK(cudaMemcpy2DAsync(tmp, sizeof(double) * K, X0d, sizeof(double) * sp, sizeof(double) * K,
                           rows, cudaMemcpyHostToDevice, st), "x0");
      if constexpr (sizeof(T) == 8) {
        CK(cudaMemcpy2DAsync(S, sizeof(T) * ld3, tmp, sizeof(double) * K, sizeof(double) * K, rows,
                             cudaMemcpyDeviceToDevice, st), "x0");
      } else {
        CK((convert_mat<double, T>(st, rows, K, tmp, K, S, ld3)), "x0");
      }
    } else if (X0) {
      src = X0;
      rows = x0_rows > 0 ? std::min(x0_rows, n) : n;
    } else if (g->X && g->K == K && !o.cold) {
      src = g->X;
      rows = n;
      dev_src = true;
    }
    if (X0d) {
      // staged above
    } else if (!src) {
      CK(gauss_block<T>(st, n, K, stream_key(o.seed, 1, 0), S, ld3), "x0");
    } else if constexpr (sizeof(T) == 4) {
      const long long sp = (!dev_src && x0_pitch > 0) ? x0_pitch : K;
      CK(cudaMemcpy2DAsync(S, sizeof(T) * ld3, src, sizeof(float) * sp, sizeof(float) * K, rows,
                           dev_src ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st), "x0");
    } else {
      // the FP32 start block widened to FP64 on the device (a host block is copied first)
      const float* fsrc = src;
      float* tmp = nullptr;
      if (!dev_src) {
        tmp = get<float>((size_t)rows * K);  // tracked: freed with the run on every path
        if (!tmp) return fail(c, SC_ENOMEM, "sc_lobpcg: start block");
        const long long sp = x0_pitch > 0 ? x0_pitch : K;
        CK(cudaMemcpy2DAsync(tmp, sizeof(float) * K, src, sizeof(float) * sp, sizeof(float) * K,
                             rows, cudaMemcpyHostToDevice, st), "x0");
        fsrc = tmp;
      }
      CK((convert_mat<float, T>(st, rows, K, fsrc, K, S, ld3)), "x0");
    }
    CK(cudaStreamSynchronize(st), "x0");
    CK(cudaEventRecord(ev0, st), "event");
    l0 = launches_total();
    if (kc > 0) {
      Gy = get<double>((size_t)kc * 2 * kp);
      Ty = get<T>((size_t)kc * 2 * kp);
      if (!Gy || !Ty) return fail(c, SC_ENOMEM, "sc_lobpcg: out of device memory or HBM budget");
      CK(project_off(S, ld3, K), "constraint");
    }
    // X <- CholQR(CholQR(X0)):  X slot -> T1 -> X slot
    bool bad = false;
    int rc = cholqr_step(S, ld3, K, T1, kp, &bad);
    if (rc != SC_OK) return rc;
    if (!bad) rc = cholqr_step(T1, kp, K, S, ld3, &bad);
    if (rc != SC_OK) return rc;
    if (bad) return fail(c, SC_EBREAKDOWN, "start block is rank deficient");
    CK(spmm(S, ld3, LS, ld3, K), "spmm");
    // S'LS is symmetric in exact arithmetic: the upper tiles are computed and mirrored
    CK(gram_seg(S, ld3, {{0, K}}, LS, ld3, {{0, K}}, G, K, true), "gram");
    CK(rr(K, G), "rr");
    CK(tall(st, n, cat<T>(S, ld3, K), Y, K, K, S2, ld3, nullptr, 0, (T)0), "tall");
    CK(tall(st, n, cat<T>(LS, ld3, K), Y, K, K, LS2, ld3, nullptr, 0, (T)0), "tall");
    std::swap(S, S2);
    std::swap(LS, LS2);
    CK(residual<T>(st, al, n, K, S, LS, ld3, theta, S + kp, rho2, pdeg), "residual");
    it = 0;
    over = o.iters <= 0;
    Sa = S;
    return SC_OK;
  }

  // Fixed-pass solves (no host decision between passes) replay the pass from a CUDA graph: the
  // pass is the same launch sequence every time except that S / S2 and LS / LS2 swap roles, so
  // one executable graph per buffer parity is recorded and relaunched.  Recording starts after
  // one pass with P has run eagerly, by when the autotuner has measured every shape and the
  // run's allocator holds a scratch block of every size, so a recorded pass allocates nothing.
  // The passes that re-orthonormalize X, and passes while a profile or a test hook is armed,
  // run eagerly; a recording that fails turns graphs off for the run (the pass then runs
  // eagerly, with the same kernels).
  int pass() override {
    if (over) return SC_OK;
    if (graph_eligible()) {
      const int par = S == Sa ? 0 : 1;
      if (!gexec[par] && eager_p >= 1) record(par);
      if (gexec[par]) {
        CK(cudaGraphLaunch(gexec[par], st), "graph");
        note_launches(glaunch[par]);
        g_graph_replays.fetch_add(1, std::memory_order_relaxed);
        std::swap(S, S2);
        std::swap(LS, LS2);
        ++done_passes;
        if (++it >= o.iters) over = true;
        return SC_OK;
      }
    }
    const bool withP = haveP;
    const int rc = pass_body();
    if (rc == SC_OK && withP) ++eager_p;
    return rc;
  }
  bool graph_eligible() const {
    return graphs && haveP && (done_passes + 1) % kReorth != 0 && c->inject_kind == 0 &&
           !prof_active();
  }
  void record(int par) {
    T *s0 = S, *s1 = S2, *l0s = LS, *l1s = LS2;
    const bool hp = haveP, ov = over;
    const int dp = done_passes, it0 = it;
    const uint64_t k0 = t_launches;
    cudaGraph_t gr = nullptr;
    bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      ra.capturing = true;
      ra.miss = false;
      const int rc = pass_body();
      ra.capturing = false;
      const cudaError_t ec = cudaStreamEndCapture(st, &gr);
      ok = rc == SC_OK && ec == cudaSuccess && gr != nullptr && !ra.miss;
    }
    const uint64_t k = t_launches - k0;
    unnote_launches(k);
    // the pass was recorded, not run: its host-side state changes are undone
    S = s0;
    S2 = s1;
    LS = l0s;
    LS2 = l1s;
    haveP = hp;
    over = ov;
    done_passes = dp;
    it = it0;
    if (ok) {
      cudaGraphExec_t ex = nullptr;
      ok = cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess;
      if (ok) {
        gexec[par] = ex;
        glaunch[par] = k;
      }
    }
    if (gr) cudaGraphDestroy(gr);
    if (!ok) {
      graphs = false;
      cudaGetLastError();
      c->err.clear();
    }
  }

  // One LOBPCG pass (Sec. II.B), issued on the run's stream.  The host reads the residual
  // norms between passes only when it has to decide something (a stopping tolerance or soft
  // locking); otherwise passes are issued back to back without synchronization.
  // The pass in stages around its small dense solves and its SpMM, so that a lockstep batch
  // can issue each of those for all of its runs in one launch (sc_lobpcg_batch); a single run
  // calls the stages and the solves in order (pass_body).  ps_* hold the pass's active set.
  std::vector<int> ps_act;
  int ps_ka = 0, ps_w = 0, ps_offP = 0;
  bool ps_all = true;
  T *ps_WR = nullptr, *ps_WP = nullptr;
  long long ps_ldw = 0;

  int pass_body() {
    bool go = false;
    int rc = pass_select(&go);
    if (rc != SC_OK || !go) return rc;
    if ((rc = stage_project()) != SC_OK) return rc;
    CK(chol_a(), "chol");
    if ((rc = stage_second_gram()) != SC_OK) return rc;
    CK(chol_b(), "chol");
    if ((rc = stage_images_pre()) != SC_OK) return rc;
    if ((rc = stage_spmm()) != SC_OK) return rc;
    if ((rc = stage_rr_gram()) != SC_OK) return rc;
    CK(rr_pass(), "rr");
    return stage_update();
  }

  // Active set: every column, unless a tolerance asks the host to look at the residuals.
  int pass_select(bool* go) {
    *go = false;
    const bool watch = o.tol_abs > 0 || o.tol_lock > 0;
    std::vector<int>& act = ps_act;
    act.clear();
    if (watch) {
      int hs = 0;
      CK(cudaMemcpyAsync(hrho.data(), rho2, sizeof(double) * K, cudaMemcpyDeviceToHost, st), "rho");
      CK(cudaMemcpyAsync(&hs, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st), "rho");
      CK(cudaStreamSynchronize(st), "rho");
      if (hs) {  // a breakdown or a timed-out wait: stop here, finish() reports it
        over = true;
        return SC_OK;
      }
      double mx = 0.0;
      for (int j = 0; j < K; ++j) {
        double r = std::sqrt(std::max(hrho[j], 0.0));
        mx = std::max(mx, r);
        if (r > o.tol_lock) act.push_back(j);
      }
      if (o.tol_abs > 0 && mx <= o.tol_abs) {
        converged = 1;
        over = true;
        return SC_OK;
      }
      if (act.empty()) {
        converged = o.tol_abs > 0 ? 1 : 0;
        over = true;
        return SC_OK;
      }
    } else {
      act.resize(K);
      for (int j = 0; j < K; ++j) act[j] = j;
    }
    const int ka = (int)act.size();
    ps_ka = ka;
    ps_all = ka == K;
    T* Rslot = S + kp;
    T* Pslot = S + 2 * kp;
    // Working copies of the active R and P columns: the S slots themselves when every column
    // is active; otherwise gathered into W1 = [R_a | P_a] (n x 2kp).
    ps_WR = Rslot;
    ps_WP = Pslot;
    ps_ldw = ld3;
    ps_offP = kp;
    if (!ps_all) {
      CK(cudaMemcpyAsync(dcols, act.data(), sizeof(int) * ka, cudaMemcpyHostToDevice, st), "cols");
      CK(gather_cols<T>(st, n, Rslot, ld3, W1, 2 * kp, dcols, ka), "gather");
      ps_WR = W1;
      ps_WP = W1 + kp;
      ps_ldw = 2 * kp;
      if (haveP) CK(gather_cols<T>(st, n, Pslot, ld3, ps_WP, ps_ldw, dcols, ka), "gather");
      // the gathered column list must stay valid until the copy ran
      CK(cudaStreamSynchronize(st), "cols");
    }
    ps_w = haveP ? 2 * ka : ka;
    *go = true;
    return SC_OK;
  }

  // (0) hard locking: the residual block leaves the span of the constraint block (P and X stay
  //     in its complement as combinations of blocks that are)
  // (1) project [R_a P_a] against X: F = X'[R_a P_a]; [R_a P_a] -= X F in one pass over X
  // (2) first half of the Cholesky-QR of [R_a P_a]: its Gram, into G
  int stage_project() {
    const int ka = ps_ka, w = ps_w, offP = ps_offP;
    T *WR = ps_WR, *WP = ps_WP;
    const long long ldw = ps_ldw;
    if (kc > 0) CK(project_off(WR, ldw, ka), "constraint");
    if (haveP)
      CK(gram_seg(S, ld3, {{0, K}}, WR, ldw, {{0, ka}, {offP, ka}}, G, w, false), "gram");
    else
      CK(gram_seg(S, ld3, {{0, K}}, WR, ldw, {{0, ka}}, G, w, false), "gram");
    CK(cast_mat<T>(st, K, w, G, w, Tm, w, -1.0), "cast");
    {
      TallSeg<T> sr{WR, ldw, WR, ldw, Tm, w, 0, ka};
      TallSeg<T> sp{WP, ldw, WP, ldw, Tm + ka, w, 0, haveP ? ka : 0};
      CK(tall2(st, n, cat<T>(S, ld3, K), sr, sp, (T)1), "tall");
    }
    // Cholesky-QR twice of [R_a P_a] (R first, so P is orthogonalized against R too), into the
    // R and P slots.  A breakdown inside the P columns is handled on the device: the kernel
    // keeps the R transform, zeroes P's, and clears *dP, which the Rayleigh-Ritz step reads to
    // solve without P.  A residual column whose pivot falls below the tolerance (it lies in the
    // span of X and the R columns before it, to working accuracy: converged columns' residuals
    // sink to rounding noise) is dropped from this pass's basis, and so are residual and
    // direction columns whose norms are at rounding level (res_floor, dir_floor); their zero
    // columns are kept out of the Rayleigh-Ritz solve.
    if (haveP)
      CK(gram_seg(WR, ldw, {{0, ka}, {offP, ka}}, WR, ldw, {{0, ka}, {offP, ka}}, G, w, true), "gram");
    else
      CK(gram_seg(WR, ldw, {{0, ka}}, WR, ldw, {{0, ka}}, G, w, true), "gram");
    return SC_OK;
  }
  cudaError_t chol_a() {
    return chol(ps_w, G, TmA, dfail, ps_ka, haveP ? dP : nullptr, ps_ka, ddrop, res_floor,
                dir_floor);
  }
  int stage_second_gram() {
    const int wq = ps_w;
    Cat3<T> Vw = haveP ? cat<T>(ps_WR, ps_ldw, ps_ka, ps_WP, ps_ldw, ps_ka)
                       : cat<T>(ps_WR, ps_ldw, ps_ka);
    CK(tall(st, n, Vw, TmA, wq, wq, Q1, 2 * kp, nullptr, 0, (T)0), "tall");
    CK(gram_seg(Q1, 2 * kp, {{0, wq}}, Q1, 2 * kp, {{0, wq}}, G, wq, true), "gram");
    return SC_OK;
  }
  cudaError_t chol_b() {
    return chol(ps_w, G, TmB, dfail, ps_ka, haveP ? dP : nullptr, ps_ka, nullptr);
  }
  int stage_images_pre() {
    const int wq = ps_w, ka = ps_ka;
    if (haveP) {
      // [R P] = Q1 TmB in one pass over Q1: two output segments (TmB is upper triangular, so
      // the R columns take zeros from Q1's P columns)
      TallSeg<T> sr{S + kp, ld3, nullptr, 0, TmB, wq, 0, ka};
      TallSeg<T> sp{S + 2 * kp, ld3, nullptr, 0, TmB + ka, wq, 0, ka};
      CK(tall2(st, n, cat<T>(Q1, 2 * kp, wq), sr, sp, (T)0), "tall");
    } else {
      // R = Q1_R T_RR uses only the R columns of Q1
      CK(tall(st, n, cat<T>(Q1, 2 * kp, ka), TmB, wq, ka, S + kp, ld3, nullptr, 0, (T)0), "tall");
    }
    return SC_OK;
  }
  // (3) [LR_a LP_a] = L [R_a P_a]: the one multiplication by L of the pass (Sec. III), taken on
  //     the orthonormalized block so that its images are products with L rather than images
  //     carried through the Cholesky factors (in FP32 those lose accuracy as fast as the
  //     factors grow ill-conditioned near convergence).  With every column active the R and P
  //     slots are adjacent (R slot padding is zero) and one SpMM covers both.
  bool spmm_single() const { return haveP && ps_all; }
  int stage_spmm() {
    const int ka = ps_ka;
    if (spmm_single()) {
      CK(spmm(S + kp, ld3, LS + kp, ld3, kp + ka), "spmm");
    } else {
      CK(spmm(S + kp, ld3, LS + kp, ld3, ka), "spmm");
      if (haveP) CK(spmm(S + 2 * kp, ld3, LS + 2 * kp, ld3, ka), "spmm");
    }
    return SC_OK;
  }
  int stage_rr_gram() {
    const int ka = ps_ka;
    // test hook: this pass's direction block is reported as broken down, as the Cholesky-QR
    // does when P has sunk into span{X, R} (the Rayleigh-Ritz step then runs without P)
    if (haveP && c->inject_kind == SC_INJECT_P_BREAKDOWN && done_passes == c->inject_arg)
      CK(cudaMemsetAsync(dP, 0, sizeof(int), st), "inject");
    // (4) Rayleigh-Ritz on S = [X R_a P_a]; S'LS is symmetric in exact arithmetic: the upper
    //     tiles are computed and mirrored
    const int m = rr_m();
    if (haveP)
      CK(gram_seg(S, ld3, {{0, K}, {kp, ka}, {2 * kp, ka}}, LS, ld3, {{0, K}, {kp, ka}, {2 * kp, ka}}, G, m, true), "gram");
    else
      CK(gram_seg(S, ld3, {{0, K}, {kp, ka}}, LS, ld3, {{0, K}, {kp, ka}}, G, m, true), "gram");
    return SC_OK;
  }
  int rr_m() const { return K + ps_ka + (haveP ? ps_ka : 0); }
  cudaError_t rr_pass() { return rr(rr_m(), G, haveP ? dP : nullptr, ps_ka, dfb); }
  // (5) update into S2 / LS2: P = [R_a P_a] Y_RP, X = X Y_X + P (L-images alike);
  //     R = LX - X theta
  int stage_update() {
    const int ka = ps_ka;
    const bool useP = haveP;
    T* Rslot = S + kp;
    T* LRslot = LS + kp;
    T* Pslot = S + 2 * kp;
    T* LPslot = LS + 2 * kp;
    const T* Yrp = Y + (size_t)K * K;
    Cat3<T> RP = useP ? cat<T>(Rslot, ld3, ka, Pslot, ld3, ka) : cat<T>(Rslot, ld3, ka);
    Cat3<T> LRP = useP ? cat<T>(LRslot, ld3, ka, LPslot, ld3, ka) : cat<T>(LRslot, ld3, ka);
    fork();  // the L-images on the second stream
    CK(tall(st2, n, LRP, Yrp, K, K, LS2 + 2 * kp, ld3, nullptr, 0, (T)0), "tall");
    CK(tall(st2, n, cat<T>(LS, ld3, K), Y, K, K, LS2, ld3, LS2 + 2 * kp, ld3, (T)1), "tall");
    CK(tall(st, n, RP, Yrp, K, K, S2 + 2 * kp, ld3, nullptr, 0, (T)0), "tall");
    CK(tall(st, n, cat<T>(S, ld3, K), Y, K, K, S2, ld3, S2 + 2 * kp, ld3, (T)1), "tall");
    join();
    std::swap(S, S2);
    std::swap(LS, LS2);
    haveP = true;
    // Every kReorth passes X is re-orthonormalized by Cholesky-QR, LX transformed alike.  In
    // exact arithmetic X stays orthonormal and the transform is the identity; in FP32 its
    // departure from orthonormality grows pass by pass, and with a basis that is not
    // orthonormal the standard Rayleigh-Ritz solve lets Ritz vectors merge.
    if ((done_passes + 1) % kReorth == 0) {
      CK(gram_seg(S, ld3, {{0, K}}, S, ld3, {{0, K}}, G, K, true), "gram");
      CK(chol(K, G, Tm), "chol");
      CK(tall(st, n, cat<T>(S, ld3, K), Tm, K, K, T1, kp, nullptr, 0, (T)0), "tall");
      CK(tall(st, n, cat<T>(LS, ld3, K), Tm, K, K, W1, kp, nullptr, 0, (T)0), "tall");
      CK(cudaMemcpy2DAsync(S, sizeof(T) * ld3, T1, sizeof(T) * kp, sizeof(T) * K, n,
                           cudaMemcpyDeviceToDevice, st), "reorth");
      CK(cudaMemcpy2DAsync(LS, sizeof(T) * ld3, W1, sizeof(T) * kp, sizeof(T) * K, n,
                           cudaMemcpyDeviceToDevice, st), "reorth");
    }
    CK(residual<T>(st, al, n, K, S, LS, ld3, theta, S + kp, rho2, pdeg), "residual");
    ++done_passes;
    if (++it >= o.iters) over = true;
    return SC_OK;
  }

  int finish(float* X_out, sc_eig_info* info) override {
    CK(cudaEventRecord(ev1, st), "event");
    CK(cudaStreamSynchronize(st), "sync");
    int st_final = 0;
    int rc = read_status(&st_final);
    if (rc != SC_OK) return rc;
    if (st_final & 32) return fail(c, SC_ETIMEOUT, "a bounded device wait gave up");
    if (st_final & ST_NONFINITE) return fail(c, SC_EBREAKDOWN, "non-finite values in Rayleigh-Ritz");
    if (st_final & ST_CHOL_FAIL) return fail(c, SC_EBREAKDOWN, "residual block lost rank");
    int fallbacks = 0, dropped = 0;
    CK(cudaMemcpyAsync(&fallbacks, dfb, sizeof(int), cudaMemcpyDeviceToHost, st), "out");
    CK(cudaMemcpyAsync(&dropped, ddrop, sizeof(int), cudaMemcpyDeviceToHost, st), "out");
    CK(cudaMemcpyAsync(hrho.data(), rho2, sizeof(double) * K, cudaMemcpyDeviceToHost, st), "out");
    CK(cudaMemcpyAsync(hth.data(), theta, sizeof(double) * K, cudaMemcpyDeviceToHost, st), "out");
    // resident block (float, n x K) for warm starts and the embedding
    if (!g->X || g->K != K) {
      if (g->X) ctx_free(c, g->X);
      g->X = (float*)run_alloc(&ra, sizeof(float) * (size_t)n * K);
      g->K = g->X ? K : 0;
    }
    if (g->X) {
      if constexpr (sizeof(T) == 4) {
        CK(cudaMemcpy2DAsync(g->X, sizeof(float) * K, S, sizeof(T) * ld3, sizeof(float) * K, n,
                             cudaMemcpyDeviceToDevice, st), "resident");
      } else {
        CK((convert_mat<T, float>(st, n, K, S, ld3, g->X, K)), "resident");
        if (X_out)
          CK(cudaMemcpyAsync(X_out, g->X, sizeof(float) * (size_t)n * K, cudaMemcpyDeviceToHost,
                             st), "resident");
        CK(cudaStreamSynchronize(st), "resident");
      }
    }
    if (X_out && sizeof(T) == 4) {
      CK(cudaMemcpy2DAsync(X_out, sizeof(float) * K, S, sizeof(T) * ld3, sizeof(float) * K, n,
                           cudaMemcpyDeviceToHost, st), "xout");
    }
    if (Xout64) {
      if constexpr (sizeof(T) == 8) {
        CK(cudaMemcpy2DAsync(Xout64, sizeof(double) * K, S, sizeof(T) * ld3, sizeof(double) * K, n,
                             cudaMemcpyDeviceToHost, st), "xout");
      } else {
        double* tmp = get<double>((size_t)n * K);
        if (!tmp) return fail(c, SC_ENOMEM, "sc_lobpcg64: result block");
        CK((convert_mat<T, double>(st, n, K, S, ld3, tmp, K)), "xout");
        CK(cudaMemcpyAsync(Xout64, tmp, sizeof(double) * (size_t)n * K, cudaMemcpyDeviceToHost,
                           st), "xout");
      }
    }
    CK(cudaStreamSynchronize(st), "sync");
    if (info) {
      info->K = K;
      info->iters_done = done_passes;
      info->fallbacks = fallbacks;
      info->dropped = dropped;
      info->converged = converged;
      for (int j = 0; j < K; ++j) {
        info->lambda[j] = hth[j];
        info->resid[j] = std::sqrt(std::max(hrho[j], 0.0));
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev0, ev1);
      info->ms = ms;
      info->kernels = launches_total() - l0;
    }
    if (o.tol_abs > 0 && !converged) return fail(c, SC_ENOTCONV, "tolerance not reached");
    return SC_OK;
  }
};

RunBase* make_run(sc_ctx* c, sc_graph* g, int K, const sc_lobpcg_opts* o, cudaStream_t st) {
  if (o->prec == SC_PREC_FP64) return new LobRun<double>(c, g, K, o, st);
  return new LobRun<float>(c, g, K, o, st);
}

int check_lobpcg_args(sc_ctx* c, sc_graph* g, int K, const sc_lobpcg_opts* o) {
  if (!c) return SC_EINVAL;
  if (!g || !o || K < 1 || K > SC_MAX_K || o->iters < 0)
    return fail(c, SC_EINVAL, "sc_lobpcg: invalid argument (null pointer or size out of range)");
  if ((int64_t)3 * K > g->csr.n) return fail(c, SC_EINVAL, "sc_lobpcg: need 3K <= n");
  if (o->prec < SC_PREC_MIXED || o->prec > SC_PREC_MIXED_DD) return fail(c, SC_EINVAL, "bad precision");
  if (o->precond != SC_PRECOND_NONE && o->precond != SC_PRECOND_JACOBI)
    return fail(c, SC_EINVAL, "sc_lobpcg: unknown preconditioner");
  return SC_OK;
}

}  // namespace

namespace {

// Hard locking (Sec. IV): blocks of nb columns, each solved by a LobRun constrained to the
// complement of the Ritz vectors of the blocks before it (held in Yc, n x K).
template <typename T>
int lobpcg_blocks_t(sc_ctx* c, sc_graph* g, int K, int nb, const sc_lobpcg_opts* o,
                    const float* X0, float* X_out, sc_eig_info* info) {
  const int n = g->csr.n;
  Alloc al = alloc_of(c);
  const long long ldy = (K + 3) & ~3;  // 16-byte rows for the tensor-map Gram
  T* Yc = al.get<T>((size_t)n * ldy);
  if (!Yc) return fail(c, SC_ENOMEM, "sc_lobpcg_blocks: out of device memory or HBM budget");
  CK(cudaMemsetAsync(Yc, 0, sizeof(T) * (size_t)n * ldy, c->stream), "blocks");
  sc_eig_info acc{};
  acc.K = K;
  acc.converged = 1;
  int rc = SC_OK;
  for (int b0 = 0, b = 0; b0 < K && rc == SC_OK; b0 += nb, ++b) {
    const int kb = std::min(nb, K - b0);
    sc_lobpcg_opts ob = *o;
    ob.cold = 1;
    ob.seed = o->seed + (uint64_t)b;  // a distinct seeded start block for each block
    LobRun<T> r(c, g, kb, &ob, c->stream);
    r.Yc = Yc;
    r.kc = b0;
    r.ldyc = ldy;
    r.x0_pitch = X0 ? K : 0;
    rc = r.setup(X0 ? X0 + b0 : nullptr, 0);
    while (rc == SC_OK && !r.finished()) rc = r.pass();
    sc_eig_info bi{};
    if (rc == SC_OK) rc = r.finish(nullptr, &bi);
    if (rc != SC_OK) break;
    CK(cudaMemcpy2DAsync(Yc + b0, sizeof(T) * ldy, r.S, sizeof(T) * r.ld3, sizeof(T) * kb, n,
                         cudaMemcpyDeviceToDevice, c->stream), "blocks");
    for (int j = 0; j < kb; ++j) {
      acc.lambda[b0 + j] = bi.lambda[j];
      acc.resid[b0 + j] = bi.resid[j];
    }
    acc.iters_done += bi.iters_done;
    acc.fallbacks += bi.fallbacks;
    acc.dropped += bi.dropped;
    acc.converged = acc.converged && bi.converged;
    acc.ms += bi.ms;
    acc.kernels += bi.kernels;
  }
  if (rc == SC_OK) {
    // the n x K result as FP32: the graph's resident block and X_out
    if (g->X) ctx_free(c, g->X);
    g->X = (float*)ctx_alloc(c, sizeof(float) * (size_t)n * K);
    g->K = g->X ? K : 0;
    if (!g->X) {
      rc = fail(c, SC_ENOMEM, "sc_lobpcg_blocks: resident block");
    } else {
      if constexpr (sizeof(T) == 4) {
        CK(cudaMemcpy2DAsync(g->X, sizeof(float) * K, Yc, sizeof(T) * ldy, sizeof(float) * K, n,
                             cudaMemcpyDeviceToDevice, c->stream), "blocks");
      } else {
        CK((convert_mat<T, float>(c->stream, n, K, Yc, ldy, g->X, K)), "blocks");
      }
      if (X_out)
        CK(cudaMemcpyAsync(X_out, g->X, sizeof(float) * (size_t)n * K, cudaMemcpyDeviceToHost,
                           c->stream), "blocks");
    }
    CK(cudaStreamSynchronize(c->stream), "blocks");
  }
  al.put(Yc);
  cudaStreamSynchronize(c->stream);
  if (info && rc == SC_OK) *info = acc;
  return rc;
}

}  // namespace

int sc_lobpcg_blocks(sc_ctx* c, sc_graph* g, int K, int nb, const sc_lobpcg_opts* o,
                     const float* X0, float* X_out, sc_eig_info* info) {
  if (!c) return SC_EINVAL;
  if (!g || !o || K < 1 || K > SC_MAX_K || nb < 1 || nb > K || K > g->csr.n)
    return fail(c, SC_EINVAL, "sc_lobpcg_blocks: invalid argument (null pointer or size out of range)");
  int rc = check_lobpcg_args(c, g, nb, o);
  if (rc != SC_OK) return rc;
  cudaSetDevice(c->device);
  if (o->prec == SC_PREC_FP64) return lobpcg_blocks_t<double>(c, g, K, nb, o, X0, X_out, info);
  return lobpcg_blocks_t<float>(c, g, K, nb, o, X0, X_out, info);
}

int sc_lobpcg(sc_ctx* c, sc_graph* g, int K, const sc_lobpcg_opts* o, const float* X0,
              int32_t x0_rows, float* X_out, sc_eig_info* info) {
  int rc = check_lobpcg_args(c, g, K, o);
  if (rc != SC_OK) return rc;
  cudaSetDevice(c->device);
  RunBase* r = make_run(c, g, K, o, c->stream);
  rc = r->setup(X0, x0_rows);
  while (rc == SC_OK && !r->finished()) rc = r->pass();
  if (rc == SC_OK) rc = r->finish(X_out, info);
  delete r;
  return rc;
}

int sc_lobpcg64(sc_ctx* c, sc_graph* g, int K, const sc_lobpcg_opts* o, const double* X0,
                int32_t x0_rows, double* X_out, sc_eig_info* info) {
  int rc = check_lobpcg_args(c, g, K, o);
  if (rc != SC_OK) return rc;
  cudaSetDevice(c->device);
  if (o->prec == SC_PREC_FP64) {
    LobRun<double> r(c, g, K, o, c->stream);
    r.X0d = X0;
    r.Xout64 = X_out;
    rc = r.setup(nullptr, x0_rows);
    while (rc == SC_OK && !r.finished()) rc = r.pass();
    if (rc == SC_OK) rc = r.finish(nullptr, info);
    return rc;
  }
  LobRun<float> r(c, g, K, o, c->stream);
  r.X0d = X0;
  r.Xout64 = X_out;
  rc = r.setup(nullptr, x0_rows);
  while (rc == SC_OK && !r.finished()) rc = r.pass();
  if (rc == SC_OK) rc = r.finish(nullptr, info);
  return rc;
}

namespace {

// Lockstep batch: FP32 mixed-precision runs with the same fixed pass count advance together,
// and each pass's two Cholesky-QR transforms, its SpMM and its Rayleigh-Ritz solve go out for
// all runs at once -- one launch per kernel shape (descriptor tables written once, grouped by
// shape) on the batch stream, which joins the runs' streams before and after.  The Gram,
// update and residual kernels stay per run, on the runs' streams, where they overlap.  From
// the second lockstep pass on, the whole batch pass is recorded into one CUDA graph per buffer
// parity and relaunched.  Each run's results are bitwise its single-run results.
struct Lockstep {
  sc_ctx* c;
  std::vector<LobRun<float>*> r;
  cudaStream_t bs = nullptr;
  cudaEvent_t evb = nullptr;
  std::vector<cudaEvent_t> evr;
  void* dmem = nullptr;
  CholDesc* dchol[2] = {nullptr, nullptr};
  RrDesc* drr = nullptr;
  SpmmDesc* dspmm[2] = {nullptr, nullptr};
  std::vector<BatchGroup> gchol[2], grr;
  std::vector<LobRun<float>*> rr_one;  // solved one by one (no batched kernel shape)
  long long rows = 0;
  int nvec_max = 0, lock_passes = 0;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  uint64_t glaunch[2] = {0, 0};
  bool graphs = true;

  ~Lockstep() {
    for (cudaGraphExec_t& x : gexec)
      if (x) cudaGraphExecDestroy(x);
    if (bs) cudaStreamSynchronize(bs);
    if (dmem) ctx_free(c, dmem);
    for (cudaEvent_t e : evr) cudaEventDestroy(e);
    if (evb) cudaEventDestroy(evb);
    if (bs) cudaStreamDestroy(bs);
  }
  static bool eligible(const std::vector<RunBase*>& runs) {
    const char* v = std::getenv("SC_BATCH_LOCKSTEP");
    if (v && std::strcmp(v, "0") == 0) return false;
    if (runs.empty()) return false;
    int iters = -1;
    for (RunBase* b : runs) {
      auto* q = dynamic_cast<LobRun<float>*>(b);
      if (!q || q->dense64 || !q->use_tc || q->o.tol_abs > 0 || q->o.tol_lock > 0 || q->kc > 0)
        return false;
      if (iters >= 0 && q->o.iters != iters) return false;
      iters = q->o.iters;
      if ((q->kp + q->K + 3) / 4 > 128) return false;  // the SpMM's widest kernel shape
    }
    return true;
  }
  // batch stream after every run's work so far / every run after the batch stream
  void to_batch() {
    for (size_t q = 0; q < r.size(); ++q) {
      cudaEventRecord(evr[q], r[q]->st);
      cudaStreamWaitEvent(bs, evr[q], 0);
    }
  }
  void from_batch() {
    cudaEventRecord(evb, bs);
    for (auto* q : r) cudaStreamWaitEvent(q->st, evb, 0);
  }
  // Descriptor tables, after the first pass (every run has P from then on).
  int build() {
    if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess)
      return fail(c, SC_ECUDA, "stream creation failed");
    cudaEventCreateWithFlags(&evb, cudaEventDisableTiming);
    evr.resize(r.size());
    for (auto& e : evr) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    const char* ge = std::getenv("SC_CUDA_GRAPHS");
    graphs = !(ge && std::strcmp(ge, "0") == 0);
    std::vector<CholDesc> ca, cb;
    std::vector<RrDesc> rd;
    std::vector<SpmmDesc> sp[2];
    for (auto* q : r) {
      const int K = q->K, w = 2 * K, m = 3 * K;
      float* Wg = nullptr;
      if (size_t f = chol_batch_scratch(w)) {
        Wg = q->template get<float>(f);
        if (!Wg) return fail(c, SC_ENOMEM, "sc_lobpcg_batch: scratch");
      }
      CholDesc a{w, w, K, K, q->G, q->TmA, Wg, q->dstatus, q->dfail, q->dP, q->ddrop,
                 q->pivot_tol, q->res_floor, q->dir_floor};
      CholDesc b{w, w, K, K, q->G, q->TmB, Wg, q->dstatus, q->dfail, q->dP, nullptr,
                 q->pivot_tol, 0.0, 0.0};
      ca.push_back(a);
      cb.push_back(b);
      float* Ag = nullptr;
      float* tri = nullptr;
      float* lamx = nullptr;
      int* mx = nullptr;
      if (size_t f = rr_batch_scratch(m, K)) {
        Ag = q->template get<float>(f);
        if (!Ag) return fail(c, SC_ENOMEM, "sc_lobpcg_batch: scratch");
      }
      if (rr_batch_cluster(m)) {
        tri = q->template get<float>((size_t)3 * m);
        lamx = q->template get<float>((size_t)K);
        mx = q->template get<int>(1);
        if (!tri || !lamx || !mx) return fail(c, SC_ENOMEM, "sc_lobpcg_batch: scratch");
      }
      rd.push_back(RrDesc{m, K, m, K, q->G, q->theta, q->Y, q->dstatus, q->dP, q->dfb, Ag, tri,
                          lamx, mx});
      const int nv = (q->kp + K + 3) / 4;
      nvec_max = std::max(nvec_max, nv);
      // parity 0 = the pass starts with S at its setup buffer (Sa); the first pass has swapped
      const int cur = q->S == q->Sa ? 0 : 1;
      for (int par = 0; par < 2; ++par) {
        float* Sx = par == cur ? q->S : q->S2;
        float* LSx = par == cur ? q->LS : q->LS2;
        const CsrDev& g = q->g->csr;
        sp[par].push_back(SpmmDesc{rows, g.n, nv, g.row_ptr, g.col_idx, g.val, g.degf,
                                   Sx + q->kp, LSx + q->kp, q->ld3, q->ld3});
      }
      rows += q->n;
    }
    std::vector<int> one;
    chol_batch_plan(ca, gchol[0], one);
    chol_batch_plan(cb, gchol[1], one);
    rr_batch_plan(rd, grr, one);
    for (int i : one)
      for (auto* q : r)
        if (q->theta == rd[i].theta) rr_one.push_back(q);
    const size_t nb = r.size();
    const size_t bytes = 2 * nb * sizeof(CholDesc) + nb * sizeof(RrDesc) + 2 * nb * sizeof(SpmmDesc) + 64;
    dmem = ctx_alloc(c, bytes);
    if (!dmem) return fail(c, SC_ENOMEM, "sc_lobpcg_batch: descriptor tables");
    char* p = (char*)dmem;
    dchol[0] = (CholDesc*)p;
    dchol[1] = dchol[0] + nb;
    drr = (RrDesc*)(dchol[1] + nb);
    dspmm[0] = (SpmmDesc*)(drr + nb);
    dspmm[1] = dspmm[0] + nb;
    // the runs' setup and first pass were issued on their streams (and the table memory on the
    // context's): the tables go in after them
    for (auto* q : r) CK(cudaStreamSynchronize(q->st), "batch");
    CK(cudaStreamSynchronize(c->stream), "batch");
    CK(cudaMemcpy(dchol[0], ca.data(), nb * sizeof(CholDesc), cudaMemcpyHostToDevice), "batch");
    CK(cudaMemcpy(dchol[1], cb.data(), nb * sizeof(CholDesc), cudaMemcpyHostToDevice), "batch");
    CK(cudaMemcpy(drr, rd.data(), nb * sizeof(RrDesc), cudaMemcpyHostToDevice), "batch");
    CK(cudaMemcpy(dspmm[0], sp[0].data(), nb * sizeof(SpmmDesc), cudaMemcpyHostToDevice), "batch");
    CK(cudaMemcpy(dspmm[1], sp[1].data(), nb * sizeof(SpmmDesc), cudaMemcpyHostToDevice), "batch");
    return SC_OK;
  }
  // One lockstep pass, issued (or recorded) on the runs' streams and the batch stream.
  int issue(int par) {
    int rc = SC_OK;
    for (auto* q : r) {
      bool go = false;
      if ((rc = q->pass_select(&go)) != SC_OK) return rc;
      if (!go) return fail(c, SC_EINVAL, "sc_lobpcg_batch: lockstep pass without work");
      if ((rc = q->stage_project()) != SC_OK) return rc;
    }
    to_batch();
    CK(chol_batch_launch(bs, dchol[0], gchol[0]), "chol");
    from_batch();
    for (auto* q : r)
      if ((rc = q->stage_second_gram()) != SC_OK) return rc;
    to_batch();
    CK(chol_batch_launch(bs, dchol[1], gchol[1]), "chol");
    from_batch();
    for (auto* q : r)
      if ((rc = q->stage_images_pre()) != SC_OK) return rc;
    to_batch();
    CK(spmm_batch_launch(bs, dspmm[par], (int)r.size(), rows, nvec_max), "spmm");
    from_batch();
    for (auto* q : r)
      if ((rc = q->stage_rr_gram()) != SC_OK) return rc;
    for (auto* q : rr_one) CK(q->rr_pass(), "rr");
    to_batch();
    CK(rr_batch_launch(bs, drr, grr), "rr");
    from_batch();
    for (auto* q : r)
      if ((rc = q->stage_update()) != SC_OK) return rc;
    return SC_OK;
  }
  void record(int par) {
    struct Saved {
      float *S, *S2, *LS, *LS2;
      bool haveP, over;
      int done, it;
    };
    std::vector<Saved> sv;
    for (auto* q : r) sv.push_back(Saved{q->S, q->S2, q->LS, q->LS2, q->haveP, q->over,
                                         q->done_passes, q->it});
    const uint64_t k0 = t_launches;
    cudaGraph_t gr = nullptr;
    bool ok = cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      from_batch();  // the runs' streams join the recording
      for (auto* q : r) {
        q->ra.capturing = true;
        q->ra.miss = false;
      }
      const int rc = issue(par);
      to_batch();  // and leave it
      bool miss = false;
      for (auto* q : r) {
        q->ra.capturing = false;
        miss = miss || q->ra.miss;
      }
      const cudaError_t ec = cudaStreamEndCapture(bs, &gr);
      ok = rc == SC_OK && ec == cudaSuccess && gr != nullptr && !miss;
    }
    const uint64_t k = t_launches - k0;
    unnote_launches(k);
    for (size_t i = 0; i < r.size(); ++i) {
      auto* q = r[i];
      q->S = sv[i].S;
      q->S2 = sv[i].S2;
      q->LS = sv[i].LS;
      q->LS2 = sv[i].LS2;
      q->haveP = sv[i].haveP;
      q->over = sv[i].over;
      q->done_passes = sv[i].done;
      q->it = sv[i].it;
    }
    if (ok) {
      cudaGraphExec_t ex = nullptr;
      ok = cudaGraphInstantiate(&ex, gr, 0) == cudaSuccess;
      if (ok) {
        gexec[par] = ex;
        glaunch[par] = k;
      }
    }
    if (gr) cudaGraphDestroy(gr);
    if (!ok) {
      graphs = false;
      cudaGetLastError();
      c->err.clear();
    }
  }
  int pass() {
    auto* q0 = r[0];
    const int par = q0->S == q0->Sa ? 0 : 1;
    const bool replayable = graphs && lock_passes >= 1 && (q0->done_passes + 1) % q0->kReorth != 0 &&
                            c->inject_kind == 0 && !prof_active();
    if (replayable && !gexec[par]) record(par);
    if (replayable && gexec[par]) {
      to_batch();
      CK(cudaGraphLaunch(gexec[par], bs), "graph");
      from_batch();
      note_launches(glaunch[par]);
      g_graph_replays.fetch_add(1, std::memory_order_relaxed);
      for (auto* q : r) {
        std::swap(q->S, q->S2);
        std::swap(q->LS, q->LS2);
        ++q->done_passes;
        if (++q->it >= q->o.iters) q->over = true;
      }
      ++lock_passes;
      return SC_OK;
    }
    const int rc = issue(par);
    if (rc == SC_OK) ++lock_passes;
    return rc;
  }
};

}  // namespace

static std::atomic<uint64_t> g_lockstep_passes{0};
uint64_t sc_ctx_batch_lockstep_passes(const sc_ctx*) { return g_lockstep_passes.load(); }

// Batched solves: each run on its own stream.  FP32 mixed-precision runs with one fixed pass
// count go in lockstep (Lockstep above); otherwise the runs are issued pass by pass in turn,
// and their kernels -- in particular the one-CTA small dense solves -- overlap on the device.
int sc_lobpcg_batch(sc_ctx* c, int count, sc_graph* const* graphs, const int* K,
                    const sc_lobpcg_opts* opts, sc_eig_info* infos) {
  if (!c) return SC_EINVAL;
  if (count < 0 || (count > 0 && (!graphs || !K || !opts)))
    return fail(c, SC_EINVAL, "sc_lobpcg_batch: invalid argument (null pointer or size out of range)");
  for (int q = 0; q < count; ++q) {
    int rc = check_lobpcg_args(c, graphs[q], K[q], &opts[q]);
    if (rc != SC_OK) return rc;
  }
  cudaSetDevice(c->device);
  std::vector<cudaStream_t> streams(count);
  std::vector<RunBase*> runs(count, nullptr);
  int rc = SC_OK;
  for (int q = 0; q < count && rc == SC_OK; ++q) {
    if (cudaStreamCreateWithFlags(&streams[q], cudaStreamNonBlocking) != cudaSuccess) {
      rc = fail(c, SC_ECUDA, "stream creation failed");
      streams[q] = nullptr;
      break;
    }
    runs[q] = make_run(c, graphs[q], K[q], &opts[q], streams[q]);
    rc = runs[q]->setup(nullptr, 0);
  }
  // the first pass (no direction block yet) run by run; then lockstep when the runs allow it
  for (int q = 0; q < count && rc == SC_OK; ++q)
    if (!runs[q]->finished()) rc = runs[q]->pass();
  bool lock = rc == SC_OK && Lockstep::eligible(runs) && !runs[0]->finished();
  Lockstep ls;
  ls.c = c;
  if (lock) {
    for (RunBase* b : runs) ls.r.push_back(dynamic_cast<LobRun<float>*>(b));
    rc = ls.build();
    while (rc == SC_OK && !runs[0]->finished()) {
      rc = ls.pass();
      g_lockstep_passes.fetch_add(1, std::memory_order_relaxed);
    }
    if (ls.bs) cudaStreamSynchronize(ls.bs);
  }
  bool any = true;
  while (rc == SC_OK && any) {
    any = false;
    for (int q = 0; q < count && rc == SC_OK; ++q)
      if (!runs[q]->finished()) {
        rc = runs[q]->pass();
        any = true;
      }
  }
  for (int q = 0; q < count && rc == SC_OK; ++q) rc = runs[q]->finish(nullptr, infos ? &infos[q] : nullptr);
  for (int q = 0; q < count; ++q) {
    delete runs[q];
    if (streams[q]) cudaStreamDestroy(streams[q]);
  }
  return rc;
}

int sc_embed_rows(sc_ctx* c, const float* X, int32_t n, int K, float* E, int on_device) {
  if (!c) return SC_EINVAL;
  if (!X || !E || n < 1 || K < 1)
    return fail(c, SC_EINVAL, "sc_embed_rows: invalid argument (null pointer or size out of range)");
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
  if (!c) return SC_EINVAL;
  if (!E || !labels_out || n < 1 || d < 1 || k < 1 || k > n || iters < 0)
    return fail(c, SC_EINVAL, "sc_kmeans: invalid argument (null pointer or size out of range)");
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

int sc_eigengap(const double* lam, int l, double ratio, double floor, int* k_out) {
  if (!k_out || (l > 0 && !lam) || l < 0 || l > SC_MAX_K || !(ratio > 1.0) ||
      !(floor >= 0.0) || !std::isfinite(floor) || !std::isfinite(ratio))
    return SC_EINVAL;
  double v[SC_MAX_K];
  for (int i = 0; i < l; ++i) {
    if (!std::isfinite(lam[i])) return SC_EINVAL;
    v[i] = lam[i];
  }
  std::sort(v, v + l);
  *k_out = 0;
  if (l < 3) return SC_OK;
  auto inc = [&](int i) {
    const double d = v[i + 1] - v[i];
    return d > floor ? d : 0.0;
  };
  double prev = inc(0);
  for (int i = 1; i + 1 < l; ++i) {
    const double d = inc(i);
    if (d > 0.0 && d > ratio * prev) {
      *k_out = i + 1;
      return SC_OK;
    }
    prev = std::max(prev, d);
  }
  return SC_OK;
}

int sc_cpqr_assign(sc_ctx* c, const float* Y, int32_t n, int K, int on_device,
                   int32_t* labels_out, int32_t* pivots_out) {
  if (!c) return SC_EINVAL;
  if (!Y || !labels_out || n < 1 || K < 1 || K > n || K > SC_MAX_K)
    return fail(c, SC_EINVAL, "sc_cpqr_assign: invalid argument (null pointer or size out of range)");
  cudaSetDevice(c->device);
  Alloc al = alloc_of(c);
  const float* dY = Y;
  float* tY = nullptr;
  int* dl = al.get<int>((size_t)n);
  int* dp = al.get<int>((size_t)K);
  if (!dl || !dp) {
    al.put(dl);
    al.put(dp);
    return fail(c, SC_ENOMEM, "sc_cpqr_assign");
  }
  if (!on_device) {
    tY = al.get<float>((size_t)n * K);
    if (!tY) {
      al.put(dl);
      al.put(dp);
      return fail(c, SC_ENOMEM, "sc_cpqr_assign");
    }
    CK(cudaMemcpyAsync(tY, Y, sizeof(float) * (size_t)n * K, cudaMemcpyHostToDevice, c->stream), "cpqr");
    dY = tY;
  }
  int rc = SC_OK;
  cudaError_t e = cpqr_assign(c->stream, al, n, K, dY, K, dp, dl, c->d_status);
  if (e != cudaSuccess) rc = fail(c, SC_ECUDA, std::string("cpqr: ") + cudaGetErrorString(e));
  if (rc == SC_OK) {
    CK(cudaMemcpyAsync(labels_out, dl, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, c->stream), "cpqr");
    if (pivots_out)
      CK(cudaMemcpyAsync(pivots_out, dp, sizeof(int) * (size_t)K, cudaMemcpyDeviceToHost, c->stream), "cpqr");
    CK(cudaStreamSynchronize(c->stream), "cpqr");
    int hs = 0;
    rc = read_status(c, &hs);
    if (rc == SC_OK && (hs & ST_NONFINITE)) rc = fail(c, SC_EBREAKDOWN, "cpqr: non-finite polar factor");
  } else {
    cudaStreamSynchronize(c->stream);
  }
  al.put(tY);
  al.put(dl);
  al.put(dp);
  return rc;
}

int sc_partition(sc_ctx* c, sc_graph* g, int K, int k, const sc_lobpcg_opts* o, int kmeans_iters,
                 int32_t* labels_out, sc_eig_info* info) {
  if (!c) return SC_EINVAL;
  if (!g || !o || !labels_out || k < 1 || k > g->csr.n)
    return fail(c, SC_EINVAL, "sc_partition: invalid argument (null pointer or size out of range)");
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
                 dC, b, false, c->d_status, c->probe_spins()), "gram_tc");
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
static int update_t(sc_ctx* c, int prec, int64_t n, int a, int b, const T* A, int64_t lda,
                    const T* W, const T* Cin, int64_t ldc, double beta, T* out, int64_t ldo,
                    int on_device) {
  Alloc al = alloc_of(c);
  const int V = 16 / sizeof(T);
  const int ap = (a + V - 1) / V * V, bp = (b + V - 1) / V * V;
  T* dA = al.get<T>((size_t)n * ap + 1);
  T* dW = al.get<T>((size_t)a * b + 1);
  T* dC = Cin ? al.get<T>((size_t)n * bp + 1) : nullptr;
  T* dO = al.get<T>((size_t)n * bp + 1);
  int rc = SC_OK;
  if (!dA || !dW || !dO || (Cin && !dC)) {
    rc = fail(c, SC_ENOMEM, "sc_tall_update: out of device memory or HBM budget");
  } else {
    cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (n > 0) {
      e = cudaMemcpy2DAsync(dA, sizeof(T) * ap, A, sizeof(T) * lda, sizeof(T) * a, n, kin, c->stream);
      if (e == cudaSuccess && Cin)
        e = cudaMemcpy2DAsync(dC, sizeof(T) * bp, Cin, sizeof(T) * ldc, sizeof(T) * b, n, kin, c->stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dW, W, sizeof(T) * (size_t)a * b, kin, c->stream);
    if (e == cudaSuccess)
      e = tall_gemm<T>(c->stream, n, cat<T>(dA, ap, a), dW, b, b, dO, bp, dC, bp, (T)beta,
                       c->d_status, prec == SC_PREC_MIXED);
    if (e == cudaSuccess && n > 0)
      e = cudaMemcpy2DAsync(out, sizeof(T) * ldo, dO, sizeof(T) * bp, sizeof(T) * b, n, kout, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "sc_tall_update");
  }
  al.put(dA);
  al.put(dW);
  al.put(dC);
  al.put(dO);
  cudaStreamSynchronize(c->stream);
  if (rc != SC_OK) return rc;
  int hs = 0;
  rc = read_status(c, &hs);
  if (rc != SC_OK) return rc;
  if (hs & 32) return fail(c, SC_ETIMEOUT, "sc_tall_update: a bounded device wait gave up");
  return SC_OK;
}

int sc_tall_update(sc_ctx* c, int prec, int64_t n, int a, int b, const void* A, int64_t lda,
                   const void* W, const void* Cin, int64_t ldc, double beta, void* out,
                   int64_t ldo, int on_device) {
  if (!c) return SC_EINVAL;
  if (n < 0 || a < 1 || b < 1 || !A || !W || !out || lda < a || ldo < b || (Cin && ldc < b) ||
      prec < SC_PREC_MIXED || prec > SC_PREC_MIXED_DD)
    return fail(c, SC_EINVAL, "sc_tall_update: invalid argument");
  cudaSetDevice(c->device);
  if (prec == SC_PREC_FP64)
    return update_t<double>(c, prec, n, a, b, (const double*)A, lda, (const double*)W,
                            (const double*)Cin, ldc, beta, (double*)out, ldo, on_device);
  return update_t<float>(c, prec, n, a, b, (const float*)A, lda, (const float*)W,
                         (const float*)Cin, ldc, beta, (float*)out, ldo, on_device);
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
  if (!c) return SC_EINVAL;
  if (!G || !theta || !Y || m < 1 || K < 1 || K > m || m > 3 * SC_MAX_K)
    return fail(c, SC_EINVAL, "sc_rr_solve: invalid argument (null pointer or size out of range)");
  cudaSetDevice(c->device);
  if (prec == SC_PREC_FP64) return rr_t<double>(c, m, K, G, theta, Y);
  return rr_t<float>(c, m, K, G, theta, Y);
}

int sc_partition_batch(sc_ctx* c, int count, sc_graph* const* graphs, const int* K, const int* k,
                       const sc_lobpcg_opts* opts, int kmeans_iters, int32_t* const* labels_out,
                       sc_eig_info* infos) {
  if (!c || count < 0 || (count > 0 && (!graphs || !K || !k || !opts || !labels_out)))
    return SC_EINVAL;
  int rc = sc_lobpcg_batch(c, count, graphs, K, opts, infos);
  if (rc != SC_OK) return rc;
  for (int q = 0; q < count && rc == SC_OK; ++q) {
    sc_graph* g = graphs[q];
    Alloc al = alloc_of(c);
    const int n = g->csr.n;
    float* E = al.get<float>((size_t)n * K[q]);
    if (!E) return fail(c, SC_ENOMEM, "sc_partition_batch");
    CK(rownorm<float>(c->stream, n, K[q], g->X, K[q], E, K[q]), "embed");
    rc = kmeans_dev(c, E, n, K[q], k[q], kmeans_iters, opts[q].seed, nullptr, labels_out[q],
                    nullptr, nullptr, nullptr, nullptr);
    cudaStreamSynchronize(c->stream);
    al.put(E);
  }
  return rc;
}

// ---- serving loop ---------------------------------------------------------------------
// A worker thread owns the context.  Requests wait in a bounded queue; the worker admits
// them while slots and the HBM budget allow (continuous batching at LOBPCG-pass granularity:
// a request that arrives while others run joins at the next pass boundary), advances every
// active solve by one pass per round on its own stream, and finishes each with the row
// embedding and k-means.  Graphs stay resident by id, so a streaming delta warm-starts from
// the block its graph kept.

namespace {
using Clock = std::chrono::steady_clock;

struct SrvReq {
  uint64_t ticket;
  sc_request r;
  std::vector<int32_t> src, dst;
  Clock::time_point t0;
};

struct SrvResult {
  int status = SC_EAGAIN;
  std::vector<int32_t> labels;
  sc_eig_info info{};
  double latency_ms = 0.0;
};

struct SrvSlot {
  SrvReq req;
  sc_graph* g = nullptr;
  RunBase* run = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;  // recorded after the last pass was issued
  size_t est = 0;
};

size_t footprint(const sc_request& r) {
  const size_t kp = (size_t)(r.K + 3) / 4 * 4;
  const size_t el = r.prec == SC_PREC_FP64 ? 8 : 4;
  return (size_t)r.n * kp * 21 * el + (size_t)r.m * 48 + (size_t)r.n * 64 + (1u << 20);
}
}  // namespace

struct sc_server {
  sc_ctx* c = nullptr;
  int max_slots = 1, queue_cap = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<SrvReq> queue;
  std::unordered_map<uint64_t, SrvResult> results;
  std::unordered_map<int, sc_graph*> graphs;
  std::vector<SrvSlot> active;
  uint64_t next = 1, completed = 0;
  size_t reserved = 0;
  bool stop = false;
  std::thread worker;
};

static void srv_complete(sc_server* s, SrvSlot& sl, int status) {
  SrvResult res;
  res.status = status;
  if (status == SC_OK && sl.run) {
    // outputs (and the resident block the embedding reads) first; a tolerance that was not
    // met is reported but still yields labels
    status = sl.run->finish(nullptr, &res.info);
    res.status = status;
  }
  if (status == SC_OK || status == SC_ENOTCONV) {
    sc_ctx* c = s->c;
    const int n = sl.g->csr.n, K = sl.req.r.K;
    Alloc al = alloc_of(c);
    float* E = al.get<float>((size_t)n * K);
    if (!E) {
      res.status = SC_ENOMEM;
    } else {
      res.labels.resize(n);
      cudaError_t e = rownorm<float>(c->stream, n, K, sl.g->X, K, E, K);
      int krc = e == cudaSuccess ? kmeans_dev(c, E, n, K, sl.req.r.k, sl.req.r.kmeans_iters,
                                              sl.req.r.seed, nullptr, res.labels.data(), nullptr,
                                              nullptr, nullptr, nullptr)
                                 : SC_ECUDA;
      if (krc != SC_OK) res.status = krc;
      cudaStreamSynchronize(c->stream);
      al.put(E);
    }
  }
  res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - sl.req.t0).count();
  delete sl.run;
  sl.run = nullptr;
  if (sl.done) cudaEventDestroy(sl.done);
  sl.done = nullptr;
  if (sl.st) cudaStreamDestroy(sl.st);
  sl.st = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  s->reserved -= sl.est;
  s->results[sl.req.ticket] = std::move(res);
  s->completed++;
  s->cv_done.notify_all();
}

// Build or update the slot's graph and set up its solve; returns an sc_status.
static int srv_start(sc_server* s, SrvSlot& sl) {
  sc_ctx* c = s->c;
  const sc_request& r = sl.req.r;
  int rc = SC_OK;
  if (r.kind == SC_REQ_COLD) {
    auto it = s->graphs.find(r.graph_id);
    if (it != s->graphs.end()) {
      sc_graph_destroy(it->second);
      s->graphs.erase(it);
    }
    sc_graph* g = nullptr;
    rc = sc_build_laplacian(c, r.n, (int64_t)sl.req.src.size(), sl.req.src.data(), sl.req.dst.data(),
                            nullptr, SC_SYM_LOGICAL, 0, &g);
    if (rc != SC_OK) return rc;
    s->graphs[r.graph_id] = g;
    sl.g = g;
  } else {
    auto it = s->graphs.find(r.graph_id);
    if (it == s->graphs.end()) return fail(c, SC_EINVAL, "delta for an unknown graph id");
    sl.g = it->second;
    rc = sc_stream_update(c, sl.g, r.n, (int64_t)sl.req.src.size(), sl.req.src.data(),
                          sl.req.dst.data(), nullptr, 0);
    if (rc != SC_OK) return rc;
  }
  sc_lobpcg_opts o{r.iters, r.tol_abs, 0.0, r.prec, r.seed, r.kind == SC_REQ_COLD ? 1 : 0,
                   SC_PRECOND_NONE};
  rc = check_lobpcg_args(c, sl.g, r.K, &o);
  if (rc != SC_OK) return rc;
  if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess)
    return fail(c, SC_ECUDA, "stream creation failed");
  sl.run = make_run(c, sl.g, r.K, &o, sl.st);
  return sl.run->setup(nullptr, 0);
}

static void srv_loop(sc_server* s) {
  cudaSetDevice(s->c->device);
  for (;;) {
    std::vector<SrvReq> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->active.empty() && s->queue.empty())
        s->cv_work.wait_for(lk, std::chrono::milliseconds(20),
                            [&] { return s->stop || !s->queue.empty(); });
      if (s->stop && s->queue.empty() && s->active.empty()) break;
      const size_t budget = s->c->budget;
      // Requests on one graph run one at a time, in arrival order: a graph that is being
      // solved (or has an earlier request still queued) must not be rebuilt or merged into
      // while kernels of the running solve read its CSR and resident block.
      std::unordered_set<int> busy;
      for (const SrvSlot& sl : s->active) busy.insert(sl.req.r.graph_id);
      for (auto it = s->queue.begin(); it != s->queue.end() &&
                                       (int)(s->active.size() + admit.size()) < s->max_slots;) {
        const int gid = it->r.graph_id;
        if (busy.count(gid)) {
          ++it;  // stays queued, and keeps later requests on the same graph behind it
          continue;
        }
        busy.insert(gid);
        size_t est = footprint(it->r);
        if (budget && est > budget) {  // can never fit: reject
          SrvResult res;
          res.status = SC_ENOMEM;
          s->results[it->ticket] = std::move(res);
          s->completed++;
          it = s->queue.erase(it);
          s->cv_done.notify_all();
          continue;
        }
        if (budget && s->c->in_use + s->reserved + est > budget && !(s->active.empty() && admit.empty()))
          break;  // wait for memory to free up
        s->reserved += est;
        admit.push_back(std::move(*it));
        admit.back().r.src = nullptr;
        it = s->queue.erase(it);
      }
    }
    for (auto& rq : admit) {
      SrvSlot sl;
      sl.est = footprint(rq.r);
      sl.req = std::move(rq);
      int rc = srv_start(s, sl);
      if (rc != SC_OK) {
        srv_complete(s, sl, rc);
        continue;
      }
      s->active.push_back(std::move(sl));
    }
    // Issue work: a fixed-pass solve (no stopping tolerance: the host decides nothing between
    // passes) has all of its passes queued on its stream at once, so the device always holds
    // work of every admitted request; a solve with a tolerance advances one pass per round.
    // An event after the last pass marks the solve's device work.
    for (auto& sl : s->active) {
      if (!sl.run || sl.done) continue;
      const bool fixed = sl.req.r.tol_abs <= 0;
      int rc = SC_OK;
      do {
        rc = sl.run->pass();
      } while (rc == SC_OK && fixed && !sl.run->finished());
      if (rc == SC_OK && sl.run->finished()) {
        if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(sl.done, sl.st) != cudaSuccess)
          rc = fail(s->c, SC_ECUDA, "event");
      }
      if (rc != SC_OK) {
        delete sl.run;
        sl.run = nullptr;
        srv_complete(s, sl, rc);
      }
    }
    // retire the solves whose device work is done (outputs, embedding and k-means), in
    // admission order; the others keep running on the device meanwhile
    std::vector<SrvSlot> keep;
    bool progressed = !admit.empty();
    for (auto& sl : s->active) {
      if (!sl.run) {  // failed and completed above
        progressed = true;
        continue;
      }
      const cudaError_t q = sl.done ? cudaEventQuery(sl.done) : cudaErrorNotReady;
      if (q == cudaSuccess) {
        srv_complete(s, sl, SC_OK);
        progressed = true;
      } else if (q != cudaErrorNotReady) {
        cudaGetLastError();
        srv_complete(s, sl, SC_ECUDA);
        progressed = true;
      } else {
        keep.push_back(std::move(sl));
      }
    }
    s->active.swap(keep);
    if (!progressed && !s->active.empty()) {
      // nothing finished and nothing admitted: wait briefly for an arrival or the device
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::microseconds(200),
                          [&] { return s->stop || !s->queue.empty(); });
    }
  }
}

int sc_server_create(sc_ctx* c, int max_slots, int queue_cap, sc_server** out) {
  if (!c || !out || max_slots < 1 || queue_cap < 1) return SC_EINVAL;
  sc_server* s = new sc_server();
  s->c = c;
  s->max_slots = max_slots;
  s->queue_cap = queue_cap;
  s->worker = std::thread(srv_loop, s);
  *out = s;
  return SC_OK;
}

int sc_server_submit(sc_server* s, const sc_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket || r->n < 1 || r->m < 0 || (r->m > 0 && (!r->src || !r->dst)) ||
      (r->kind != SC_REQ_COLD && r->kind != SC_REQ_DELTA) || r->K < 1 || r->k < 1)
    return SC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int)s->queue.size() >= s->queue_cap) return SC_EAGAIN;
  SrvReq q;
  q.ticket = s->next++;
  q.r = *r;
  q.src.assign(r->src, r->src + r->m);
  q.dst.assign(r->dst, r->dst + r->m);
  q.t0 = Clock::now();
  s->results[q.ticket] = SrvResult{};
  *ticket = q.ticket;
  s->queue.push_back(std::move(q));
  s->cv_work.notify_one();
  return SC_OK;
}

static int srv_take(sc_server* s, uint64_t ticket, int32_t* labels_out, int32_t n_cap,
                    sc_eig_info* info, double* latency_ms) {
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return SC_EINVAL;
  if (it->second.status == SC_EAGAIN) return SC_EAGAIN;
  SrvResult res = std::move(it->second);
  s->results.erase(it);
  if (res.status == SC_OK && labels_out) {
    if ((int32_t)res.labels.size() > n_cap) return SC_EINVAL;
    std::memcpy(labels_out, res.labels.data(), sizeof(int32_t) * res.labels.size());
  }
  if (info) *info = res.info;
  if (latency_ms) *latency_ms = res.latency_ms;
  return res.status;
}

int sc_server_poll(sc_server* s, uint64_t ticket, int32_t* labels_out, int32_t n_cap,
                   sc_eig_info* info, double* latency_ms) {
  if (!s) return SC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  return srv_take(s, ticket, labels_out, n_cap, info, latency_ms);
}

int sc_server_wait(sc_server* s, uint64_t ticket, int timeout_ms, int32_t* labels_out,
                   int32_t n_cap, sc_eig_info* info, double* latency_ms) {
  if (!s) return SC_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] {
    auto it = s->results.find(ticket);
    return it == s->results.end() || it->second.status != SC_EAGAIN;
  };
  if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return SC_ETIMEOUT;
  return srv_take(s, ticket, labels_out, n_cap, info, latency_ms);
}

int sc_server_stats(sc_server* s, int* active, int* queued, uint64_t* completed) {
  if (!s) return SC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (active) *active = (int)s->active.size();
  if (queued) *queued = (int)s->queue.size();
  if (completed) *completed = s->completed;
  return SC_OK;
}

void sc_server_destroy(sc_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->graphs) sc_graph_destroy(kv.second);
  delete s;
}
