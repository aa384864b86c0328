// Shared declarations of the GB300 spectral-clustering library (sm_103a).
#pragma once
#include <functional>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

namespace sc {

// Tile (i, j) of tile number t of a Gram over an na x nb tile grid, numbered row by row over
// all tiles, or (sym, na == nb) over the tiles with i <= j only.
__device__ __forceinline__ int2 tile_coord(int t, int nb, int sym) {
  if (!sym) return make_int2(t / nb, t % nb);
  int i = 0;
  while (t >= nb - i) {
    t -= nb - i;
    ++i;
  }
  return make_int2(i, i + t);
}


// ---- device status word bits (written by kernels, read back by the host) ----------------
enum : int {
  ST_EDGE_RANGE = 1,   // an edge endpoint outside [0, n)
  ST_NNZ_OVERFLOW = 2, // stored nonzeros would exceed 2^31 - 1
  ST_CHOL_FAIL = 4,    // Cholesky pivot below tolerance
  ST_ROW_TOO_LONG = 8, // internal: a row exceeded the sort capacity
  ST_NONFINITE = 16,   // NaN/Inf met in a small dense solve
};

// Up to three column blocks viewed as one n x (c0 + c1 + c2) matrix (row-major blocks).
template <typename T>
struct Cat3 {
  const T* p[3];
  long long ld[3];
  int c[3];
  int nblk;
  __host__ __device__ int cols() const {
    int s = 0;
    for (int i = 0; i < nblk; ++i) s += c[i];
    return s;
  }
};

template <typename T>
inline Cat3<T> cat(const T* p0, long long ld0, int c0) {
  Cat3<T> r{};
  r.p[0] = p0; r.ld[0] = ld0; r.c[0] = c0; r.nblk = 1;
  return r;
}
template <typename T>
inline Cat3<T> cat(const T* p0, long long ld0, int c0, const T* p1, long long ld1, int c1) {
  Cat3<T> r = cat(p0, ld0, c0);
  r.p[1] = p1; r.ld[1] = ld1; r.c[1] = c1; r.nblk = 2;
  return r;
}
template <typename T>
inline Cat3<T> cat(const T* p0, long long ld0, int c0, const T* p1, long long ld1, int c1,
                   const T* p2, long long ld2, int c2) {
  Cat3<T> r = cat(p0, ld0, c0, p1, ld1, c1);
  r.p[2] = p2; r.ld[2] = ld2; r.c[2] = c2; r.nblk = 3;
  return r;
}

// Launch accounting: every kernel launch of the library goes through note_launch().
void note_launch();
void note_launches(uint64_t k);  // k launches replayed from a CUDA graph
uint64_t launches_total();

// Per-kernel timing with CUDA events on the launching stream.  A ProfScope placed around a
// launch records an event pair when profiling is on for that kernel name.
void prof_begin(cudaStream_t st, const char* name);
void prof_end(cudaStream_t st, const char* name);
bool prof_active();  // an event-pair profile is being taken (no graph replay meanwhile)
struct ProfScope {
  cudaStream_t st;
  const char* name;
  ProfScope(cudaStream_t s, const char* n) : st(s), name(n) { prof_begin(st, name); }
  ~ProfScope() { prof_end(st, name); }
};

// Seeded N(0,1) start block (SplitMix64 counter stream `key`, Box-Muller on consecutive
// uniform pairs, rounded to float): element e of the n x K row-major block -> X[e/K][e%K].
template <typename T>
cudaError_t gauss_block(cudaStream_t st, long long n, int K, unsigned long long key, T* X,
                        long long ldx);

// ---- kernel entry points (host wrappers, all asynchronous on `st`) -----------------------

// CSR build (Sec. II.A): edge list -> symmetrized CSR.  Returns cudaError_t of the launches;
// sizes that depend on device results are returned through the host pointers after an
// internal stream synchronisation.
struct CsrDev {
  int n = 0;
  long long nnz = 0;
  int* row_ptr = nullptr;  // n+1
  int* col_idx = nullptr;  // nnz
  float* val = nullptr;    // nnz (algebraic) or null (logical: all ones)
  float* degf = nullptr;   // n
  double* degd = nullptr;  // n
  double deg_max = 0;
};

// Allocation callbacks used by multi-phase host routines.
struct Alloc {
  void* (*alloc)(void* self, size_t bytes);
  void (*free)(void* self, void* p);
  void* self;
  template <typename T>
  T* get(size_t count) { return (T*)alloc(self, count * sizeof(T)); }
  void put(void* p) { if (p) free(self, p); }
};

cudaError_t build_csr(cudaStream_t st, Alloc& al, int n, long long m, const int* d_src,
                      const int* d_dst, const float* d_w, int algebraic, int* d_status,
                      CsrDev* out, int* host_status);
cudaError_t merge_csr(cudaStream_t st, Alloc& al, const CsrDev& a, const CsrDev& b,
                      int algebraic, int* d_status, CsrDev* out, int* host_status);

// SpMM: Y = D V - W V (n x k block, row stride ldv/ldy, ld multiple of 16 bytes).  shape: a
// kernel shape index from spmm_shapes (lanes per row x chunks per lane), -1 = the default.
template <typename T>
cudaError_t spmm_lap(cudaStream_t st, const CsrDev& g, const T* V, long long ldv, T* Y,
                     long long ldy, int k, int shape = -1);
// Householder tridiagonalization of an m x m FP64 matrix on a cluster of 8 CTAs
// (k_tridiag_cl.cu), in FP32 (m <= 512) or FP64 (m <= 256): d, e, beta and the scaled reflector
// rows (row stride lda) of Ag.
cudaError_t tridiag_cluster(cudaStream_t st, int m, int K, const double* G, int ldg, float* Ag,
                            int lda, float* d, float* e, float* beta, const int* pflag, int mP);
cudaError_t tridiag_cluster(cudaStream_t st, int m, int K, const double* G, int ldg, double* Ag,
                            int lda, double* d, double* e, double* beta, const int* pflag, int mP);
// Kernel shapes valid for nvec 16-byte column chunks (at most 13); out[0] is the default.
int spmm_shapes(int nvec, int* out);

// Project autotuner (tune.cu): the fastest variant per key, measured on first use (each
// variant issued by run(v) on stream st), cached for the process and persisted to
// SC_AUTOTUNE_FILE; SC_TUNE_<KERNEL> forces a variant, SC_AUTOTUNE=0 returns `fallback` for
// keys not yet chosen.
// SC_TUNE_<KERNEL>=<variant> (kernel name upper-cased), or -1 when unset.
int tune_override(const char* kernel);
int tune_pick(const std::string& key, const char* kernel, cudaStream_t st, int nvar,
              int fallback, const std::function<cudaError_t(int)>& run);
int tune_lookup(const std::string& key);
int tune_table_size();

// Gram: C (a x b, FP64 row-major, ldc) = A' B over n rows.  `sym` = A and B are the same
// matrix: only the upper tile triangle is computed and mirrored.  Workspace from `al`.
template <typename T>
cudaError_t gram(cudaStream_t st, Alloc& al, long long n, const Cat3<T>& A, const Cat3<T>& B,
                 double* C, int ldc, bool sym, int use_tc);

// Tensor-core Gram (3-term split TF32 on tcgen05): C = A' B for FP32 blocks A = columns
// [0, a) of a row-major block with stride lda (16-byte aligned, lda % 4 == 0), B alike.
// segA/segB: (start, count) pairs listing the columns that appear in the compact output C.
cudaError_t gram_tc(cudaStream_t st, Alloc& al, long long n, const float* A, long long lda,
                    int a, const int* segA, int nsegA, const float* B, long long ldb, int b,
                    const int* segB, int nsegB, double* C, int ldc, bool sym, int* d_status,
                    long long probe_spins = 0);

// Tall GEMM: out (n x b, ldo) = beta * Cin + A (n x a) W (a x b, row-major ldw, type T).
// use_tc (FP32 only): run on tcgen05 tensor cores as 3-term split TF32 products when the shape
// fits (k_tall_tc.cu), otherwise on CUDA cores.
template <typename T>
cudaError_t tall_gemm(cudaStream_t st, long long n, const Cat3<T>& A, const T* W, int ldw,
                      int b, T* out, long long ldo, const T* Cin, long long ldc, T beta,
                      int* d_status = nullptr, bool use_tc = false);
// One output segment of a tall update: columns go to out (stride ldo), plus beta * Cin,
// computed with the W block (stride ldw) whose rows start at row wskip of the concatenated A
// (the rows before it are zero for this segment).
template <typename T>
struct TallSeg {
  T* out;
  long long ldo;
  const T* Cin;
  long long ldc;
  const T* W;
  int ldw;
  int wskip;
  int b;
};
// [out_0 | out_1] = beta [Cin_0 | Cin_1] + A [W_0 | W_1] in one pass over A
template <typename T>
cudaError_t tall_gemm2(cudaStream_t st, long long n, const Cat3<T>& A, const TallSeg<T>& s0,
                       const TallSeg<T>& s1, T beta, int* d_status = nullptr,
                       bool use_tc = false);
cudaError_t tall_gemm_tc(cudaStream_t st, long long n, const Cat3<float>& A,
                         const TallSeg<float>& s0, const TallSeg<float>& s1, float beta,
                         int* d_status);


// Residual: R = LX - X diag(theta); rho2[j] = sum_i R_ij^2 (FP64).  With deg non-null the
// block stored is D^-1 R (rows with d_i = 0 unscaled: the Jacobi preconditioner), while rho2
// stays the norms of R.  Workspace from `al`.
template <typename T>
cudaError_t residual(cudaStream_t st, Alloc& al, long long n, int K, const T* X, const T* LX,
                     long long ld, const double* theta, T* R, double* rho2,
                     const T* deg = nullptr);

// Gather / scatter of a column subset (cols[j] -> j).
template <typename T>
cudaError_t gather_cols(cudaStream_t st, long long n, const T* src, long long lds, T* dst,
                        long long ldd, const int* cols, int kc);

// dst (rows x cols, T) = scale * src (FP64).
template <typename T>
cudaError_t cast_mat(cudaStream_t st, int rows, int cols, const double* src, int lds, T* dst,
                     int ldd, double scale);

// dst (rows x cols, To, row stride ldd) = src (Ti, row stride lds), element by element
// (FP32 <-> FP64).
template <typename Ti, typename To>
cudaError_t convert_mat(cudaStream_t st, long long rows, int cols, const Ti* src, long long lds,
                        To* dst, long long ldd);

// Row normalization E_i = X_i / ||X_i||.
template <typename T>
cudaError_t rownorm(cudaStream_t st, long long n, int K, const T* X, long long ldx, float* E,
                    long long lde);

// Small dense: Tm = D C^-T for the scaled Cholesky D G D = C C' of G (ka x ka FP64).
// Tm is ka x ka upper triangular (row-major, T).  Status bit ST_CHOL_FAIL on breakdown.
// With pflag != null and a breakdown at a column >= keep, the transform of the leading keep
// columns is returned (zeros elsewhere) and *pflag is cleared instead of reporting failure.
// A column whose norm is at or below its floor (rfloor for columns < keep, pfloor for the
// rest) counts as zero.  With ndrop > 0, a breakdown at a column < ndrop, or a zero column
// anywhere, drops that column alone (zero column of Tm) and adds one to *ndropped (if given).
template <typename T>
cudaError_t chol_inv(cudaStream_t st, Alloc& al, int ka, const double* G, int ldg, T* Tm,
                     int* d_status, double pivot_tol, int* fail_col = nullptr, int keep = 0,
                     int* pflag = nullptr, int ndrop = 0, int* ndropped = nullptr,
                     double rfloor = 0.0, double pfloor = 0.0);

// Rayleigh-Ritz in an orthonormal basis: K smallest eigenpairs of symmetric m x m G (FP64).
// theta[K] FP64 (device), Y (m x K, T, row-major).  Arithmetic in T.
// pflag (optional, device): 0 = the trailing mP basis columns were dropped; the solve then
// uses the leading m - mP block, zeroes the rest of Y, bumps *nfallback and re-arms *pflag.
// A basis column i >= K with G_ii exactly 0 (a column the Cholesky-QR dropped: its row of G
// is zero) gets a diagonal above the Gershgorin bound of G, so its spurious eigenvalue is
// never among the K smallest.
template <typename T>
cudaError_t rr_eig(cudaStream_t st, Alloc& al, int m, int K, const double* G, int ldg,
                   double* theta, T* Y, int* d_status, int* pflag = nullptr, int mP = 0,
                   int* nfallback = nullptr);

// Cluster assignment by QR with column pivoting (FP64): piv (K, device) = the pivot rows of
// Y (n x K FP32, stride ldy), labels (n, device) = argmax_j |(Y Q)_ij| with Q the polar factor
// of Y'[:, piv].
cudaError_t cpqr_assign(cudaStream_t st, Alloc& al, long long n, int K, const float* Y,
                        long long ldy, int* piv, int* labels, int* d_status);

// k-means.
cudaError_t kmeanspp(cudaStream_t st, Alloc& al, int n, int d, int k, const float* E,
                     long long lde, const double* u_host, int* seeds_dev);
cudaError_t lloyd(cudaStream_t st, Alloc& al, int n, int d, int k, const float* E,
                  long long lde, const int* seeds_dev, int iters, int* labels_dev,
                  double* cent_dev, int* iters_run, double* inertia);

// k-means assignment on tensor cores (3-term split TF32 distances ||c||^2 - 2 e.c; a row whose
// margin is below 4 tie is re-decided with FP64 distances to the centroids within 4 tie of its
// best, tie being the CUDA-core kernel's margin): labels of the n x d rows E against the k x d
// centroids,
// k <= 256; *changes += rows whose label changed (all rows when first).  Returns
// cudaErrorNotSupported when the shape does not fit (the caller uses the CUDA-core kernel).
cudaError_t assign_tc(cudaStream_t st, long long n, int d, int k, const float* E, long long lde,
                      const float* C32, const float* cn, const double* C64, int* labels,
                      int* changes, int first, float tie, const int* ctl, int* d_status);

// ---- lockstep batches (sc_lobpcg_batch): one launch per kernel shape for all runs ---------
// A descriptor holds one run's arguments of the single-run call; a batched launch runs one CTA
// (one cluster for the cluster tridiagonalization, a share of the rows for the SpMM) per
// descriptor with the single-run kernel's arithmetic, so every run's results are bitwise its
// single-run results.  Descriptor tables live in device memory, written once per batch.
struct CholDesc {
  int ka, ldg, keep, ndrop;
  const double* G;
  float* Tm;
  float* Wg;  // ka x ka scratch when the factorization does not fit in shared memory
  int *status, *fail_col, *pflag, *ndropped;
  double pivot_tol, rfloor, pfloor;
};
struct RrDesc {
  int m, K, ldg, mP;
  const double* G;
  double* theta;
  float* Y;
  int *status, *pflag, *nfallback;
  float* Ag;   // global-memory working set (rr_batch_scratch floats) or null
  float* tri;  // 3 m floats (d, e, beta of the cluster tridiagonalization) or null
  float* lamx;  // K floats: the eigenvalues, when tri is set (found one CTA per eigenvalue)
  int* mx;      // the solved size, when tri is set (for the column back-transformation)
};
struct SpmmDesc {
  long long row0;  // first row of this graph in the batch's concatenated row range
  int n, nvec;     // rows; 16-byte column chunks per row
  const int *rp, *ci;
  const float *val, *deg, *V;
  float* Y;
  long long ldv, ldy;
};
// A run of consecutive descriptors launched together: kind (the kernel shape), its first
// descriptor and count, the template parameter and the dynamic shared memory it needs.
struct BatchGroup {
  int kind, first, count, param;
  size_t smem;
  int aux;  // the group's largest K (Rayleigh-Ritz cluster group)
};
// Orders the descriptors by kernel shape and returns the groups; entries whose shape has no
// batched form are left out of every group (their indices in *single) and run one by one.
void chol_batch_plan(std::vector<CholDesc>& d, std::vector<BatchGroup>& groups,
                     std::vector<int>& single);
cudaError_t chol_batch_launch(cudaStream_t st, const CholDesc* dtab,
                              const std::vector<BatchGroup>& groups);
size_t chol_batch_scratch(int ka);  // floats of Wg needed (0: shared memory suffices)
void rr_batch_plan(std::vector<RrDesc>& d, std::vector<BatchGroup>& groups, std::vector<int>& single);
cudaError_t rr_batch_launch(cudaStream_t st, const RrDesc* dtab, const std::vector<BatchGroup>& groups);
size_t rr_batch_scratch(int m, int K);  // floats of Ag (0: none); tri needs 3 m when m > 160
bool rr_batch_cluster(int m);           // the group tridiagonalizes on a cluster of CTAs
cudaError_t tridiag_cluster_batch(cudaStream_t st, int count, const RrDesc* dtab, int mmax);
cudaError_t spmm_batch_launch(cudaStream_t st, const SpmmDesc* dtab, int count, long long rows,
                              int nvec_max);

}  // namespace sc
