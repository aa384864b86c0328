/*
 * sc.h -- C ABI of the GB300 spectral-clustering library (libsc_gb300.so).
 *
 * The library computes the hot path of spectral clustering as described in
 * Zhuzhunashvili & Knyazev, "Preconditioned Spectral Clustering for Stochastic Block
 * Partition Streaming Graph Challenge" (HPEC 2017):
 *   graph edge list -> symmetrized Laplacian L = D - W            (Sec. II.A, Sec. III)
 *   -> LOBPCG for the K smallest eigenpairs of L, cold or warm     (Sec. II.B, Sec. III)
 *   -> unit-normalized rows of the eigenvector block -> k-means    (Sec. II.A)
 *   -> streaming stages that warm-start from the previous block    (Sec. III, Sec. IV)
 *
 * Conventions (all entry points):
 *  - Every call returns an sc_status; nothing aborts, throws or traps.  The message of the
 *    last failure on a context is returned by sc_last_error().
 *  - Host arrays passed in are borrowed for the duration of the call and copied.  Output
 *    arrays are caller-allocated with the sizes stated per call.  Opaque objects
 *    (sc_ctx, sc_graph, sc_server) are allocated by the library and freed by the caller.
 *  - "on_device" arguments say whether the array pointers are device pointers (1) on the
 *    context's device or host pointers (0).  Device arrays must stay valid until the call
 *    returns.  All device work is issued on the context stream; calls return after that
 *    stream has finished the call's work.
 *  - Dense blocks are row-major: element (i, j) of an n x K block is at [i * K + j].
 *  - Limits: 1 <= n < 2^31, stored nonzeros < 2^31, 1 <= K <= SC_MAX_K, 3K <= n for LOBPCG.
 *  - A context is not thread-safe; use one per host thread.  A server is thread-safe.
 */
#ifndef SC_GB300_H
#define SC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SC_MAX_K 512

typedef struct sc_ctx sc_ctx;
typedef struct sc_graph sc_graph;
typedef struct sc_server sc_server;

typedef enum {
  SC_OK = 0,
  SC_EINVAL = -1,      /* bad argument (sizes, ranges, null pointers)                  */
  SC_ENOMEM = -2,      /* device allocation failed or the context HBM budget is spent  */
  SC_EBREAKDOWN = -3,  /* LOBPCG trial basis lost rank even after dropping P          */
  SC_ENOTCONV = -4,    /* tolerance requested but not reached within the iterations    */
  SC_ETIMEOUT = -5,    /* a bounded device wait gave up                                */
  SC_ECUDA = -6,       /* CUDA runtime error (message in sc_last_error)                */
  SC_EAGAIN = -7       /* server: queue full / result not ready yet                    */
} sc_status;

/* Arithmetic of the LOBPCG path.
 *  SC_PREC_MIXED:    FP32 blocks and SpMM; Gram products on tcgen05 tensor cores as
 *                    3-term split-TF32 products, FP32 accumulation in tensor memory and FP64
 *                    sums across CTAs (the Gram matrices are FP64); the small dense solves
 *                    (Cholesky-QR factors, Rayleigh-Ritz eigenproblem) in FP32.
 *  SC_PREC_FP32:     as MIXED, but Gram products on FP32 CUDA cores (FP64 cross-CTA sums).
 *  SC_PREC_FP64:     every step in FP64 (the plain form and the 1e-10 check mode).
 *  SC_PREC_MIXED_DD: as MIXED, with the small dense solves in FP64 (results cast to FP32
 *                    for the tall updates). */
typedef enum {
  SC_PREC_MIXED = 0,
  SC_PREC_FP32 = 1,
  SC_PREC_FP64 = 2,
  SC_PREC_MIXED_DD = 3
} sc_precision;

/* Symmetrization W <- W + W' (Sec. II.A): logical sum (unweighted, duplicates merged,
 * every stored weight 1) or algebraic sum (weights added, duplicates accumulate). */
typedef enum { SC_SYM_LOGICAL = 0, SC_SYM_ALGEBRAIC = 1 } sc_sym;

/* ---- context -------------------------------------------------------------------------
 * sc_ctx_create: bind to CUDA device `device`.  `cuda_stream` is a cudaStream_t to issue
 * work on (borrowed, must outlive the context) or NULL for a stream the context owns.
 * `hbm_budget` caps the bytes the context and its graphs may hold on the device (0 = no
 * cap); allocations beyond it fail with SC_ENOMEM. */
int sc_ctx_create(sc_ctx** out, int device, void* cuda_stream, size_t hbm_budget);
/* Destroy the graphs and servers created on a context before the context itself. */
void sc_ctx_destroy(sc_ctx* ctx);
const char* sc_last_error(const sc_ctx* ctx);
/* Bytes currently held on the device by this context and its graphs. */
size_t sc_ctx_bytes_in_use(const sc_ctx* ctx);
/* High-water mark of the device bytes the context held since the previous call (or since
 * creation); the mark is reset to the current use.  Not thread-safe (like the context). */
size_t sc_ctx_bytes_peak(sc_ctx* ctx);
/* Number of kernels the library has launched so far in this process (launch accounting;
 * kernels replayed from a CUDA graph count once per replay). */
uint64_t sc_ctx_kernel_launches(const sc_ctx* ctx);
/* Number of LOBPCG passes replayed from CUDA graphs so far in this process.  A solve with a
 * fixed pass count (tol_abs = tol_lock = 0) records its pass once per buffer parity, after one
 * eager pass with the direction block, and replays it: the same kernels on the same buffers,
 * so results are bitwise those of eager passes.  The environment variable SC_CUDA_GRAPHS=0
 * (read when a solve starts) keeps every pass eager. */
uint64_t sc_ctx_graph_replays(const sc_ctx* ctx);
/* Number of lockstep batch passes issued so far in this process (sc_lobpcg_batch).  A batch
 * whose runs are all SC_PREC_MIXED with the same fixed pass count (no tolerance, no constraint
 * block) runs its first pass run by run and the rest in lockstep: per pass, the two
 * Cholesky-QR transforms, the SpMM and the Rayleigh-Ritz solve of every run go out as one
 * launch per kernel shape, from descriptor tables written once per batch; from the second
 * lockstep pass on the whole batch pass is replayed from a CUDA graph.  Results are bitwise
 * those of single solves.  SC_BATCH_LOCKSTEP=0 (read per call) issues runs in turn instead. */
uint64_t sc_ctx_batch_lockstep_passes(const sc_ctx* ctx);
/* Kernel timing: between sc_profile_begin and sc_profile_end, every launch of a kernel
 * named in `kernels` (comma-separated names such as "spmm,gram,rr_eig", or "*" for all) is
 * bracketed by CUDA events on the stream it is launched on.  sc_profile_end synchronizes the
 * context stream and writes one line "name launches total_ms" per kernel into `report`
 * (NUL-terminated, truncated to len).  Process-wide: one profiling window at a time. */
int sc_profile_begin(sc_ctx* ctx, const char* kernels);
int sc_profile_end(sc_ctx* ctx, char* report, size_t len);

/* ---- fault injection for tests ---------------------------------------------------------
 * Failure handling is exercised without faulting the GPU: a test arms one injected failure
 * on a context and the later calls on that context see it, until it is disarmed
 * (SC_INJECT_NONE).  The paper has no counterpart; these hooks exist for tests.
 *  SC_INJECT_WAIT_TIMEOUT: every tensor-core Gram launch (SC_PREC_MIXED, MIXED_DD) adds, after
 *    its copies and MMAs have completed, a bounded wait on an mbarrier phase that nothing
 *    completes, giving up after `arg` (>= 1) polls.  The kernel records the time-out in the
 *    context's status word and returns normally, so the call fails with SC_ETIMEOUT and the
 *    context stays usable.
 *  SC_INJECT_P_BREAKDOWN: LOBPCG pass number `arg` (0-based, counted from the first pass that
 *    has a direction block P, i.e. arg >= 1) reports P as broken down, as the Cholesky-QR of
 *    [R P] does when P has sunk into span{X, R}; that pass's Rayleigh-Ritz step runs on
 *    [X R] only (counted in sc_eig_info.fallbacks).
 * Errors: SC_EINVAL (unknown kind, a wait limit < 1). */
enum { SC_INJECT_NONE = 0, SC_INJECT_WAIT_TIMEOUT = 1, SC_INJECT_P_BREAKDOWN = 2 };
int sc_debug_inject(sc_ctx* ctx, int kind, long long arg);

/* ---- Laplacian (Sec. II.A; Sec. III stores the directed adjacency sparse) --------------
 * sc_build_laplacian: directed edge list (src[e] -> dst[e], e < m, 0 <= src, dst < n) to
 * the symmetrized CSR of W and the degrees D of L = D - W.  Self-loops are dropped (they
 * add the same amount to D and W).  `w` = per-edge weights (NULL = all 1); with
 * SC_SYM_LOGICAL weights are ignored.  Columns within a row come out sorted ascending.
 * Out-of-range endpoints give SC_EINVAL.  The graph owns its device CSR until
 * sc_graph_destroy. */
int sc_build_laplacian(sc_ctx* ctx, int32_t n, int64_t m, const int32_t* src,
                       const int32_t* dst, const float* w, int sym, int on_device,
                       sc_graph** out);
int sc_graph_info(const sc_graph* g, int32_t* n, int64_t* nnz, double* deg_max);
/* Copy the CSR to host arrays: row_ptr[n+1], col_idx[nnz], val[nnz] (may be NULL),
 * deg[n] (may be NULL). */
int sc_graph_copy_csr(const sc_graph* g, int32_t* row_ptr, int32_t* col_idx, float* val,
                      double* deg);
void sc_graph_destroy(sc_graph* g);

/* sc_lap_apply: Y = L V = D V - W V for an n x k block V (one SpMM; Sec. III: LOBPCG needs
 * one product of the graph matrix with a multi-vector per iteration).  prec selects FP32 (V, Y float*) or FP64 (double*);
 * V and Y are n x k row-major, host or device per on_device. */
int sc_lap_apply(sc_ctx* ctx, sc_graph* g, int k, int prec, const void* V, void* Y,
                 int on_device);

/* ---- LOBPCG (Sec. II.B; Sec. III random / warm start; Sec. IV soft locking) -----------
 * iters:    loop passes after the initial Rayleigh-Ritz on the start block.
 * tol_abs:  stop before a pass when max_j ||r_j|| <= tol_abs (0 = run all passes).
 * tol_lock: soft locking; columns with ||r_j|| <= tol_lock leave the active set (0 = off).
 * prec:     sc_precision.
 * seed:     seed of the Gaussian start block when one is generated.
 * cold:     1 = ignore a resident block and start cold.
 * precond:  sc_precond.  SC_PRECOND_NONE is the unpreconditioned iteration the paper ran
 *           (Sec. III); SC_PRECOND_JACOBI applies T = D^-1 (rows of isolated vertices
 *           unscaled) to the residual block before it enters the trial basis (the optional
 *           preconditioner T of LOBPCG, Sec. II.B).  Residual norms, tolerances and locking
 *           always refer to the unpreconditioned residual. */
enum { SC_PRECOND_NONE = 0, SC_PRECOND_JACOBI = 1 };
typedef struct {
  int iters;
  double tol_abs;
  double tol_lock;
  int prec;
  uint64_t seed;
  int cold;
  int precond;
} sc_lobpcg_opts;

typedef struct {
  int K;
  int iters_done;      /* passes run                                              */
  int fallbacks;       /* passes that had to drop the direction block P           */
  int converged;       /* 1 when tol_abs > 0 was reached                          */
  double lambda[SC_MAX_K]; /* Ritz values, ascending                              */
  double resid[SC_MAX_K];  /* ||L x_j - lambda_j x_j||_2 of the returned pairs     */
  float ms;            /* device time of the call (CUDA events on the ctx stream) */
  uint64_t kernels;    /* kernels launched by the call                           */
  int dropped;         /* residual columns dropped from a pass's trial basis
                          (Cholesky pivot below tolerance: the column had sunk to
                          rounding noise in the span of X and the other columns)  */
} sc_eig_info;

/* sc_lobpcg: the K smallest eigenpairs of the graph's Laplacian.
 * Start block: X0 (host n x K float, row-major) if non-NULL; its first x0_rows rows are
 * used and the rows below are zero-filled (snowball warm start, Sec. III); otherwise the
 * graph's resident block from the previous call (warm start) unless opts->cold, otherwise
 * a seeded Gaussian block (SplitMix64 + Box-Muller, seed opts->seed).  After the call the
 * graph keeps the new block resident for the next warm start.  X_out (host n x K float)
 * may be NULL.  info may be NULL. */
int sc_lobpcg(sc_ctx* ctx, sc_graph* g, int K, const sc_lobpcg_opts* opts, const float* X0,
              int32_t x0_rows, float* X_out, sc_eig_info* info);

/* sc_lobpcg64: sc_lobpcg with the start block and the result block in FP64 (Sec. II.B; the
 * FP64 form is the check mode whose Ritz vectors are compared with an FP64 reference).
 * X0: host n x K double (row-major; its first x0_rows rows, zero fill below) or NULL (the
 * resident or seeded Gaussian block, as sc_lobpcg).  X_out: host n x K double or NULL.  With
 * SC_PREC_FP64 the start block, every step and X_out are FP64; with the other precisions X0
 * is rounded to FP32 and X_out is the FP32 block widened.  The resident block kept for warm
 * starts is FP32, as after sc_lobpcg.  Errors as sc_lobpcg. */
int sc_lobpcg64(sc_ctx* ctx, sc_graph* g, int K, const sc_lobpcg_opts* opts, const double* X0,
                int32_t x0_rows, double* X_out, sc_eig_info* info);

/* sc_embed_rows: E_i = X_i / ||X_i||_2 (rows of norm < 1e-30 stay zero), n x K float. */
int sc_embed_rows(sc_ctx* ctx, const float* X, int32_t n, int K, float* E, int on_device);

/* ---- k-means on the embedded rows (Sec. II.A) -------------------------------------------
 * E: n x d float (row-major).  Seeds: init_idx[k] if non-NULL, else k-means++ driven by
 * the SplitMix64 uniforms of `seed` (decisions taken in FP64).  Lloyd: at most `iters`
 * assignment/update rounds, nearest centroid by squared distance (ties -> lowest index),
 * empty clusters keep their centroid, early exit when an assignment repeats.
 * Outputs (host, may be NULL except labels_out): labels_out[n], centroids_out[k*d]
 * (float), seeds_out[k], inertia (sum of squared distances), iters_run. */
int sc_kmeans(sc_ctx* ctx, const float* E, int32_t n, int d, int k, int iters,
              uint64_t seed, const int32_t* init_idx, int on_device, int32_t* labels_out,
              float* centroids_out, int32_t* seeds_out, double* inertia, int* iters_run);

/* sc_lobpcg_blocks: hard locking (Sec. IV) -- the K smallest eigenpairs computed nb columns
 * at a time: block b (columns b nb ...) runs sc_lobpcg in the orthogonal complement of the
 * Ritz vectors of the blocks before it (its start block and every residual block are
 * projected off them).  The device holds one block's workspace (3 nb columns wide) plus the
 * n x K result instead of a 3K-wide workspace.  Start blocks are the columns of X0 (host,
 * n x K FP32) when given, else seeded Gaussian blocks (seed + b); opts->cold is ignored and
 * opts->iters / tol_abs / tol_lock / precond apply to every block.  X_out (host n x K FP32)
 * may be NULL.  info: lambda and resid of all K pairs in block order; iters_done, fallbacks,
 * dropped, ms and kernels summed over blocks; converged = every block converged.  The result
 * becomes the graph's resident block.  Needs 1 <= nb <= K <= SC_MAX_K and 3 nb <= n. */
int sc_lobpcg_blocks(sc_ctx* ctx, sc_graph* g, int K, int nb, const sc_lobpcg_opts* opts,
                     const float* X0, float* X_out, sc_eig_info* info);

/* sc_lobpcg_batch: sc_lobpcg (seeded start block, or the resident block when !cold) for
 * `count` graphs at once.  Each solve runs on its own stream and the passes of all solves
 * are issued in turn, so their kernels overlap on the device -- in particular the one-CTA
 * small dense solves of different graphs run on different SMs.  Results are identical to
 * solving each graph alone (every reduction has a fixed order).  infos[count] may be NULL. */
int sc_lobpcg_batch(sc_ctx* ctx, int count, sc_graph* const* graphs, const int* K,
                    const sc_lobpcg_opts* opts, sc_eig_info* infos);

/* ---- end to end ------------------------------------------------------------------------
 * sc_partition: the spectral partition of Sec. II.A -- LOBPCG for the K smallest eigenpairs
 * of L (Sec. II.B) -> the rows of the eigenvector block scaled to unit length -> k-means (k
 * clusters, kmeans_iters Lloyd rounds, k-means++ seeded by opts->seed) -> labels_out[n]
 * (host).  The eigenvector block stays resident on the graph for a later warm start
 * (Sec. III).  Errors: those of sc_lobpcg and sc_kmeans; SC_EINVAL for k < 1 or k > n. */
int sc_partition(sc_ctx* ctx, sc_graph* g, int K, int k, const sc_lobpcg_opts* opts,
                 int kmeans_iters, int32_t* labels_out, sc_eig_info* info);

/* sc_cpqr_assign: cluster labels from an eigenvector block by QR with column pivoting, the
 * assignment the paper names beside k-means++ (Sec. II.A; Damle, Minden & Ying, arXiv
 * 1609.08251).  The K pivot rows of Y are chosen greedily (the row of the current residual
 * with the largest norm, lowest index on ties, then every residual row is projected off its
 * direction); Q is the polar factor of C = Y'[:, pivots]; label_i = argmax_j |(Y Q)_ij|
 * (lowest j on ties).  One cluster per column: k = K.  Arithmetic in FP64.
 * Y: n x K FP32 row-major, on the device when on_device = 1, else host (copied).
 * labels_out: n int32 (host).  pivots_out: K int32 (host) or NULL.
 * Errors: SC_EINVAL (null pointer, K < 1, K > n or K > SC_MAX_K), SC_ENOMEM, SC_ECUDA,
 * SC_EBREAKDOWN (non-finite polar factor). */
int sc_cpqr_assign(sc_ctx* ctx, const float* Y, int32_t n, int K, int on_device,
                   int32_t* labels_out, int32_t* pivots_out);

/* sc_eigengap: the number of clusters read off the smallest Laplacian eigenvalues (Sec. II.A:
 * the eigenvalues below the first significantly large increment count the clusters, and no
 * such increment means no reliable multi-way partition).  lam: l eigenvalues (host, any
 * order; sorted internally), e.g. sc_eig_info.lambda of an sc_lobpcg run with l slightly
 * above the expected count.  With d_i = lam_{i+1} - lam_i of the ascending values and
 * increments <= floor taken as 0 (floor: the accuracy of the eigenvalues), *k_out is i + 1
 * for the first i >= 1 with d_i > 0 and d_i > ratio * max(d_0 .. d_{i-1}), else 0.  Host
 * arithmetic in FP64, no device work.
 * Errors: SC_EINVAL (null pointer, l < 0 or l > SC_MAX_K, ratio <= 1, floor < 0 or not
 * finite, a non-finite eigenvalue). */
int sc_eigengap(const double* lam, int l, double ratio, double floor, int* k_out);

/* sc_partition_batch: sc_partition over `count` graphs with batched LOBPCG (labels_out[q]
 * has n_q entries; host). */
int sc_partition_batch(sc_ctx* ctx, int count, sc_graph* const* graphs, const int* K,
                       const int* k, const sc_lobpcg_opts* opts, int kmeans_iters,
                       int32_t* const* labels_out, sc_eig_info* infos);

/* ---- streaming (Sec. III: emerging edges, snowball) -------------------------------------
 * sc_stream_update: add m_delta directed edges to the graph and grow it to n_new >= n
 * vertices (new vertices numbered after the old ones, Sec. III).  The CSR is merged in
 * place of the old one (same symmetrization mode); the resident eigenvector block, if
 * any, gains zero rows for the new vertices so the next sc_lobpcg warm-starts. */
int sc_stream_update(sc_ctx* ctx, sc_graph* g, int32_t n_new, int64_t m_delta,
                     const int32_t* src, const int32_t* dst, const float* w, int on_device);

/* ---- serving loop (continuous batching of partition requests) ----------------------------
 * The paper's streaming setting (Sec. III: a graph G is partitioned, then G + g as new edges
 * and vertices arrive, each stage warm-started from the previous eigenvector block) served
 * as a request loop; the loop itself (queueing, admission, batching) has no counterpart in
 * the paper.  A server owns a context (used only by its worker thread; its HBM budget is the admission
 * limit).  Requests wait in a queue of queue_cap entries; up to max_slots solves run at once,
 * each advancing one LOBPCG pass per round on its own stream, and a request that arrives
 * while others run joins at the next pass boundary.  Graphs stay resident by graph_id:
 *   SC_REQ_COLD  -- build graph graph_id from the edge list (replacing a previous one) and
 *                   partition it from a seeded Gaussian start block;
 *   SC_REQ_DELTA -- add the edges to graph graph_id, grow it to n vertices (new vertices
 *                   numbered last) and partition it warm-started from its resident block
 *                   (zero rows for new vertices, Sec. III).
 * Requests on one graph_id run one at a time in submission order (a later request on a
 * graph waits while an earlier one is queued or running); requests on other graphs proceed.
 * Edge arrays are copied by sc_server_submit.  Results are identical to running the same
 * request alone.  A request whose estimated footprint exceeds the budget fails SC_ENOMEM.
 * The server functions are thread-safe. */
enum { SC_REQ_COLD = 0, SC_REQ_DELTA = 1 };
typedef struct {
  int kind;
  int graph_id;
  int32_t n;
  int64_t m;
  const int32_t* src;
  const int32_t* dst;
  int K;            /* LOBPCG block size                       */
  int k;            /* clusters                                */
  int iters;        /* LOBPCG passes (cap when tol_abs > 0)     */
  int kmeans_iters;
  int prec;         /* sc_precision                            */
  double tol_abs;   /* 0 = run `iters` passes                  */
  uint64_t seed;
} sc_request;
int sc_server_create(sc_ctx* ctx, int max_slots, int queue_cap, sc_server** out);
/* SC_EAGAIN when the queue is full. */
int sc_server_submit(sc_server* s, const sc_request* r, uint64_t* ticket);
/* Result of a finished request (labels_out: n_cap entries, host); SC_EAGAIN while pending.
 * latency_ms = submit to completion.  The ticket is consumed when the result is returned. */
int sc_server_poll(sc_server* s, uint64_t ticket, int32_t* labels_out, int32_t n_cap,
                   sc_eig_info* info, double* latency_ms);
/* As sc_server_poll, blocking up to timeout_ms (SC_ETIMEOUT when it runs out). */
int sc_server_wait(sc_server* s, uint64_t ticket, int timeout_ms, int32_t* labels_out,
                   int32_t n_cap, sc_eig_info* info, double* latency_ms);
int sc_server_stats(sc_server* s, int* active, int* queued, uint64_t* completed);
/* Finishes queued and running requests, then frees the server and its resident graphs. */
void sc_server_destroy(sc_server* s);

/* ---- component entry points (the steps of one LOBPCG pass, exposed for testing) -------
 * sc_gram: C = A' B in FP64 (a x b, row-major) for n x a block A and n x b block B
 * (row-major with leading dimensions lda, ldb in elements).  prec selects float or double
 * blocks and the arithmetic (MIXED = tensor cores, FP32 = CUDA cores, FP64).
 * A, B device or host per on_device; C host. */
int sc_gram(sc_ctx* ctx, int prec, int64_t n, int a, int b, const void* A, int64_t lda,
            const void* B, int64_t ldb, double* C, int on_device);

/* sc_tall_update: out = beta Cin + A W, the tall-skinny update of a LOBPCG pass (the new
 * X = [X R P] Y and its L-image, P = [R P] Y_RP; Knyazev 2001, Sec. II.B), for an n x a block A
 * (row-major, leading dimension lda), an a x b matrix W (row-major, dense), an optional n x b
 * Cin (NULL = no accumulate input; leading dimension ldc) and the n x b result out (leading
 * dimension ldo).  prec: SC_PREC_MIXED = tcgen05 tensor cores, 3-term split TF32 products with
 * FP32 accumulation (when the shape fits; otherwise CUDA cores); SC_PREC_FP32 / MIXED_DD = FP32
 * CUDA cores; SC_PREC_FP64 = double arrays and arithmetic.  Arrays are device or host per
 * on_device; the call returns after the result is written.
 * Errors: SC_EINVAL (sizes, null pointers), SC_ENOMEM, SC_ECUDA, SC_ETIMEOUT. */
int sc_tall_update(sc_ctx* ctx, int prec, int64_t n, int a, int b, const void* A, int64_t lda,
                   const void* W, const void* Cin, int64_t ldc, double beta, void* out,
                   int64_t ldo, int on_device);

/* sc_rr_solve: Rayleigh-Ritz in an orthonormal trial basis: the K smallest eigenpairs of
 * the symmetric m x m matrix G (host, FP64, row-major; symmetrized on entry).  theta[K]
 * ascending (host FP64), Y[m*K] (host FP64, row-major, orthonormal columns).
 * prec: SC_PREC_FP64 solves in FP64, otherwise in FP32. */
int sc_rr_solve(sc_ctx* ctx, int prec, int m, int K, const double* G, double* theta,
                double* Y);

/* ---- Gram without allocation -------------------------------------------------------------
 * sc_gram_static: C = A' B (FP64, a x b row-major) for FP32 device blocks A (n x a, stride
 * lda) and B (n x b, stride ldb), computed like sc_gram with SC_PREC_FP32 (CUDA cores, FP64
 * sums across row chunks) but allocating nothing: no cudaMalloc or cudaFree, no allocation by
 * any library, no context.  It is meant for callers that cannot allocate device memory, for
 * instance code inside a host framework that owns and partitions all device memory, or a
 * latency-critical loop that must not enter the allocator.  A, B and C are device pointers on
 * the current device; work is issued on cuda_stream (NULL = the legacy default stream) and
 * the call returns without waiting for it.
 * Scratch: the FP64 partial sums of the row chunks (split-K partials) live in one fixed
 * 8 MiB device array that the library defines (every GPU that loads the library holds it
 * until the process exits).  The array holds 256 chunk-tile partials of 64 x 64 entries, so
 * when the output has more than 128 such tiles (ceil(a/64) ceil(b/64) > 128, e.g. a and b
 * both above 704) every tile gets a single chunk: each entry is then one FP32 accumulation
 * over all n rows, with an error that grows with n instead of with the chunk length.
 * The first call on a device looks up that array's device address; make that first call
 * before any stream capture.  All calls share the array and it keeps the previous call's
 * contents, so calls whose work overlaps on the GPU (other streams, other threads) race and
 * must be serialized by the caller.
 * Limits: 1 <= a, b <= SC_GRAM_STATIC_MAX_COLS (SC_EINVAL beyond); n >= 0.
 * Errors: SC_EINVAL (sizes, null pointers), SC_ECUDA (launch or symbol lookup failed).
 * The paper has no counterpart: this entry point exists for callers that cannot allocate. */
#define SC_GRAM_STATIC_MAX_COLS 1024
int sc_gram_static(int64_t n, int a, int b, const float* A, int64_t lda, const float* B,
                   int64_t ldb, double* C, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SC_GB300_H */
