/*
 * graphgp.h -- C ABI of the GB300 GraphGP library (Vecchia approximation of a
 * Gaussian process on an arbitrary 3-D point cloud).
 *
 * Method: "GraphGP: Scalable Gaussian Processes with Vecchia's Approximation".
 * Citations below name the paper's section, equation or algorithm.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers ending in _d are DEVICE pointers on the current CUDA device;
 *    pointers ending in _h are HOST pointers.  The caller owns every buffer it
 *    passes; the library never frees or retains them after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call is stream-ordered.  Calls that must read a device
 *    value on the host (graph build, status queries, save) synchronise
 *    `stream` and say so.
 *  - Handles (graphgp_graph_t, graphgp_factor_t) own device memory allocated
 *    with the stream-ordered allocator on the stream given at creation, until
 *    the matching *_destroy call.  A handle may be used on any stream, but
 *    calls that use one handle must not overlap on the device.
 *  - Vectors (xi, v and their cotangents) are float[N] in GRAPH ORDER: the
 *    depth-sorted generation order of Sec. 2.2 ("Batch construction").
 *    order[pos] gives the input index of the point at position pos.
 *  - Every call returns a graphgp_status.  Argument errors are reported
 *    before any work is enqueued and leave outputs untouched.  Errors found on
 *    the device (a bounded wait that timed out, a non-positive pivot) are
 *    recorded in the handle and returned by graphgp_sync_status.
 *  - Sizes: 1 <= k <= 64 neighbours (the range the paper gives for its GPU
 *    method, Sec. 2.3), 1 <= d <= 3, k <= n0 <= N, n0 <= 2048, N < 2^31.
 */
#ifndef GRAPHGP_H
#define GRAPHGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct graphgp_graph_s* graphgp_graph_t;
typedef struct graphgp_factor_s* graphgp_factor_t;

typedef enum {
  GRAPHGP_OK = 0,
  GRAPHGP_ERR_INVALID = -1, /* bad argument or size */
  GRAPHGP_ERR_OOM = -2,     /* device allocation failed */
  GRAPHGP_ERR_CUDA = -3,    /* a CUDA runtime call failed */
  GRAPHGP_ERR_TIMEOUT = -4, /* a bounded device wait gave up */
  GRAPHGP_ERR_NAN = -5,     /* non-finite input coordinates */
  GRAPHGP_ERR_IO = -6,      /* file could not be read or written */
  GRAPHGP_WARN_NOT_PD = 1   /* some pivots were clamped (Sec. 2.1, Eq. 2) */
} graphgp_status;

/* Stationary covariance kappa(r) (Sec. 2.1).  Matern with half-integer
 * smoothing nu in {1/2, 3/2, 5/2} in closed form, and the squared
 * exponential.  The nugget is added to K_ii only (same point, never to two
 * distinct coincident points). */
typedef enum {
  GRAPHGP_MATERN12 = 0, /* s2 * exp(-r/l)                                   */
  GRAPHGP_MATERN32 = 1, /* s2 * (1 + sqrt3 r/l) exp(-sqrt3 r/l)             */
  GRAPHGP_MATERN52 = 2, /* s2 * (1 + sqrt5 r/l + 5r^2/(3l^2)) exp(-sqrt5 r/l) */
  GRAPHGP_SQEXP = 3     /* s2 * exp(-r^2/(2 l^2))                           */
} graphgp_kernel_type;

typedef struct {
  int32_t type;       /* graphgp_kernel_type */
  int32_t reserved;   /* must be 0 */
  double sigma2;      /* marginal variance s2 > 0 */
  double lengthscale; /* l > 0 */
  double nugget;      /* >= 0, added on the diagonal */
  double rescue_tol;  /* precision policy of the per-point conditionals (not
                         in the paper, which runs one precision).  Every
                         conditional is factored in FP32 (in increments of
                         the field when its nearest neighbour is close, see
                         graphgp_factor); its relative error is estimated a
                         priori as
                           est = 2^-20 max_j (M_jj / p_j)
                                 (1 + 2^-8 Var(w) / sigma_i^2)
                         (M the covariance the row factors, p_j its Cholesky
                         pivots: a lower bound on M's scaled condition
                         number; Var(w) / sigma_i^2 the cancellation in the
                         conditional variance).  A row with est > rescue_tol,
                         a floored pivot or a non-finite result is recomputed
                         in FP64; so is the dense block when 2^-24 (K_00 /
                         p_min)^2 exceeds it.  0 = default 2^-7; < 0 = every
                         conditional in FP64 (slow on GB300: FP64 runs at a
                         small fraction of the FP32 rate).  Must be finite. */
} graphgp_kernel;

typedef struct {
  int32_t n0;         /* size of the dense initial block (Sec. 2.2; the
                         dense initial batch of Alg. 1); 0 = default
                         min(N, max(k, 256)) */
  int32_t split_rule; /* k-d split dimension: 0 = widest bounding-box extent
                         (ties to the lowest dimension), 1 = level mod 3
                         (d = 3 only) */
  int64_t max_spin;   /* bound on device spin iterations; 0 = default */
} graphgp_build_opts;

/* ---- graph construction (Sec. 2.2, Sec. 2.3 last paragraph) ------------
 * Builds the bit-reversed left-balanced k-d tree over points_d (float[N][d],
 * d = 1, 2 or 3, row-major, input order; points of d < 3 are held as 3-D
 * points with zero in the missing coordinates, which changes no distance and
 * no split), the k nearest PRECEDING neighbours of every point with tree
 * index >= n0 (key: FP32 squared distance, ties to the lower tree index),
 * the depth of every point (d_i = 1 + max over c(i), dense block = 0), and
 * the depth-sorted graph order (ties by k-d tree in-order rank).
 * Synchronises `stream` (the host needs the number of depth levels).
 * Returns GRAPHGP_ERR_NAN for non-finite coordinates; -0.0 is read as +0.0. */
int graphgp_build_graph(const float* points_d, int64_t N, int d, int k,
                        const graphgp_build_opts* opts, void* stream,
                        graphgp_graph_t* out);

/* Creates a graph handle from host arrays that already hold a graph in graph
 * order: points_h float[N][3] in INPUT order, order_h int32[N] (position ->
 * input index), nbr_h int32[(N-n0)*k] (row pos-n0 holds the positions of
 * c(pos), each < level_offsets[depth(pos)]), level_offsets_h
 * int64[num_levels+1] with level_offsets_h[0] = 0, level_offsets_h[1] = n0,
 * level_offsets_h[num_levels] = N.  Used by graphgp_graph_load.  Validates
 * every index; synchronises `stream`. */
int graphgp_graph_import(const float* points_h, int64_t N, int k, int n0,
                         const int32_t* order_h, const int32_t* nbr_h,
                         const int64_t* level_offsets_h, int num_levels,
                         void* stream, graphgp_graph_t* out);

/* num_levels counts depth levels including the dense level 0, so the
 * level_offsets array has num_levels+1 entries.  bytes = device bytes held. */
int graphgp_graph_info(graphgp_graph_t g, int64_t* N, int* k, int* n0,
                       int* num_levels, size_t* bytes);

/* Copies the graph out.  order_d int32[N], nbr_d int32[(N-n0)*k] (positions,
 * nearest first), level_offsets_h int64[num_levels+1].  Any pointer may be
 * NULL to skip it.  Synchronises `stream` when level_offsets_h != NULL. */
int graphgp_graph_export(graphgp_graph_t g, int32_t* order_d, int32_t* nbr_d,
                         int64_t* level_offsets_h, void* stream);

/* Copies the k-d tree out (only for graphs made by graphgp_build_graph):
 * tree_point_d int32[N] (tree index -> input index), split_dim_d uint8[N],
 * inorder_d int32[N] (tree index -> in-order rank), depth_d int32[N] (tree
 * index -> depth), nbr_tree_d int32[(N-n0)*k] (tree index j >= n0 -> tree
 * indices of c(j), nearest first).  Any pointer may be NULL.  Fails with
 * GRAPHGP_ERR_INVALID if the tree arrays were released. */
int graphgp_graph_export_tree(graphgp_graph_t g, int32_t* tree_point_d,
                              uint8_t* split_dim_d, int32_t* inorder_d,
                              int32_t* depth_d, int32_t* nbr_tree_d,
                              void* stream);

/* Versioned binary checkpoint of a graph (points, order, neighbours, level
 * offsets).  Save synchronises `stream`. */
int graphgp_graph_save(graphgp_graph_t g, const char* path, void* stream);
int graphgp_graph_load(const char* path, void* stream, graphgp_graph_t* out);

void graphgp_graph_destroy(graphgp_graph_t g);

/* ---- factor (Sec. 2.1, Eq. 2; Alg. 1) -----------------------------------
 * For every position i >= n0: the weights b_i = K_ic K_cc^-1 of Eq. 2 and
 * sigma_i^2 = K_ii - K_ic K_cc^-1 K_ci, by a Cholesky factor in FP32 (sigma^2
 * accumulated compensated).  Rows whose nearest neighbour is close (variogram
 * g = kappa(0) - kappa(r) below kappa(0)/2) are factored in increments of
 * the field centred on that neighbour, an exact change of variables whose
 * covariances are sums of variogram values; the others in the covariance
 * form.  Rows flagged by kern->rescue_tol are recomputed in FP64.  Dense
 * block: L0 = chol(K_00) over positions 0..n0-1 and its inverse, sigma_i =
 * L0_ii (FP64 when flagged).  logdet = 2 sum_i log sigma_i is reduced in FP64
 * from the stored FP32 sigma.  Pivots below 1e-7 (kappa(0) + nugget) are
 * clamped to that value and counted (see graphgp_sync_status).  Allocates
 * stream-ordered scratch (a list of rows for the FP64 pass, FP64 work arrays
 * of 2 n0^2 doubles). */
int graphgp_factor(graphgp_graph_t g, const graphgp_kernel* kern, void* stream,
                   graphgp_factor_t* out);

/* b_d float[(N-n0)*k] (row-major, same neighbour order as the graph),
 * sigma_d float[N], L0_d float[n0*n0] (row-major, lower triangle, upper
 * entries zero).  Any pointer may be NULL. */
int graphgp_factor_export(graphgp_factor_t f, float* b_d, float* sigma_d,
                          float* L0_d, void* stream);

void graphgp_factor_destroy(graphgp_factor_t f);

/* Synchronises `stream`, then reports device-side conditions recorded in the
 * handles (either may be NULL): GRAPHGP_ERR_TIMEOUT if a bounded wait gave
 * up, else GRAPHGP_WARN_NOT_PD if the factor clamped pivots, else OK.
 * n_not_pd (nullable) receives the number of clamped rows. */
int graphgp_sync_status(graphgp_graph_t g, graphgp_factor_t f, void* stream,
                        int64_t* n_not_pd);

/* ---- sweeps (Alg. 1; Sec. 3 "inverse and log-determinant") --------------
 * generate: v = L xi, i.e. v_0 = L0 xi_0, then level by level
 *           v_i = b_i . v_c(i) + sigma_i xi_i.
 * whiten:   xi = L^-1 v, i.e. xi_0 = L0^-1 v_0, xi_i = (v_i - b_i.v_c(i))/sigma_i.
 * logdet:   out_d[0] = log det(L L^T) = 2 sum log sigma_i (double, device).
 * nll:      out_d[0] = 0.5 xi.xi + 0.5 logdet with xi = whiten(v) (double).
 * generate's v_d must not overlap xi_d (GRAPHGP_ERR_INVALID): v_d is written
 * while xi_d is still being read. */
int graphgp_generate(graphgp_graph_t g, graphgp_factor_t f, const float* xi_d,
                     float* v_d, void* stream);
int graphgp_whiten(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                   float* xi_d, void* stream);
int graphgp_logdet(graphgp_factor_t f, double* out_d, void* stream);
int graphgp_nll(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                double* out_d, void* stream);

/* The same value as graphgp_nll, computed without allocating device memory
 * during the call (the paper has no counterpart; this serves callers that
 * cannot allocate while they run, e.g. a serving loop that reserved all
 * device memory for resident graphs up front, or a latency-critical path that
 * must not pay cudaMalloc's device-wide synchronisation).  The reduction
 * scratch is a 514 KiB array inside the library, one FP64 slot per eight
 * dense rows (up to 256) and one per whiten tile (4096 points): graphs with
 * N > 2^28 points or more than 8192 depth levels are rejected with
 * GRAPHGP_ERR_INVALID, before any work and without writing out_d.  The
 * array's device address is looked up on the first call made on each device
 * (make that call before any stream capture) and kept for the life of the
 * process: a cudaDeviceReset on that device voids it, so do not call this
 * entry point after resetting the device.  The array stays allocated on
 * every device that loaded the library until the process exits.  All calls share it: calls that
 * overlap on the GPU race, so never run two concurrently on one device.
 * The final sum runs in a fixed order. */
int graphgp_nll_noalloc(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                        double* out_d, void* stream);

/* ---- on-the-fly sweeps (Alg. 1 as printed: factors never stored) --------
 * The same operators as graphgp_generate / graphgp_whiten / graphgp_nll with
 * the conditioning factor of every point (Sec. 2.1 Eq. 2) recomputed inside
 * the pass from the coordinates and `kern` (same validity rules as
 * graphgp_factor), so no graphgp_factor_t is needed and the device holds the
 * graph alone (about k + 4 words per point instead of 2k + 5).  For kernel
 * parameters that change at every step.  Requires k <= 32, else
 * GRAPHGP_ERR_INVALID (k <= 16: one thread per point; 16 < k <= 32: one warp
 * per point).  Results are bit-identical to graphgp_factor followed by the
 * stored-factor sweep (the factor and the dot products run in the same
 * order); the log-determinant equals graphgp_logdet up to the order of its
 * FP64 partial sums.
 *   generate_fused: v_d = L xi_d.
 *   whiten_fused:   xi_d = L^-1 v_d; logdet_d (nullable, double, device) is
 *                   overwritten with log det(L L^T).
 *   nll_fused:      nll_d[0] = 0.5 xi.xi + 0.5 logdet (uses the graph's work
 *                   vector; do not overlap with other calls on the graph).
 * not_pd_d (nullable, uint64 on the device) has the number of floored pivots
 * ADDED to it.  Each call allocates stream-ordered scratch for the dense
 * block (2 n0^2 floats). */
int graphgp_generate_fused(graphgp_graph_t g, const graphgp_kernel* kern, const float* xi_d,
                           float* v_d, uint64_t* not_pd_d, void* stream);
int graphgp_whiten_fused(graphgp_graph_t g, const graphgp_kernel* kern, const float* v_d,
                         float* xi_d, double* logdet_d, uint64_t* not_pd_d, void* stream);
int graphgp_nll_fused(graphgp_graph_t g, const graphgp_kernel* kern, const float* v_d,
                      double* nll_d, uint64_t* not_pd_d, void* stream);

/* NLL value and gradient in one pass with the factors recomputed, never
 * stored (Sec. 2.3 derivatives of the conditioning steps): nll_d[0] =
 * nll(v), vbar_d = nllbar dNLL/dv (overwritten), thetabar_d += nllbar
 * dNLL/d(lengthscale, sigma2, nugget) -- what graphgp_factor + graphgp_nll +
 * graphgp_nll_backward return, with one computation of every row's
 * conditional instead of two.  The form for kernel parameters that change at
 * every step (a fit).  k <= 32 (one thread per point for k <= 16, one warp
 * per point above); each call allocates stream-ordered scratch for the dense
 * block and the FP64 rescue list.  not_pd_d as for the other on-the-fly
 * calls.  vbar and thetabar agree with the stored-factor calls to rounding
 * (atomic sums). */
int graphgp_nll_grad_fused(graphgp_graph_t g, const graphgp_kernel* kern,
                           const float* v_d, double nllbar, double* nll_d,
                           float* vbar_d, double* thetabar_d, uint64_t* not_pd_d,
                           void* stream);

/* ---- adjoints (Sec. 2.3 "forward and backward derivatives") -------------
 * Vector-Jacobian products.  thetabar_d is double[3] =
 * [d/d lengthscale, d/d sigma2, d/d nugget] and is ACCUMULATED (+=).  The
 * per-point factors are recomputed, not stored.
 * generate_backward: given vbar = dL/dv for v = generate(xi), writes
 *   xibar_d (overwritten) and adds the kernel-parameter gradient.
 * whiten_backward: given xibar = dL/dxi for xi = whiten(v) and a scalar
 *   logdetbar = dL/dlogdet, writes vbar_d (overwritten) and adds thetabar.
 * nll_backward: gradient of nll(v) times nllbar: vbar_d, thetabar_d.
 * thetabar_d may be NULL: then only the vector cotangent is formed (the
 * sweeps and scatters) and the per-row factor backward, which recomputes
 * every row's conditional, is skipped -- the case of a fixed kernel.
 * The transposed sums (a position's cotangent from all rows that condition
 * on it) are formed with atomic adds, so vbar_d / xibar_d and thetabar_d
 * agree between calls to rounding, not bit for bit. */
int graphgp_generate_backward(graphgp_graph_t g, graphgp_factor_t f,
                              const float* xi_d, const float* v_d,
                              const float* vbar_d, float* xibar_d,
                              double* thetabar_d, void* stream);
int graphgp_whiten_backward(graphgp_graph_t g, graphgp_factor_t f,
                            const float* v_d, const float* xi_d,
                            const float* xibar_d, double logdetbar,
                            float* vbar_d, double* thetabar_d, void* stream);
int graphgp_nll_backward(graphgp_graph_t g, graphgp_factor_t f,
                         const float* v_d, double nllbar, float* vbar_d,
                         double* thetabar_d, void* stream);

/* ---- position ranges (sharding factor, NLL and NLL gradient) ------------
 * Not a paper operation: the pieces with which several GPUs (one process
 * each) split the factor, the NLL and its gradient by contiguous ranges of
 * graph positions (the conditionals of Eq. 2 are independent per point once
 * the neighbours' coordinates and field values are known).  Each process
 * holds the whole graph; the sums over disjoint ranges that cover 0..N add
 * up to graphgp_factor's log-determinant, graphgp_nll and
 * graphgp_nll_backward.
 * graphgp_factor_rows: a factor handle holding the conditionals of positions
 *   [pos_begin, pos_end) only; pos_begin is 0 (the dense block is then
 *   factored too, and pos_end >= n0 is required) or >= n0.  b and sigma of
 *   other positions are zero.  Its logdet covers its own positions.  Such a
 *   handle is accepted only by graphgp_factor_export, graphgp_logdet,
 *   graphgp_sync_status and the two calls below; the whole-graph sweeps and
 *   adjoints return GRAPHGP_ERR_INVALID for it.
 * graphgp_nll_rows: out_d[0] = 0.5 sum_{own i} xi_i^2 + 0.5 logdet(f), with
 *   v_d float[N] valid at the own positions and at every neighbour of them.
 * graphgp_nll_backward_rows: the own positions' part of the NLL gradient
 *   times nllbar: ACCUMULATED into vbar_d float[N] (own positions and their
 *   neighbours; sum vbar_d over the ranges) and into thetabar_d double[3].
 *   Uses the graph's work vectors (do not overlap with other calls on it). */
int graphgp_factor_rows(graphgp_graph_t g, const graphgp_kernel* kern, int64_t pos_begin,
                        int64_t pos_end, void* stream, graphgp_factor_t* out);
int graphgp_nll_rows(graphgp_graph_t g, graphgp_factor_t f, const float* v_d, double* out_d,
                     void* stream);
int graphgp_nll_backward_rows(graphgp_graph_t g, graphgp_factor_t f, const float* v_d,
                              double nllbar, float* vbar_d, double* thetabar_d, void* stream);

/* Gradient of nll(v) times nllbar with respect to the point coordinates
 * (Sec. 2.3's derivatives carried through the stationary kernel kappa(r) to
 * the points), with the graph -- order, neighbour lists, depth levels --
 * held fixed, as it is for every other derivative here.  pbar_d is
 * float[N][3] in INPUT order (the layout of the points given to
 * graphgp_build_graph; for d < 3 the trailing columns belong to the zero
 * padding), overwritten.  Matern-1/2 is not differentiable at r = 0; a pair
 * of coincident points contributes 0 there.  Uses the graph's work vectors
 * (do not overlap with other calls on the graph) and allocates
 * stream-ordered scratch of 24 N bytes. */
int graphgp_nll_backward_points(graphgp_graph_t g, graphgp_factor_t f,
                                const float* v_d, double nllbar, float* pbar_d,
                                void* stream);

/* ---- serving (continuous batching over resident instances) -------------
 * Not a paper algorithm: an engine that serves the operations above, each
 * request on one resident instance (a graph with its factor).  A native
 * scheduler thread admits queued requests in arrival order while a stream
 * slot is free and the device bytes of the requests in flight stay within
 * hbm_budget (0 = 8 GiB); requests on different slots overlap on the device.
 * One request per instance runs at a time.  With use_graphs, the first
 * request of each (instance, operation, slot) is captured into a CUDA graph
 * that later requests replay.
 *   op GENERATE: in_h = xi[N] -> out_h = v[N]
 *   op WHITEN:   in_h = v[N]  -> out_h = xi[N]
 *   op LOGDET:   scal_h[0] = logdet
 *   op NLL_GRAD: in_h = v[N]  -> out_h = dNLL/dv[N], scal_h[0] = NLL,
 *                scal_h[1..3] = dNLL/d(lengthscale, sigma2, nugget)
 * in_h/out_h are host buffers (pinned for asynchronous copies); out_h and
 * scal_h may be NULL (results land in the slot's staging buffers).  The
 * caller keeps every buffer alive until the request completes.  Instances
 * must stay alive until graphgp_server_destroy, and must not be used by
 * other calls while the server runs. */
typedef struct graphgp_server_s* graphgp_server_t;
enum { GRAPHGP_OP_GENERATE = 0, GRAPHGP_OP_WHITEN = 1, GRAPHGP_OP_LOGDET = 2,
       GRAPHGP_OP_NLL_GRAD = 3 };

int graphgp_server_create(int n_slots, size_t hbm_budget, int use_graphs,
                          graphgp_server_t* out);
/* Before graphgp_server_start only (synchronises the device). */
int graphgp_server_register(graphgp_server_t sv, graphgp_graph_t g,
                            graphgp_factor_t f, int* instance_id);
int graphgp_server_start(graphgp_server_t sv);
/* arrival_s: the request's arrival time on the host monotonic clock
 * (CLOCK_MONOTONIC seconds; <= 0 means now).  Writes a ticket. */
int graphgp_server_submit(graphgp_server_t sv, int instance_id, int op,
                          const float* in_h, float* out_h, double* scal_h,
                          double arrival_s, uint64_t* ticket);
/* Waits up to timeout_s for a ticket; returns its status (GRAPHGP_ERR_TIMEOUT
 * if still running).  times_out (nullable) = [arrival, admit, done]. */
int graphgp_server_wait(graphgp_server_t sv, uint64_t ticket, double timeout_s,
                        double* times_out);
int graphgp_server_stats(graphgp_server_t sv, int64_t* completed, int64_t* errors,
                         int64_t* queued, size_t* bytes_in_flight);
/* Drains the queue, joins the scheduler and frees the server (not the
 * instances). */
void graphgp_server_destroy(graphgp_server_t sv);

/* Self-test of the bounded device waits of the level sweeps (not a paper
 * operation): a small cooperative launch waits at a level barrier that no
 * block ever reaches, giving up after max_spin polls (1 <= max_spin <= 2^30).
 * Synchronises `stream`.  Returns GRAPHGP_ERR_TIMEOUT when the waits gave up
 * and recorded the timeout as designed (the context stays usable). */
int graphgp_selftest_wait_timeout(int64_t max_spin, void* stream);

/* Writes the compute capability the library's device code was loaded for
 * (cudaFuncAttributes::binaryVersion of one of its kernels: major*10+minor,
 * 103 on GB300).  Not a paper operation.  Loads the module on the current
 * device if needed. */
int graphgp_binary_version(int* version);

const char* graphgp_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* GRAPHGP_H */
