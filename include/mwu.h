/*
 * mwu.h -- C ABI of a GB300 (sm_103a) solver for positive linear programs by the
 * multiplicative-weight-update (MWU) method with step-size search of
 * arXiv 2307.03307 ("Efficient Parallel Implementation of the Multiplicative
 * Weight Update Method for Graph-based Linear Programs").
 *
 * Problem statement (Sec. 2.2, Eq. NormFeasibleLP): find x >= 0 with
 *     P x <= 1  (packing rows, P in R_+^{m_P x n})  and  C x >= 1  (covering rows),
 * to a (1+eps)-relative approximation.  Pure packing (max c^T x, P x <= 1) and
 * pure covering (min c^T x, C x >= 1) embed the objective as one extra row
 * (1/M) c^T x >= 1 or <= 1 and search on M (Sec. 2.2); densest subgraph fixes D
 * in W z >= 1, O z <= D (Sec. 3, Eq. densest_linalg) and searches on D.
 *
 * Conventions for every entry point:
 *   - Every call returns an int status (mwu_status); nothing aborts or throws
 *     across this boundary.  Negative values are errors; mwu_last_error(ctx)
 *     gives a one-line message.
 *   - Input pointers may be host or device memory (the library copies with
 *     cudaMemcpyDefault during mwu_create and never keeps a caller pointer).
 *   - All device work of a context is issued on opt.stream (NULL = a stream
 *     the context creates).  A context is not thread safe.
 *   - Indices are int32; sizes int64.  Vectors of the FP32 form are float32,
 *     of the FP64 form float64.
 *   - MWU_FAULT_ALLOC_AT=k in the environment makes the k-th device allocation
 *     of each context fail (a host-side fault injection): the call returns
 *     MWU_ERR_OOM and releases everything it had allocated.
 */
#ifndef MWU_H_
#define MWU_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
    MWU_OK = 0,
    MWU_FEASIBLE = 0,       /* probe ended with max(Px) <= (1+eps) min(Cx), min(Cx) >= 1 (Theorem 4.1) */
    MWU_INFEASIBLE = 1,     /* d = 0, alpha < 1 (Alg. 2), or packing rows past 1+eps          */
    MWU_MAX_ITER = 2,       /* iteration cap reached (5000 in Sec. 6)                           */
    MWU_RUNNING = 3,        /* mwu_iterate returned before the probe ended                      */
    MWU_ERR_INVALID = -1,   /* bad argument or malformed matrix                                 */
    MWU_ERR_CUDA = -2,      /* a CUDA call failed                                               */
    MWU_ERR_OOM = -3,       /* device allocation failed                                         */
    MWU_ERR_NUMERIC = -4,   /* NaN/Inf met in a reduction                                       */
    MWU_ERR_TIMEOUT = -5,   /* a bounded loop gave up: the step search ran more turns than
                               max_passes + 4 (MWU_SEARCH_GUARD=n in the environment sets
                               that bound, a test hook); the context stays usable          */
    MWU_ERR_STATE = -6      /* call out of order (e.g. candidates before a direction)           */
} mwu_status;

/* Infeasibility reasons reported in mwu_iter_stats.reason. */
enum { MWU_REASON_NONE = 0, MWU_REASON_COVERED = 1, MWU_REASON_PACKING = 2,
       MWU_REASON_D_ZERO = 3, MWU_REASON_ALPHA = 4, MWU_REASON_MAX_ITER = 5,
       MWU_REASON_RATIO = 6 /* FEASIBLE by the scale-invariant rule (stop_rule = 1) */ };

/* ------------------------------------------------------------ problem kind */
typedef enum {
    MWU_PACKING = 0,   /* max c^T x s.t. P x <= 1 ; C is the objective row (1/M) c^T        */
    MWU_COVERING = 1,  /* min c^T x s.t. C x >= 1 ; P is the objective row (1/M) c^T        */
    MWU_MIXED = 2,     /* feasibility: P x <= 1, C x >= 1 (no objective, no target)          */
    MWU_DENSEST = 3    /* min D s.t. W z >= 1, O z <= D ; P = O/D, C = W, built from a graph */
} mwu_kind;

/* --------------------------------------------------------- matrix kinds */
/* Sec. 3 matrices and their implicit forms (Sec. 5.1.2).  Edge lists are
 * int32 pairs (u_e, v_e) interleaved, u_e != v_e, each undirected edge once. */
typedef enum {
    MWU_MAT_CSR = 0,          /* explicit CSR rows x cols (rowptr, colidx, val or NULL = ones)   */
    MWU_MAT_INCIDENCE = 1,    /* M, n_vertices x n_edges: M[w,e] = 1 iff w in e (Eq. incidence)  */
    MWU_MAT_INCIDENCE_T = 2,  /* M^T, n_edges x n_vertices (vertex cover, Sec. 3)                */
    MWU_MAT_PAIR = 3,         /* O, n_vertices x 2 n_edges: O[w, 2e+b] = 1 iff w is endpoint b   */
    MWU_MAT_INTERWEAVE = 4,   /* W, n_edges x 2 n_edges: W[e,2e] = W[e,2e+1] = 1 (Eq. interweaved)*/
    MWU_MAT_NONE = 5          /* side given by the objective row                                 */
} mwu_mat_kind;

typedef struct {
    int32_t kind;              /* mwu_mat_kind                                               */
    int32_t rows, cols;        /* CSR only (implicit kinds derive them)                      */
    int64_t nnz;               /* CSR only                                                   */
    const int32_t *rowptr;     /* CSR: rows+1 entries, rowptr[0] = 0, non-decreasing         */
    const int32_t *colidx;     /* CSR: nnz column indices in [0, cols)                       */
    const float *val;          /* CSR: nnz values >= 0, finite; NULL = all ones              */
    const int32_t *edges;      /* implicit kinds: 2*n_edges int32 (u0,v0,u1,v1,...)          */
    int32_t n_vertices;        /* implicit kinds                                             */
    int64_t n_edges;           /* implicit kinds                                             */
    const float *row_bound;    /* optional, rows entries > 0: row j reads (A x)_j <= b_j
                                  (packing) or >= b_j (covering), i.e. diag(1/b) A
                                  (Appendix A.1 bounds); NULL = all ones                   */
} mwu_matrix;

/* --------------------------------------------------------------- options */
enum { MWU_STEP_KARY = 0,      /* K candidates per pass (Alg. 3 generalised; K = 1 is Alg. 3) */
       MWU_STEP_BINARY = 1,    /* Alg. 3 as printed: one candidate per pass                  */
       MWU_STEP_STANDARD = 2,  /* alpha = 1 (Alg. 1)                                         */
       MWU_STEP_NEWTON = 3 };  /* Newton's method on f(alpha) = 1 (Sec. 4.2): warm start from
                                  the previous alpha (else the exponential phase), one
                                  candidate and Psi', Phi' per pass, then the (1-eps)^p
                                  backoff, one value per pass; a passing value that covers
                                  every row ends the search with the smallest covering step
                                  (Alg. 3's early exit)                                     */
enum { MWU_PREC_F32_R64 = 0,   /* FP32 vectors and per-element math, FP64 reductions         */
       MWU_PREC_FP64 = 1 };    /* everything FP64, one candidate per pass, host-driven search*/

typedef struct {
    double eps;                /* (0,1); default 0.1                                          */
    int32_t max_iter;          /* MWU iterations per probe; default 5000 (Sec. 6)             */
    double eta_factor;         /* eta = eta_factor ln(m_P+m_C)/eps; default 10 (Alg. 1)      */
    int32_t step;              /* MWU_STEP_*; default KARY                                    */
    int32_t K;                 /* candidates per pass, 1..8; default 8 (FP64 form forces 1)  */
    int32_t max_passes;        /* candidate passes per iteration; default 6 (F32 K-candidate),
                                  16 (F32 Newton), 64 (FP64 or K = 1)                       */
    int32_t warm_start;        /* start the exponential phase at floor(log2 alpha_prev)      */
    int32_t double_single;     /* c_d = 1/eta when one side is a single row (Sec. 2.2)       */
    int32_t precision;         /* MWU_PREC_*; default F32_R64                                 */
    double outer_tol;          /* bisection stops when hi <= (1+outer_tol) lo; default eps   */
    int32_t max_probes;        /* default 64                                                  */
    int32_t use_graph;         /* capture one iteration in a CUDA graph (F32 form); default 1 */
    int32_t check_every;       /* iterations between host reads of the status; default 8     */
    int32_t group;             /* lanes per CSR row, 0 = automatic; else 1,2,4,8,16,32       */
    int32_t timing;            /* record CUDA events around each kernel class of every
                                  iteration (read with mwu_get_timing); default 0           */
    int32_t stop_rule;         /* 0 (default): a probe ends FEASIBLE once min(Cx) >= 1 with
                                  max(Px) <= (1+eps) min(Cx) (Alg. 2); 1: as soon as
                                  max(Px) <= (1+eps) min(Cx), min(Cx) > 0 -- x/min(Cx) is
                                  then the (1+eps)-relative solution of Theorem 4.1 (the LP
                                  is homogeneous).  Inside mwu_solve a probe also ends as
                                  soon as its certificate closes the search bracket.     */
    double grad_tol;           /* gradient test d_i > 0 iff g_i < (1 - grad_tol) h_i; < 0
                                  selects the default: 2^-16 for F32_R64 (a few FP32
                                  roundings of g/h, below which d = 0 is undecidable in
                                  FP32), 0 for FP64 (the exact test of Alg. 2)             */
    void *stream;              /* cudaStream_t for all of the context's work.  NULL = a
                                  blocking stream the context creates and owns: it waits
                                  for work queued on the legacy default stream, so inputs
                                  written there before a call are complete when read.
                                  With a stream of its own, the caller orders its inputs
                                  on that stream                                             */
    int32_t max_newton;        /* Newton evaluations per step search; default 8              */
    double newton_tol;         /* Newton has converged once |alpha' - alpha| <= newton_tol
                                  alpha; <= 0 selects eps/20                                 */
    int32_t batch_workers;     /* mwu_solve_batch: threads per block of the persistent batch
                                  solve, 256, 512 or 1024; 0 (default) = autotuned together
                                  with batch_cluster: the first solve times the whole batch
                                  in each configuration of mwu_batch_tuning and keeps the
                                  fastest                                                  */
    int32_t drop_covered;      /* 1: keep only the unsatisfied covering rows, the last step
                                  of the loop of Alg. 1 and Alg. 2 (C <- {c_j : c_j^T x < 1}):
                                  a row with (Cx)_j >= 1 leaves smin, h, Phi and Phi'.  x
                                  never decreases, so the active rows are those with
                                  (Cx)_j < 1.  On the vertex-cover split view the rows are
                                  also compacted: inside one mwu_iterate call, whenever
                                  the unsatisfied edges are at most 70 % of the current
                                  rows, a stable stream compaction keeps only them for the
                                  SpMV dz = Cd, the candidate passes and the update (the
                                  direction still reads every column); the call restores
                                  the full rows, with z = Cx, before it returns.  2: the
                                  same dropping without compaction (rows masked in place).
                                  0 (default): every row is kept, as the paper's
                                  implementation does (Sec. 4)                             */
    int32_t spmv_tiles;        /* forward SpMV of an explicit or incidence CSR side: 0
                                  (default) stages each tile of rows' input window in
                                  shared memory when the columns of 90 % of the tiles
                                  span at most 12288 (FP32) / 6144 (FP64) entries, as on
                                  banded matrices (the CSB-like tiles of Sec. 5.1); -1
                                  always uses the row-binned gather kernel               */
    int32_t h_scatter;         /* covering side of edge rows (MWU_MAT_INCIDENCE_T, vertex
                                  cover) or an explicit CSR (dominating set): 1 computes
                                  h = C^T w_c by one pass over C's rows with atomic adds
                                  into per-variable sums instead of a gather of z over
                                  each variable's column.  Faster on large graphs, but
                                  the sums' order, and so the last bits of h and the
                                  iterates, vary from run to run.  0 (default): the
                                  deterministic gather                                     */
    int32_t dv_scatter;        /* covering side given as an explicit CSR (dominating set,
                                  generalized matching): 1 computes dz = C d by a scatter
                                  over the columns of the variables with d_i > 0 (atomic
                                  adds, then the row scaling) instead of the row-wise
                                  SpMV: late in a probe few variables move, and only
                                  their columns are read.  Not bit-reproducible; 0
                                  (default): the SpMV                                       */
    int32_t col_split;         /* covering side of edge rows (MWU_MAT_INCIDENCE_T, vertex
                                  cover) without row bounds, edges sorted by first
                                  endpoint, h_scatter off: 0 (default) keeps z_e = x_u +
                                  x_v exactly (the update rebuilds z from the updated x)
                                  and computes h_i, the sum over the edges at i of
                                  e^{-eta (z_e - s_c)}, from two contiguous streams -- z
                                  over the edges whose first endpoint is i, and x_i + x_u
                                  over a list of the first endpoints u of the edges whose
                                  second endpoint is i (one gather of x each) -- with no
                                  atomics (deterministic); columns longer than 256
                                  entries are summed in 256-entry segments.  -1 keeps z
                                  incremental (z += alpha dz, Alg. 2) and gathers z over
                                  every vertex's incident edge ids                      */
    int32_t batch_cluster;     /* mwu_solve_batch with batch_workers 256 or 512: blocks per
                                  thread-block cluster, 1 (or 0, the default), 4, 8 or 16
                                  (16 where the device allows clusters beyond the portable
                                  8).  With more than 1, every instance of at least
                                  batch_cluster_edges edges is solved by a whole cluster
                                  (its sums combined across the cluster's blocks in a fixed
                                  order), the others by one block.  Ignored when
                                  batch_workers = 0 (autotuned)                            */
    int32_t batch_cluster_edges; /* smallest instance (edges) a cluster solves; 0 (default)
                                  = 2 x threads per block x blocks per cluster             */
} mwu_options;

/* Fill *opt with the defaults above.  Returns MWU_OK or MWU_ERR_INVALID (opt == NULL). */
int mwu_default_options(mwu_options *opt);

/* ------------------------------------------------------------ statistics */
typedef struct {
    int32_t status;            /* mwu_status of the probe (RUNNING if not ended)             */
    int32_t reason;            /* MWU_REASON_*                                                */
    int32_t iters;             /* MWU iterations of the current probe                        */
    int32_t last_passes;       /* candidate passes of the last iteration                     */
    int64_t evals;             /* f(alpha) evaluations of the current probe                  */
    int64_t passes;            /* candidate passes of the current probe                      */
    double alpha;              /* last accepted step size                                    */
    double ymax, zmin;         /* max(Px), min(Cx) at the current x                          */
} mwu_iter_stats;

typedef struct {
    int32_t status;            /* MWU_OK, or an error                                        */
    double objective;          /* best certified objective (c^T x / max(Px), c^T x / min(Cx),
                                  or max(Oz)/min(Wz)) over all probes                        */
    double lo, hi;             /* final bracket of the search on M or D                      */
    int32_t probes;            /* feasibility probes run                                     */
    int64_t iters;             /* MWU iterations over all probes                             */
    int64_t evals;             /* f(alpha) evaluations over all probes                       */
    int64_t passes;            /* candidate passes over all probes                           */
    double seconds;            /* wall time of the solve                                     */
    int64_t launches;          /* kernels launched by the solve (graph nodes counted)        */
} mwu_result;

/* Per-kernel-class device time of the iterations run with opt.timing = 1,
 * from CUDA events recorded on the context's stream inside the captured
 * iteration (FP32 form) or around the launches (FP64 form). */
typedef struct {
    double dir_ms;             /* gradient + direction kernel (with the deferred x update)   */
    double spmv_ms;            /* forward SpMV dy = Pd, dz = Cd                              */
    double cand_ms;            /* step-size search: all candidate passes of the iteration    */
    double update_ms;          /* y, z update with the next iteration's reductions           */
    int64_t iters;             /* iterations timed                                           */
    int64_t cand_passes;       /* candidate passes that evaluated candidates                 */
    int64_t compactions;       /* active-row compactions (drop_covered = 1, split view)      */
} mwu_timing;

typedef struct {
    double eta, c_d, eps, target;
    double s_p, S_p, s_c, S_c; /* LSE shifts (max y, min z) and shifted sums                  */
    double ymax, zmin;
    double alpha;              /* last accepted (or searched) alpha                          */
    int64_t n_positive;        /* |{i : d_i > 0}| of the last direction                      */
    int64_t n, m_P, m_C;       /* variables, packing rows, covering rows (objective row incl.)*/
    int32_t K, iters;
} mwu_scalars;

/* Vectors readable with mwu_get_vector. */
enum { MWU_VEC_X = 0, MWU_VEC_Y = 1, MWU_VEC_Z = 2, MWU_VEC_D = 3, MWU_VEC_DY = 4,
       MWU_VEC_DZ = 5, MWU_VEC_G = 6, MWU_VEC_H = 7 };

typedef struct mwu_ctx mwu_ctx;

/* ------------------------------------------------------------ lifecycle */
/* Build a solver context.  Matrices follow the paper's normalisation (Sec. 2.2):
 *   PACKING : P = the constraint matrix (CSR, INCIDENCE, ...), C kind NONE;
 *             objective_c (n floats, NULL = ones) becomes the covering row.
 *   COVERING: C = the constraint matrix, P kind NONE; objective_c becomes the packing row.
 *   MIXED   : both P and C given, objective_c ignored.
 *   DENSEST : P must be MWU_MAT_PAIR and C MWU_MAT_INTERWEAVE over the same edge list.
 * Input arrays are validated on the device (monotone rowptr, indices in range,
 * values finite and >= 0, bounds > 0, covering rows non-empty); a violation
 * returns MWU_ERR_INVALID.  The context owns every device buffer it allocates;
 * release it with mwu_destroy.  *out is NULL on failure. */
int mwu_create(int32_t kind, const mwu_matrix *P, const mwu_matrix *C,
               const float *objective_c, const mwu_options *opt, mwu_ctx **out);

/* Release a context and its device memory.  NULL is ignored. */
void mwu_destroy(mwu_ctx *ctx);

/* Message of the last error of ctx (or of the last failed mwu_create when ctx is NULL). */
const char *mwu_last_error(const mwu_ctx *ctx);

/* -------------------------------------------------------- one probe (Alg. 2) */
/* Fix the probe target (M for PACKING/COVERING, D for DENSEST; ignored for
 * MIXED) and reset the probe: eta = eta_factor ln(m_P+m_C)/eps, x_i = eps/(n
 * ||P_{:,i}||_inf), y = Px, z = Cx and their LSE reductions (Alg. 2 init). */
int mwu_set_target(mwu_ctx *ctx, double target);

/* Replace x (n entries, host or device, float32 or float64 per x_is_fp64) and
 * recompute y = Px, z = Cx and their reductions.  Keeps eta and the target.
 * MWU_ERR_NUMERIC when the reductions are not finite (an x so large that Px
 * or Cx overflows the form's precision). */
int mwu_set_x(mwu_ctx *ctx, const void *x, int32_t x_is_fp64);

/* Stage hooks that load the constraint vectors themselves, so that each kernel
 * of an iteration can be checked on inputs identical to a reference's rather
 * than on values that earlier kernels produced.
 *
 * mwu_set_state loads y (m_P entries), z (m_C entries), dy, dz (host or device
 * arrays, float32 or float64 per is_fp64; NULL leaves that vector as it is;
 * a side that is the single objective row takes one entry).  Values are
 * rounded once to the form's precision.  When y or z is given, the probe is
 * reset to RUNNING (eta, the target and x are kept) and the log-sum-exp
 * reductions of Sec. 2.2 (shifts s_p = max y, s_c = min z and the shifted sums
 * S_p, S_c, read with mwu_get_scalars) are recomputed by the reduction kernel,
 * followed by Alg. 2's stopping test; mwu_direction then computes g, h, d from
 * these y, z and the current x.  When dy or dz is given, mwu_eval_candidates,
 * mwu_eval_newton and mwu_search use them as the last direction's products
 * (Sec. 4.1 / 4.2).  MWU_ERR_INVALID when a loaded value is negative, NaN or
 * infinite; MWU_ERR_NUMERIC when a reduction is not finite.
 *
 * mwu_set_direction loads d (n entries, same conventions) and computes
 * dy = Pd, dz = Cd with the forward products of the iteration (a6 of Alg. 2:
 * the row-binned or staged SpMV, or the column scatter with dv_scatter); read
 * them with mwu_get_vector.  Requires a running probe (MWU_ERR_STATE). */
int mwu_set_state(mwu_ctx *ctx, const void *y, const void *z, const void *dy, const void *dz, int32_t is_fp64);
int mwu_set_direction(mwu_ctx *ctx, const void *d, int32_t is_fp64);

/* Run up to n_iters iterations of Alg. 2 (gradients, direction, d = 0 test,
 * dy = Pd, dz = Cd, step-size search, update, stopping test).  Returns the
 * probe status: FEASIBLE, INFEASIBLE, MAX_ITER or RUNNING; or an error.
 * stats may be NULL. */
int mwu_iterate(mwu_ctx *ctx, int32_t n_iters, mwu_iter_stats *stats);

/* Stage hooks of one iteration, for checking each step against a reference:
 * mwu_direction computes g, h, d (Alg. 2, gradient and direction lines) and
 * dy = Pd, dz = Cd at the current x without taking a step; it returns
 * MWU_INFEASIBLE when d = 0.  *n_positive may be NULL. */
int mwu_direction(mwu_ctx *ctx, int64_t *n_positive);

/* Evaluate K <= 8 step candidates on the stored y, dy, z, dz of the last
 * mwu_direction (Sec. 4.1): psi[k] = smax(y + a_k dy) - smax(y),
 * phi[k] = smin(z + a_k dz) - smin(z), zmin[k] = min(z + a_k dz).
 * Host arrays of K doubles; any output may be NULL. */
int mwu_eval_candidates(mwu_ctx *ctx, const double *alphas, int32_t K,
                        double *psi, double *phi, double *zmin);

/* Newton quantities of the last direction at one step size (Sec. 4.2):
 * out[0] = Psi(alpha), out[1] = Phi(alpha), out[2] = Psi'(alpha) =
 * <dy, e^{eta(y + alpha dy)}>/<1, e^{eta(y + alpha dy)}>, out[3] = Phi'(alpha) =
 * <dz, e^{-eta(z + alpha dz)}>/<1, e^{-eta(z + alpha dz)}>.  out: host array of
 * 4 doubles.  Requires mwu_direction; MWU_ERR_NUMERIC on NaN/Inf. */
int mwu_eval_newton(mwu_ctx *ctx, double alpha, double *out);

/* Run the configured step-size search (Alg. 3 / K-candidate form / Newton)
 * on the last direction without updating x.  *alpha < 1 means INFEASIBLE. */
int mwu_search(mwu_ctx *ctx, double *alpha, int64_t *evals);

/* ------------------------------------------------------- the whole solve */
/* Bisect on M (or D) between lo and hi (<= 0: the automatic bracket of Sec.
 * 2.2 / Sec. 3) until hi <= (1+outer_tol) lo, one probe per midpoint, and
 * report the best certified objective.  MIXED runs a single probe.  The
 * automatic bracket is computed by the first mwu_solve of a context and
 * reused: a caller that rewrites the objective or the matrix values in place
 * passes lo and hi itself. */
int mwu_solve(mwu_ctx *ctx, double lo, double hi, mwu_result *res);

/* --------------------------------------------------------- read back */
/* Copy vector `which` (MWU_VEC_*) into dst (host or device), n entries, as
 * float64 when as_fp64 else float32.  n must equal the vector's length.
 * MWU_VEC_X after mwu_solve is the best probe's x. */
int mwu_get_vector(mwu_ctx *ctx, int32_t which, void *dst, int64_t n, int32_t as_fp64);

/* Copy the current scalars. */
int mwu_get_scalars(mwu_ctx *ctx, mwu_scalars *out);

/* Accumulated per-kernel-class times (see mwu_timing); reset != 0 clears them.
 * A batch context has no per-class times (its solve is one kernel). */
int mwu_get_timing(mwu_ctx *ctx, mwu_timing *out, int32_t reset);

/* Tiles of the staged forward SpMV of each side (opt.spmv_tiles): *tiles_p and
 * *tiles_c (host, may be NULL) receive the number of row tiles of P and C, 0
 * where the side uses the row-binned kernel (or has no CSR rows). */
int mwu_spmv_tiles(mwu_ctx *ctx, int32_t *tiles_p, int32_t *tiles_c);

/* --------------------------------------- smoothed potential (autograd) */
/* pot = smax_eta(P x) - smin_eta(C x) at the given x (device, n float32) with
 * the context's eta (set by mwu_set_target), and its gradients (device
 * float32 outputs, each may be NULL):
 *   grad_x[i]      = (P^T nabla smax(Px) - C^T nabla smin(Cx))_i   (= g - h)
 *   grad_obj[i]    = d pot / d c_i for the objective row (1/M) c^T
 *                    (+w x_i/M on the packing side, -w x_i/M on the covering side)
 *   grad_vals[k]   = d pot / d val[k] for the k-th stored value of the
 *                    explicit CSR matrix (sign +w_j x_i for P, -w_j x_i for C).
 * Sec. 4.1 defines the potential (its 1/eta factor is left out here).  It
 * takes every covering row, also with drop_covered set; the context's state is
 * left at x with its reductions over the active rows. */
int mwu_potential(mwu_ctx *ctx, const float *x, double *pot,
                  float *grad_x, float *grad_obj, float *grad_vals);

/* Whether objective (n floats, NULL = not checked) and vals (the stored
 * values of the explicit CSR sides, packing side first, NULL = not checked)
 * equal, bit for bit, the copies the context made at mwu_create (a side or
 * objective given as NULL there counts as all ones).  *same = 1 or 0.  The
 * autograd wrapper refuses tensors that differ: the gradients refer to the
 * context's copies. */
int mwu_check_values(mwu_ctx *ctx, const float *objective, const float *vals, int32_t *same);

/* ------------------------------------------- allocation-free evaluation */
/* For callers that must not allocate device memory: code that runs inside a
 * custom device allocator's own hooks (an allocation from there would re-enter
 * the allocator), processes whose device memory a framework's caching
 * allocator has already reserved up to a fixed budget, and latency-critical
 * runtimes that forbid cudaMalloc after start-up because it synchronises the
 * device.  This entry point evaluates step-size candidates of one constraint
 * side without a context and without allocating anything: it calls no
 * cudaMalloc, cudaFree or allocating library routine.  The paper has no
 * counterpart to it; it computes the same values as mwu_eval_candidates.
 *
 *   v, dv   : device float32 arrays of m rows (y and dy of a packing side,
 *             sign = +1, or z and dz of a covering side, sign = -1)
 *   shift, S: that side's log-sum-exp shift (max v for sign +1, min v for
 *             sign -1) and shifted sum, as mwu_get_scalars reports them
 *   eta     : the smoothing parameter
 *   alphas  : host array of K (1..8) candidate step sizes
 *   val     : host output, K doubles: Psi(alpha_k) = smax(v + a dv) - smax(v)
 *             for sign +1, Phi(alpha_k) = smin(v + a dv) - smin(v) for -1
 *   vmin    : host output or NULL, K doubles: min(v + alpha_k dv) for
 *             sign = -1 (the covering side's minimum, Alg. 3's early-exit
 *             test); +inf for sign = +1
 *   stream  : cudaStream_t or NULL (legacy default stream); the call waits
 *             for its results (cudaStreamSynchronize on that stream)
 * Scratch lives in one file-scope static device array of
 * MWU_STATIC_MAX_BLOCKS per-block records (256 KiB) that every GPU loading the
 * library keeps until the process exits; m is limited to MWU_STATIC_MAX_ROWS
 * (blocks x rows per block) and larger m returns MWU_ERR_INVALID.  The first
 * call on each device does a one-time set-up with that device current: it
 * looks up the array's device address (cudaGetSymbolAddress) and clears its
 * completion ticket; make that first call before any stream capture.  Every
 * call shares the array and leaves the last call's records in it (the ticket
 * returns to zero at the end of each call), so calls that overlap on the GPU
 * (several streams or host threads at once) race and must be serialised by
 * the caller.  Errors: MWU_ERR_INVALID (bad argument, size beyond the
 * maximum), MWU_ERR_CUDA; mwu_last_error(NULL) describes them. */
#define MWU_STATIC_MAX_BLOCKS 1024
#define MWU_STATIC_ROWS_PER_BLOCK 16384
#define MWU_STATIC_MAX_ROWS ((int64_t)MWU_STATIC_MAX_BLOCKS * MWU_STATIC_ROWS_PER_BLOCK)
int mwu_candidates_static(const float *v, const float *dv, int64_t m, int32_t sign, double eta,
                          double shift, double S, const double *alphas, int32_t K,
                          double *val, double *vmin, void *stream);

/* ------------------------------------------------------------- batched */
/* Many independent b-matching LPs (Appendix A.1 with lb = 0: max 1^T x,
 * diag(1/b) M x <= 1, M the vertex-edge incidence) in one context.  P[k] is
 * instance k's MWU_MAT_INCIDENCE edge list (host or device) with optional
 * row_bound b (capacities > 0); the objective rows are ones.  The instances
 * are packed into one set of device arrays (the vertex -> incident-edge lists
 * built with a stable radix sort).  Options: eps, eta_factor, max_iter,
 * outer_tol, max_probes, max_passes, K, grad_tol, warm_start, step
 * (MWU_STEP_KARY or MWU_STEP_NEWTON), max_newton and newton_tol as for one
 * instance (FP32 vectors with FP64 reductions); batch_workers and
 * batch_cluster select the block and cluster size.  MWU_ERR_INVALID for other
 * matrix kinds, an empty instance, a bad endpoint or bound, or a bad block or
 * cluster size. */
int mwu_create_batch(int32_t count, const mwu_matrix *P, const mwu_options *opt,
                     mwu_ctx **out);

/* Solve every instance of a batch context in one persistent launch (captured
 * in a CUDA graph with the reset of its work queue).  With clusters, each
 * cluster first takes the next large instance, largest first, and its blocks
 * solve it together; then each block takes the next remaining instance and
 * solves it alone.  A solve is the whole of Sec. 2.2's outer search -- the
 * automatic bracket and the geometric bisection on M, and per probe the
 * iterations of Alg. 2 with the configured step search -- with no host round
 * trip.  Every sum of an instance runs in a fixed order, so its certified
 * objective does not depend on the batch or the schedule (only on the block
 * size and on the cluster size when a cluster solves it).  objective / iters:
 * host arrays of `count` entries or NULL; total: the sums (objective, probes,
 * iters, evals, passes) and the wall time.  The first call of a context with
 * batch_workers = 0 runs the autotuner first (one extra whole-batch solve per
 * configuration).  Not safe for concurrent use of one context. */
int mwu_solve_batch(mwu_ctx *ctx, double *objective, int64_t *iters, mwu_result *total);

/* The autotuner's choice (threads per block and blocks per cluster, both 0
 * before the first solve of an autotuned context) and its timings:
 * ms[0 .. MWU_BATCH_TUNE_CONFIGS) = milliseconds of the whole batch in the
 * configurations (threads, cluster) = (256, 1), (512, 1), (1024, 1),
 * (256, 4), (512, 4), (256, 8), (512, 8), (256, 16), (512, 16), in this order
 * (0 where not timed: a context with fixed batch_workers, or a cluster size
 * the device cannot hold).  Any output may be NULL. */
#define MWU_BATCH_TUNE_CONFIGS 9
int mwu_batch_tuning(mwu_ctx *ctx, int32_t *threads, int32_t *cluster, double *ms);

/* Per-instance candidate passes and probes of the last mwu_solve_batch (host
 * arrays of `count` entries, either NULL).  MWU_ERR_STATE before a solve. */
int mwu_batch_stats(mwu_ctx *ctx, int64_t *passes, int32_t *probes);

/* Per-instance start and end of its solve in the last mwu_solve_batch, in
 * milliseconds after the earliest start (the device's global timer): shows
 * which instance ends last and sets the batch time.  A diagnostic of this
 * library with no counterpart in the paper.  Host arrays of `count` entries,
 * either NULL.  MWU_ERR_INVALID for a context that is not a batch,
 * MWU_ERR_STATE before a solve. */
int mwu_batch_timeline(mwu_ctx *ctx, double *start_ms, double *end_ms);

/* ------------------------------------------------------------ diagnostics */
/* u[i] = 1 - e^{-b[i]} for b[i] >= 0, by the same device function the
 * candidate passes use (FP32).  b, u: device arrays of n floats; stream:
 * cudaStream_t or NULL; the call waits for the result.  MWU_ERR_INVALID on
 * NULL arrays or n < 0, MWU_ERR_CUDA on a launch error. */
int mwu_diag_one_minus_exp_neg(const float *b, float *u, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MWU_H_ */
