// Internal declarations shared by the translation units of libmwu.
//
// Data layout in HBM (one context):
//   variables : x[n], d[n] (and g[n], h[n] when kept for inspection), type T
//   side P    : y[m_P], dy[m_P]  (absent when P is the single objective row)
//   side C    : z[m_C], dz[m_C]  (absent when C is the single objective row)
//   structure : each side has a row view (for A x, rows j) and a column view
//               (for A^T w, one "row" per variable i listing the rows j with
//               A_ji != 0).  Implicit graph matrices (Sec. 5.1.2) keep only an
//               int32 edge list and a vertex -> slot CSR.
//   scalars   : DevState (FP64 shifts/sums, search state, status) in device memory
//   partials  : per-block FP64 records merged by the last block of each kernel
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mwu {

constexpr int KMAX = 8;           // candidates per pass (compile-time bound)
constexpr int BLOCK = 256;        // threads per block of the sweep kernels
constexpr int REC = 72;           // doubles per per-block partial record

// Row views (constraint rows of one side, for y = A x).
enum RowKind : int32_t {
    RK_NONE = 0,
    RK_CSR = 1,      // ptr/idx/val; val == nullptr -> ones
    RK_FIXED2 = 2,   // row j = edge (u,v): x[u] + x[v]; idx = int2 edge list
    RK_PAIRSUM = 3,  // row j: x[2j] + x[2j+1] (interweaved identity W)
    RK_DENSE1 = 4    // the single objective row c^T x (a reduction over variables)
};

// Column views (for A^T w: per variable i, the rows j holding it).
enum ColKind : int32_t {
    CK_NONE = 0,
    CK_CSR = 1,      // ptr/idx/val over variables, idx = row j
    CK_FIXED2 = 2,   // variable i = edge (u,v): rows u and v (incidence M)
    CK_FIXED1 = 3,   // variable i = slot: row idx[i] (pair matrix O)
    CK_HALF1 = 4,    // variable i = slot: row i/2 (interweaved W)
    CK_DENSE1 = 5,   // single objective row: coefficient c[i]
    CK_SPLIT2 = 6    // incidence transpose with edges sorted by first endpoint: variable i
                     // = vertex; its edges with first endpoint i are the contiguous rows
                     // [ptr[i] - ptr2[i], ptr[i+1] - ptr2[i+1]) (weights from the stored
                     // z), those with second endpoint i are listed through their first
                     // endpoints idx2[ptr2[i] .. ptr2[i+1]) (weights from x_i + x_u, equal
                     // to the stored z_e since that side keeps z = x_u + x_v exactly)
};

struct RowView {
    int32_t kind;
    int32_t G;            // lanes per CSR row (power of two <= 32)
    int64_t rows;
    int64_t nnz;          // stored entries (CSR), 2 rows (FIXED2 / PAIRSUM), 0 (DENSE1)
    const int32_t *ptr;   // CSR row pointer (rows+1)
    const int32_t *idx;   // CSR column index / FIXED2 edge pairs
    const float *val;     // CSR values or nullptr
    const float *rdiv;    // row divisor b_j (bounds) or nullptr
    // length bins of the rows for the forward SpMV (CSR only): short rows
    // (<= SHORT_LEN) one thread each, medium (<= MED_LEN) MED_LANES lanes each,
    // long rows cut into segments of SEG_LEN entries, one warp per segment, whose
    // partial sums the last block adds up per row in order
    int32_t n_short = 0, n_med = 0;
    const int32_t *short_rows = nullptr, *med_rows = nullptr;
    int32_t n_seg = 0, n_long = 0;
    const int32_t *seg_row = nullptr, *seg_beg = nullptr;     // per segment: its row and first entry
    const int32_t *long_rows = nullptr, *long_seg = nullptr;  // per long row: row id; segments [long_seg[i], long_seg[i+1])
    // staged SpMV (banded matrices): tiles of tile_rows consecutive rows whose
    // entries' columns span [tile_lo[t], tile_lo[t] + tile_len[t]); a tile
    // with a span of at most tile_wmax<T>() reads its input window from shared
    // memory.  n_tiles > 0 selects the staged SpMV for this side.
    int32_t n_tiles = 0, tile_rows = 0;
    const int32_t *tile_lo = nullptr, *tile_len = nullptr;
};

constexpr int TILE_SMEM = 48 * 1024;   // shared memory of one tile's input window
constexpr int HEAVY_LEN = 4096;        // columns longer than this take a whole block in the direction kernel
template <class T> constexpr int tile_wmax() { return TILE_SMEM / (int)sizeof(T); }

// split view (CK_SPLIT2): columns longer than SPLIT_HEAVY entries go through
// the segment pre-pass in SPLIT_SEG-entry pieces (one warp each)
constexpr int SPLIT_HEAVY = 256;
constexpr int SPLIT_SEG = 256;
constexpr int SPLIT_TINY = 8;
constexpr int SHORT_LEN = 16;
constexpr int MED_LEN = 256;
constexpr int MED_LANES = 16;
constexpr int SEG_LEN = 1024;

struct ColView {
    int32_t kind;
    int32_t G;
    const int32_t *ptr;
    const int32_t *idx;   // CSR: row ids ; FIXED2: edge pairs ; FIXED1: row per variable
    const float *val;
    const float *rdiv;    // divisor of row j (same array as the side's RowView)
    const float *cvec;    // DENSE1 objective values (nullptr -> ones)
    int32_t n_heavy;
    int32_t heavy_len;
    const int32_t *heavy;
    // CK_SPLIT2: ptr holds the combined column lengths (first-endpoint range
    // plus second-endpoint list), ptr2/idx2 the second-endpoint lists, xsrc
    // the variables x (type T of the problem)
    const int32_t *ptr2 = nullptr;
    const int32_t *idx2 = nullptr;
    const void *xsrc = nullptr;
    // CK_SPLIT2 columns of the problem's heavy variables (heavy_var, longer than
    // SPLIT_HEAVY) cut into SPLIT_SEG-entry segments of the combined column:
    // heavy variable h owns segments [cseg_first[h], cseg_first[h+1]), segment q
    // covers combined entries [cseg_beg[q], min(cseg_beg[q] + SPLIT_SEG,
    // ptr[cseg_var[q] + 1])); k_split_seg writes one partial sum per segment
    int32_t n_cseg = 0;
    const int32_t *cseg_first = nullptr, *cseg_var = nullptr, *cseg_beg = nullptr;
};

template <class T>
struct Side {
    RowView rv;
    ColView cv;
    int32_t sign;    // +1 packing (smax), -1 covering (smin)
    int64_t m;       // rows (1 for the objective row)
    T *v;            // y or z (nullptr for DENSE1)
    T *dv;           // dy or dz
    T *seg_part;     // per-segment partial sums of long CSR rows
    // compacted covering side (drop_covered on the vertex-cover split view):
    // rows j < m are the active edges, orig[j] their row in the full edge
    // list, vfull the full z that the direction's split view reads (the update
    // writes vfull[orig[j]] = v[j]; the rows dropped earlier keep their last
    // value, >= 1).  nullptr when the side is not compacted.
    const int32_t *orig = nullptr;
    T *vfull = nullptr;
};

// Probe status values stored on the device.
enum : int32_t { ST_FEASIBLE = 0, ST_INFEASIBLE = 1, ST_MAX_ITER = 2, ST_RUNNING = 3, ST_NUMERIC = -4,
                 ST_TIMEOUT = -5 };   // a bounded device-side loop gave up
enum : int32_t { RS_NONE = 0, RS_COVERED = 1, RS_PACKING = 2, RS_DZERO = 3, RS_ALPHA = 4, RS_MAXITER = 5,
                 RS_RATIO = 6 };

// Search phases.
// PH_COVER: a passing Newton value covered every row; one pass computes the
// smallest covering step alpha_c and the search ends with max(1, min(alpha, alpha_c)).
enum : int32_t { PH_EXP = 0, PH_REFINE = 1, PH_DONE = 2, PH_NEWTON = 3, PH_BACKOFF = 4, PH_COVER = 5 };

struct DevState {
    // problem scalars
    double eta, eps, c_d, target;
    double scale[2];            // side factors: 1/M (objective row), 1/D (O), else 1
    int32_t max_iter, K, max_passes, warm_start;
    int32_t step_mode;          // 0 kary, 1 binary (K=1 semantics), 2 standard, 3 newton
    int32_t stop_rule;          // 1: stop FEASIBLE once ymax <= (1+eps) zmin
    double grad_tol;            // gradient test: d_i > 0 iff g_i < (1 - grad_tol) h_i
    double ratio_stop;          // > 0: stop FEASIBLE once ymax <= ratio_stop * zmin
    // reductions of the current y, z (side 0 = P, side 1 = C)
    double s[2], S[2];
    double lnS[2], invS[2];     // ln S (in the candidate passes' precision) and 1/S, set with S
    double inv_eta;             // 1/eta, set with eta
    double act_hi;              // covering rows with z_j >= act_hi are dropped (1: drop_covered, +inf: kept)
    double dense_v[2], dense_dv[2];   // single objective row value and direction
    double ymax, zmin;
    // direction
    long long n_pos;
    // search
    int32_t phase, b, passes, early;
    int32_t kpass;              // candidates of the next pass (1 for a Newton pass)
    int32_t deriv;              // external pass: also return Psi'(alpha_0), Phi'(alpha_0)
    int32_t max_newton, newton_steps;
    double newton_tol;
    double bo_cur;              // backoff: last value alpha (1 - eps)^p handed out
    double dpsi, dphi;          // Psi'(alpha_0), Phi'(alpha_0) of the last Newton pass
    int32_t loop_guard;         // passes run by the device-side search loop of this iteration
    int32_t guard_limit;        // turns after which that loop gives up (ST_TIMEOUT); max_passes + 4
    long long loop_launches;    // kernels run inside the device-side search loops (all iterations)
    double lb, ub;
    double alpha[KMAX];
    double psi[KMAX], phi[KMAX], zmink[KMAX];
    int32_t okk[KMAX];
    double alpha_acc;           // accepted alpha of this iteration (0 if none)
    double alpha_prev;
    int32_t pending;            // x += alpha_acc * d not yet applied
    int32_t last_passes;
    // status
    int32_t status, reason, iter, numeric_bad;
    long long evals, total_passes;
    // last-block-done counters
    unsigned int counter[8];
};

template <class T>
struct Problem {
    Side<T> side[2];
    int64_t n;          // variables
    T *x, *d, *g, *h;   // g, h may be nullptr (not kept)
    T *hacc;            // per-variable sums of k_h_scatter (option h_scatter), else nullptr
    T *cseg_part;       // per-segment partial sums of the heavy CK_SPLIT2 columns (k_split_seg)
    int32_t dv_scatter; // bit s: side s computes dv = A d by scatter (option dv_scatter)
    int32_t x_eager;    // x += alpha d runs before the update (which then rebuilds the edge
                        // rows of a CK_SPLIT2 side as z_e = x_u + x_v), not in the next k_dir
    DevState *st;
    double *part_var;   // per-block records of variable-side kernels
    double *part_row;   // per-block records of row-side kernels
    int32_t grid_var, grid_row;   // grid sizes (blocks): variable kernels, candidate passes
    int32_t grid_upd;             // grid of the update kernel
    int32_t grid_spmv;            // grid of the forward SpMV (its own occupancy)
    int32_t grid_newton;          // grid of the one-candidate Newton pass (its own occupancy)
    int32_t grid_tiled;           // grid of the staged SpMV (its own occupancy)
    // a captured iteration: the handle of its step-search WHILE loop, which the
    // direction kernel opens and every turn of the loop sets (0 = not captured),
    // and the handle of the IF node inside the loop body that runs the
    // K-candidate pass only in the turns whose phase needs it
    int32_t cond_on;
    cudaGraphConditionalHandle cond;
    cudaGraphConditionalHandle cond_kc;
    // variables of CSR column views by column length (the longer of the two
    // sides): light ones (<= the views' heavy_len) take G_var lanes in the
    // main loop, medium ones (<= HEAVY_LEN) a warp each, heavy ones a block each
    int32_t G_var;
    int32_t n_heavy_var;
    const int32_t *heavy_var;
    int32_t n_med_var;
    const int32_t *med_var;
    // split view only (n_light_var >= 0): the variables with at most
    // SPLIT_TINY combined column entries take one thread each (tiny_var), the
    // other light ones G_var lanes each (light_var); -1: every variable is
    // visited by the G_var-lane loop
    int32_t n_tiny_var;
    const int32_t *tiny_var;
    int32_t n_light_var;
    const int32_t *light_var;
};

// ---------------------------------------------------------------- launchers
// (implemented in mwu_kernels.cu for T = float and T = double)
template <class T> cudaError_t launch_x_init(const Problem<T> &p, cudaStream_t s);                // a0: x0 + dense dots
template <class T> cudaError_t launch_x_set(const Problem<T> &p, const void *x, int fp64, cudaStream_t s);
template <class T> cudaError_t launch_rows_eval(const Problem<T> &p, cudaStream_t s);             // a1-a3 at a new x
// a2, a3 of the stored y, z (loaded by the stage hook), dense rows as the state holds them
template <class T> cudaError_t launch_rows_reduce(const Problem<T> &p, cudaStream_t s);
// single objective row applied to d (dense_dv), for a direction loaded by the stage hook
template <class T> cudaError_t launch_dense_dir(const Problem<T> &p, cudaStream_t s);
template <class T> cudaError_t launch_dir(const Problem<T> &p, int keep_gh, cudaStream_t s);      // a4-a5 (+ fused x update)
// a6: dy = Pd, dz = Cd; skip_c: dz was already written by the direction kernel
template <class T> cudaError_t launch_spmv(const Problem<T> &p, cudaStream_t s, int skip_c = 0);
// true when launch_dir(p, keep_gh) runs the edge-pair direction kernel, which also writes dz = Wd
template <class T> bool dir_fuses_dz(const Problem<T> &p, int keep_gh) {
    return !keep_gh && p.side[0].cv.kind == CK_FIXED1 && p.side[1].cv.kind == CK_HALF1 &&
           p.side[1].rv.kind == RK_PAIRSUM;
}
template <class T> cudaError_t launch_cand(const Problem<T> &p, int external, cudaStream_t s);
// a6 for a CSR side by scatter over the columns of the variables with d > 0 (option dv_scatter)
template <class T> cudaError_t launch_spmv_scatter(const Problem<T> &p, int side, cudaStream_t s);
// one-candidate Newton pass (captured iterations): returns at once unless the search is in its Newton phase
template <class T> cudaError_t launch_cand_newton(const Problem<T> &p, cudaStream_t s);    // a7: one candidate pass
template <class T> cudaError_t launch_update(const Problem<T> &p, cudaStream_t s);                // a8
template <class T> cudaError_t launch_flush(const Problem<T> &p, cudaStream_t s);                 // pending x update
template <class T> cudaError_t launch_search_begin(const Problem<T> &p, cudaStream_t s);
template <class T> cudaError_t launch_potential_grads(const Problem<T> &p, const float *x, float *gx, float *gobj,
                                                      float *gvals_p, float *gvals_c, cudaStream_t s);
template <class T> cudaError_t launch_copy_vec(const T *src, void *dst, int64_t n, int fp64, cudaStream_t s);
// *bad |= 1 if some v[i] is negative, NaN or infinite
template <class T> cudaError_t launch_check_nonneg(const T *v, int64_t n, int *bad, cudaStream_t s);
// *differ |= 1 if a (nullptr = ones) and b (device arrays of n floats) differ bitwise
cudaError_t launch_same_f32(const float *a, const float *b, int64_t n, int *differ, cudaStream_t s);
// dst[i] = (T) src[i] (device arrays)
template <class T, class U> cudaError_t launch_convert_in(const U *src, T *dst, int64_t n, cudaStream_t s);

// Packed batch of b-matching instances for the persistent solve (k_batch_solve):
// instance k owns edges [eoff[k], eoff[k+1]) (int2 (u, v), local vertex ids),
// vertices [voff[k], voff[k+1]), its vertex -> incident-edge lists at
// vptr[voff[k] + k .. voff[k+1] + k] (local offsets into eids + 2 eoff[k]).
struct BatchDesc {
    int32_t count;
    const int32_t *order;      // instances in decreasing edge count (the work queue's order)
    const int64_t *eoff, *voff;
    const int32_t *edges;
    const float *bound;        // capacity per vertex, or nullptr (all 1)
    const int32_t *vptr, *eids;
    float *x, *d, *y, *dy;     // per edge (x, d) and per vertex (y, dy)
    double *obj;
    int64_t *iters, *evals, *passes;
    int32_t *probes;
    unsigned int *queue;       // next instance to take: [0] cluster-solved, [1] block-solved
    int32_t n_cluster;         // order[0 .. n_cluster) are solved by whole clusters (set per launch)
    int64_t *t_beg, *t_end;    // per instance: %globaltimer (ns) at the start and end of its solve
    double eps, eta_factor, outer_tol, grad_tol, newton_tol;
    int32_t max_iter, max_probes, max_passes, K, warm_start;
    int32_t step_mode;         // 0 K-candidate search, 3 Newton (Sec. 4.2)
    int32_t max_newton;
};
// nt threads per block, cl blocks per cluster (1, 4, 8 or 16 with nt 256 or
// 512; 1 with 1024); the first n_cluster instances of the order are solved by whole
// clusters.  batch_blocks: the persistent grid (all blocks resident), 0 if the
// configuration cannot run.
cudaError_t launch_batch_solve(const BatchDesc &B, int nt, int cl, int n_cluster, int blocks, cudaStream_t s);
int batch_blocks(int nt, int cl, int n_sms);

// Message for mwu_last_error(NULL) from entry points without a context.
void set_global_error(const char *msg);

// Kernel occupancy helper (blocks per SM of the heaviest sweep kernel).
template <class T> int sweep_blocks_per_sm(int *var_bps, int *row_bps, int *upd_bps);
template <class T> int spmv_blocks_per_sm();
template <class T> int newton_blocks_per_sm();
template <class T> int tiled_blocks_per_sm();

// Stream compaction of the active covering rows (v < hi) of an edge-row side:
// per tile of CMP_TILE rows a count, one exclusive scan, then a stable
// scatter of the edge pairs, values and original row numbers (orig == nullptr:
// the rows are the full list, row j is its own original).  *total (device)
// receives the number of active rows.
constexpr int CMP_TILE = BLOCK * 8;
__host__ __device__ inline int64_t cmp_tiles(int64_t m) { return (m + CMP_TILE - 1) / CMP_TILE; }
template <class T>
cudaError_t launch_cmp_count(const T *v, int64_t m, double hi, int32_t *tile_off, int64_t *total, cudaStream_t s);
template <class T>
cudaError_t launch_cmp_scatter(const int32_t *pairs, const T *v, const int32_t *orig, int64_t m, double hi,
                               const int32_t *tile_off, int32_t *pairs_o, T *v_o, int32_t *orig_o, cudaStream_t s);
// z_e = (x_u + x_v) scale_1 over every row of the full edge-row side (the
// arithmetic of the update's rebuild)
template <class T> cudaError_t launch_cmp_refresh(const Problem<T> &p, cudaStream_t s);
}  // namespace mwu
