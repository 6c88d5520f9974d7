// C ABI of libmwu (include/mwu.h): context lifecycle, the probe driver of
// Alg. 2, the bisection on M or D (Sec. 2.2, Sec. 3), read-back, the smoothed
// potential for autograd, and the batched front end.
//
// Two execution forms share the kernels of mwu_kernels.cu:
//   F32_R64 : FP32 vectors, K candidates per pass, one iteration captured once
//             in a CUDA graph (gradient+direction, first candidate pass with
//             the forward SpMV, max_passes-1 further passes that exit at once
//             when the search is done, update); the host reads the status
//             every `check_every` iterations.
//   FP64    : the plain form: FP64 vectors, one candidate per pass (Alg. 3),
//             the host reads the search state after every pass.
#include "mwu.h"
#include "mwu_setup.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

using namespace mwu;

static thread_local std::string g_create_error;

struct mwu_ctx {
    int32_t kind = 0;
    mwu_options opt{};
    bool fp64 = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t body_stream = nullptr;      // captures the body of the device-side search loop
    cudaStream_t kc_stream = nullptr;        // captures the body of the IF node inside it
    bool bracket_ok = false;                 // automatic bracket of mwu_solve, once computed
    double bracket_lo = 0.0, bracket_hi = 0.0;
    Arena ar;
    std::string err;
    int64_t n = 0, mP = 0, mC = 0;
    Problem<float> pf{};
    Problem<double> pd{};
    DevState *st_dev = nullptr;
    DevState *st_host = nullptr;
    const float *objective = nullptr;
    cudaGraphExec_t gexec_chunk = nullptr;   // check_every iterations
    cudaGraphExec_t gexec_one = nullptr;     // one iteration
    // active-row compaction (drop_covered = 1 on the vertex-cover split view):
    // inside one mwu_iterate call the covering side's rows shrink to the
    // unsatisfied edges (two buffer sets, used in turn); the call restores
    // the full rows before it returns
    bool cmp_ok = false, cmp_on = false;
    int cmp_buf = 0;
    int32_t *cmp_pairs[2] = {nullptr, nullptr}, *cmp_orig[2] = {nullptr, nullptr};
    void *cmp_v[2] = {nullptr, nullptr};
    void *cmp_dv = nullptr;
    int32_t *cmp_tile = nullptr;
    int64_t *cmp_total = nullptr;
    Side<float> cmp_full_f{};
    Side<double> cmp_full_d{};
    cudaGraphExec_t gexec_chunk_c = nullptr, gexec_one_c = nullptr;   // graphs of the compacted rows
    std::vector<cudaEvent_t> ev;             // 4 per iteration of the chunk graph (timing)
    std::vector<cudaEvent_t> ev_one;         // 4 for the one-iteration graph
    mwu_timing tim{};
    int64_t launches = 0;
    void *x_best = nullptr;
    int n_sms = 0;
    double target = 1.0;
    bool have_direction = false;
    bool trace = false;          // MWU_TRACE=1: one line per probe on stderr
    int guard_limit = 0;         // MWU_SEARCH_GUARD=n: turns of the device-side search loop before it
                                 // gives up with MWU_ERR_TIMEOUT (default max_passes + 4; a test hook)
    // batch front end: the persistent solve of packed b-matching instances
    bool is_batch = false;
    BatchDesc bd{};
    int32_t batch_count = 0;
    int64_t batch_edges = 0;
    std::vector<int64_t> batch_e;            // edges per instance
    int batch_nt = 0;                        // threads per block in use (0 = not tuned yet)
    int batch_cl = 1;                        // blocks per cluster in use
    int batch_blocks = 0;
    double tune_ms[MWU_BATCH_TUNE_CONFIGS] = {};   // autotuner: whole-batch time per configuration
    cudaGraphExec_t batch_graph = nullptr;   // queue reset + the persistent launch
    int batch_graph_nt = 0, batch_graph_cl = 0;
    std::vector<int32_t> batch_order;        // instances in decreasing edge count
    std::vector<int64_t> batch_last_passes;  // per instance, of the last solve
    std::vector<int32_t> batch_last_probes;
    std::vector<int64_t> batch_t_beg, batch_t_end;   // per instance, %globaltimer ns of the last solve
};

// ------------------------------------------------------------ helpers
#define TRY_CUDA(ctx, expr)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) return fail_cuda((ctx), e_, #expr);                             \
    } while (0)

static int fail(mwu_ctx *c, int code, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}
static int fail_cuda(mwu_ctx *c, cudaError_t e, const char *what) {
    std::string m = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? MWU_ERR_OOM : MWU_ERR_CUDA, m);
}

template <class F> static cudaError_t with_prob(mwu_ctx *c, F f) {
    if (c->fp64) return f(c->pd);
    return f(c->pf);
}

static int pow2_floor(double v) {
    int g = 1;
    while (g * 2 <= v && g < 32) g *= 2;
    return g;
}

static int pow2_ceil(int v) {
    int g = 1;
    while (g < v && g < 32) g *= 2;
    return g;
}

static int choose_G(double avg, int forced) {
    if (forced > 0) return forced;
    int g = pow2_floor(avg) / 2;
    return std::max(1, std::min(32, g));
}


int mwu_default_options(mwu_options *o) {
    if (!o) return MWU_ERR_INVALID;
    std::memset(o, 0, sizeof(*o));
    o->eps = 0.1;
    o->max_iter = 5000;
    o->eta_factor = 10.0;
    o->step = MWU_STEP_KARY;
    o->K = 8;
    o->max_passes = 0;   // 0 -> form default
    o->warm_start = 0;
    o->double_single = 1;
    o->precision = MWU_PREC_F32_R64;
    o->outer_tol = 0.0;  // 0 -> eps
    o->max_probes = 64;
    o->use_graph = 1;
    o->check_every = 8;
    o->group = 0;
    o->max_newton = 8;
    o->newton_tol = 0.0;   // 0 -> eps / 20
    o->batch_workers = 0;  // 0 -> tuned online
    o->batch_cluster = 0;
    o->batch_cluster_edges = 0;
    o->drop_covered = 0;
    o->spmv_tiles = 0;     // automatic
    o->h_scatter = 0;
    o->dv_scatter = 0;
    o->col_split = 0;
    o->timing = 0;
    o->stop_rule = 0;
    o->grad_tol = -1.0;   // precision default
    o->stream = nullptr;
    return MWU_OK;
}

namespace mwu {
void set_global_error(const char *msg) { g_create_error = msg ? msg : ""; }
}  // namespace mwu

const char *mwu_last_error(const mwu_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

// ------------------------------------------------------------ views
struct SideBuild {
    RowView rv{};
    ColView cv{};
    int64_t m = 0;       // rows
    int64_t nvar = -1;   // variables implied by this matrix (-1: any)
    int32_t sign = 1;
    bool dense = false;
};

static const int32_t *copy_in_i(mwu_ctx *c, const int32_t *src, int64_t n) {
    int32_t *d = c->ar.alloc<int32_t>(n);
    if (!d) return nullptr;
    if (n > 0 && cudaMemcpyAsync(d, src, sizeof(int32_t) * (size_t)n, cudaMemcpyDefault, c->stream) != cudaSuccess)
        return nullptr;
    return d;
}
static const float *copy_in_f(mwu_ctx *c, const float *src, int64_t n) {
    float *d = c->ar.alloc<float>(n);
    if (!d) return nullptr;
    if (n > 0 && cudaMemcpyAsync(d, src, sizeof(float) * (size_t)n, cudaMemcpyDefault, c->stream) != cudaSuccess)
        return nullptr;
    return d;
}

static int check_err_flag(mwu_ctx *c, int *d_err) {
    int h = 0;
    TRY_CUDA(c, cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h != 0) return fail(c, MWU_ERR_INVALID, validation_message(h));
    return MWU_OK;
}

static int build_side(mwu_ctx *c, const mwu_matrix *A, int32_t sign, SideBuild &sb, int *d_err) {
    sb.sign = sign;
    cudaStream_t s = c->stream;
    const int forced_G = c->opt.group;
    if (!A) return fail(c, MWU_ERR_INVALID, "missing matrix");
    const float *rdiv = nullptr;
    auto load_bounds = [&](int64_t rows) -> int {
        if (!A->row_bound) return MWU_OK;
        rdiv = copy_in_f(c, A->row_bound, rows);
        if (!rdiv) return fail(c, MWU_ERR_OOM, "allocating row bounds");
        TRY_CUDA(c, validate_positive(rdiv, rows, 7, d_err, s));
        return MWU_OK;
    };
    int rc;
    switch (A->kind) {
    case MWU_MAT_CSR: {
        if (A->rows <= 0 || A->cols <= 0 || A->nnz < 0 || !A->rowptr || (A->nnz > 0 && !A->colidx))
            return fail(c, MWU_ERR_INVALID, "CSR: bad shape or null arrays");
        if (A->nnz >= (int64_t)INT32_MAX) return fail(c, MWU_ERR_INVALID, "CSR: nnz exceeds int32 indexing");
        const int32_t *ptr = copy_in_i(c, A->rowptr, A->rows + 1);
        const int32_t *idx = copy_in_i(c, A->colidx, A->nnz);
        const float *val = A->val ? copy_in_f(c, A->val, A->nnz) : nullptr;
        if (!ptr || !idx || (A->val && !val)) return fail(c, MWU_ERR_OOM, "copying CSR");
        TRY_CUDA(c, validate_csr(ptr, idx, val, A->rows, A->cols, A->nnz, sign < 0, d_err, s));
        if ((rc = check_err_flag(c, d_err)) != MWU_OK) return rc;
        if ((rc = load_bounds(A->rows)) != MWU_OK) return rc;
        int32_t *tp, *ti;
        float *tv;
        TRY_CUDA(c, csr_transpose(c->ar, ptr, idx, val, A->rows, A->cols, A->nnz, &tp, &ti, &tv, s));
        double avg_r = (double)A->nnz / (double)A->rows, avg_c = (double)A->nnz / (double)A->cols;
        sb.rv = RowView{RK_CSR, choose_G(avg_r, forced_G), A->rows, A->nnz, ptr, idx, val, rdiv};
        sb.cv = ColView{CK_CSR, choose_G(avg_c, forced_G), tp, ti, tv, rdiv, nullptr, 0, 0, nullptr};
        sb.m = A->rows;
        sb.nvar = A->cols;
        break;
    }
    case MWU_MAT_INCIDENCE:
    case MWU_MAT_INCIDENCE_T:
    case MWU_MAT_PAIR:
    case MWU_MAT_INTERWEAVE: {
        int64_t E = A->n_edges;
        int32_t nv = A->n_vertices;
        if (E <= 0 || !A->edges) return fail(c, MWU_ERR_INVALID, "implicit matrix: missing edge list");
        if (A->kind != MWU_MAT_INTERWEAVE && nv <= 0) return fail(c, MWU_ERR_INVALID, "implicit matrix: n_vertices <= 0");
        if (2 * E >= (int64_t)INT32_MAX) return fail(c, MWU_ERR_INVALID, "edge list exceeds int32 slot indexing");
        const int32_t *edges = copy_in_i(c, A->edges, 2 * E);
        if (!edges) return fail(c, MWU_ERR_OOM, "copying edge list");
        if (A->kind != MWU_MAT_INTERWEAVE) {
            TRY_CUDA(c, validate_edges(edges, E, nv, d_err, s));
            if ((rc = check_err_flag(c, d_err)) != MWU_OK) return rc;
        }
        int32_t *vptr = nullptr, *slots = nullptr, *eids = nullptr;
        if (A->kind != MWU_MAT_INTERWEAVE) {
            TRY_CUDA(c, build_vertex_slots(c->ar, edges, E, nv, &vptr, &slots, s));
            if (A->kind != MWU_MAT_PAIR) TRY_CUDA(c, slots_to_edges(c->ar, slots, 2 * E, &eids, s));
        }
        double avg = nv > 0 ? 2.0 * (double)E / (double)nv : 1.0;
        if (A->kind == MWU_MAT_INCIDENCE) {
            if (sign < 0) {   // covering vertex rows must be non-empty
                TRY_CUDA(c, validate_csr(vptr, eids, nullptr, nv, E, 2 * E, 1, d_err, s));
                if ((rc = check_err_flag(c, d_err)) != MWU_OK) return rc;
            }
            if ((rc = load_bounds(nv)) != MWU_OK) return rc;
            sb.rv = RowView{RK_CSR, choose_G(avg, forced_G), nv, 2 * E, vptr, eids, nullptr, rdiv};
            sb.cv = ColView{CK_FIXED2, 1, nullptr, edges, nullptr, rdiv, nullptr, 0, 0, nullptr};
            sb.m = nv;
            sb.nvar = E;
        } else if (A->kind == MWU_MAT_INCIDENCE_T) {
            if ((rc = load_bounds(E)) != MWU_OK) return rc;
            sb.rv = RowView{RK_FIXED2, 1, E, 2 * E, nullptr, edges, nullptr, rdiv};
            sb.cv = ColView{CK_CSR, choose_G(avg, forced_G), vptr, eids, nullptr, rdiv, nullptr, 0, 0, nullptr};
            sb.m = E;
            sb.nvar = nv;
            if (sign < 0 && !rdiv && c->opt.col_split >= 0 && !c->opt.h_scatter) {
                int32_t *cptr = nullptr, *vp2 = nullptr, *u2 = nullptr;
                int sorted = 0;
                TRY_CUDA(c, build_split_view(c->ar, edges, E, nv, &cptr, &vp2, &u2, &sorted, s));
                if (sorted) {
                    sb.cv.kind = CK_SPLIT2;
                    sb.cv.ptr = cptr;
                    sb.cv.idx = nullptr;
                    sb.cv.ptr2 = vp2;
                    sb.cv.idx2 = u2;
                }
            }
        } else if (A->kind == MWU_MAT_PAIR) {
            if ((rc = load_bounds(nv)) != MWU_OK) return rc;
            sb.rv = RowView{RK_CSR, choose_G(avg, forced_G), nv, 2 * E, vptr, slots, nullptr, rdiv};
            sb.cv = ColView{CK_FIXED1, 1, nullptr, edges, nullptr, rdiv, nullptr, 0, 0, nullptr};
            sb.m = nv;
            sb.nvar = 2 * E;
        } else {
            if ((rc = load_bounds(E)) != MWU_OK) return rc;
            sb.rv = RowView{RK_PAIRSUM, 1, E, 2 * E, nullptr, nullptr, nullptr, rdiv};
            sb.cv = ColView{CK_HALF1, 1, nullptr, nullptr, nullptr, rdiv, nullptr, 0, 0, nullptr};
            sb.m = E;
            sb.nvar = 2 * E;
        }
        break;
    }
    default:
        return fail(c, MWU_ERR_INVALID, "unsupported matrix kind");
    }
    // heavy rows of CSR row views
    if (sb.rv.kind == RK_CSR) {
        int32_t *list = nullptr, cnt = 0;
        TRY_CUDA(c, bin_list(c->ar, sb.rv.ptr, sb.rv.rows, -1, SHORT_LEN, &list, &cnt, s));
        sb.rv.short_rows = list;
        sb.rv.n_short = cnt;
        TRY_CUDA(c, bin_list(c->ar, sb.rv.ptr, sb.rv.rows, SHORT_LEN, MED_LEN, &list, &cnt, s));
        sb.rv.med_rows = list;
        sb.rv.n_med = cnt;
        // long rows: segments of SEG_LEN entries (host-side table, uploaded once)
        int32_t *lrows = nullptr, nl = 0;
        TRY_CUDA(c, bin_list(c->ar, sb.rv.ptr, sb.rv.rows, MED_LEN, INT32_MAX, &lrows, &nl, s));
        sb.rv.long_rows = lrows;
        sb.rv.n_long = nl;
        if (nl > 0) {
            std::vector<int32_t> lr(nl), hptr(sb.rv.rows + 1);
            TRY_CUDA(c, cudaMemcpyAsync(lr.data(), lrows, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, s));
            TRY_CUDA(c, cudaMemcpyAsync(hptr.data(), sb.rv.ptr, sizeof(int32_t) * (sb.rv.rows + 1),
                                        cudaMemcpyDeviceToHost, s));
            TRY_CUDA(c, cudaStreamSynchronize(s));
            std::vector<int32_t> lseg(nl + 1), srow, sbeg;
            for (int i = 0; i < nl; ++i) {
                lseg[i] = (int32_t)srow.size();
                for (int32_t k = hptr[lr[i]]; k < hptr[lr[i] + 1]; k += SEG_LEN) {
                    srow.push_back(lr[i]);
                    sbeg.push_back(k);
                }
            }
            lseg[nl] = (int32_t)srow.size();
            const int32_t ns = (int32_t)srow.size();
            int32_t *d_lseg = c->ar.alloc<int32_t>(nl + 1), *d_srow = c->ar.alloc<int32_t>(ns), *d_sbeg = c->ar.alloc<int32_t>(ns);
            if (!d_lseg || !d_srow || !d_sbeg) return fail(c, MWU_ERR_OOM, "allocating segment tables");
            TRY_CUDA(c, cudaMemcpyAsync(d_lseg, lseg.data(), sizeof(int32_t) * (nl + 1), cudaMemcpyHostToDevice, s));
            TRY_CUDA(c, cudaMemcpyAsync(d_srow, srow.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
            TRY_CUDA(c, cudaMemcpyAsync(d_sbeg, sbeg.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
            TRY_CUDA(c, cudaStreamSynchronize(s));
            sb.rv.long_seg = d_lseg;
            sb.rv.seg_row = d_srow;
            sb.rv.seg_beg = d_sbeg;
            sb.rv.n_seg = ns;
        }
        // staged SpMV for banded matrices: tiles of 4 row steps of a block; taken
        // when the input windows of at least 90 % of the tiles, holding at least
        // 90 % of the entries, fit in shared memory (a tile that does not fit runs
        // on one block from global memory: a few long rows there, like the item
        // rows of a users x items graph, would leave that block as the tail)
        if (c->opt.spmv_tiles >= 0 && sb.rv.rows > 0) {
            const int tr = 4 * (BLOCK / sb.rv.G);
            const int wmax = c->fp64 ? tile_wmax<double>() : tile_wmax<float>();
            int32_t *tlo = nullptr, *tlen = nullptr, nt = 0, fit = 0;
            int64_t fit_nnz = 0;
            TRY_CUDA(c, build_tiles(c->ar, sb.rv.ptr, sb.rv.idx, sb.rv.rows, tr, wmax, &tlo, &tlen, &nt, &fit, &fit_nnz, s));
            if (nt > 0 && (double)fit >= 0.9 * (double)nt && (double)fit_nnz >= 0.9 * (double)sb.rv.nnz) {
                sb.rv.n_tiles = nt;
                sb.rv.tile_rows = tr;
                sb.rv.tile_lo = tlo;
                sb.rv.tile_len = tlen;
            }
        }
    }
    return MWU_OK;
}

static void dense_side(SideBuild &sb, const float *c, int32_t sign) {
    sb.sign = sign;
    sb.dense = true;
    sb.rv = RowView{RK_DENSE1, 1, 1, 0, nullptr, nullptr, nullptr, nullptr};
    sb.cv = ColView{CK_DENSE1, 1, nullptr, nullptr, nullptr, nullptr, c, 0, 0, nullptr};
    sb.m = 1;
    sb.nvar = -1;
}

// Segments of SPLIT_SEG entries over the combined columns of the heavy
// variables of a CK_SPLIT2 side (host-built tables, uploaded once).
static int split_segments(mwu_ctx *c, ColView &cv, const int32_t *hv, int32_t nhv) {
    cudaStream_t s = c->stream;
    std::vector<int32_t> h_hv(nhv), h_ptr((size_t)c->n + 1);
    TRY_CUDA(c, cudaMemcpyAsync(h_hv.data(), hv, sizeof(int32_t) * nhv, cudaMemcpyDeviceToHost, s));
    TRY_CUDA(c, cudaMemcpyAsync(h_ptr.data(), cv.ptr, sizeof(int32_t) * ((size_t)c->n + 1), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(c, cudaStreamSynchronize(s));
    std::vector<int32_t> first(nhv + 1), var, beg;
    for (int32_t h = 0; h < nhv; ++h) {
        first[h] = (int32_t)var.size();
        const int32_t i = h_hv[h];
        for (int32_t k = h_ptr[i]; k < h_ptr[i + 1]; k += SPLIT_SEG) {
            var.push_back(i);
            beg.push_back(k);
        }
    }
    first[nhv] = (int32_t)var.size();
    const int32_t ns = (int32_t)var.size();
    int32_t *d_first = c->ar.alloc<int32_t>(nhv + 1), *d_var = c->ar.alloc<int32_t>(ns), *d_beg = c->ar.alloc<int32_t>(ns);
    if (!d_first || !d_var || !d_beg) return fail(c, MWU_ERR_OOM, "allocating column segment tables");
    TRY_CUDA(c, cudaMemcpyAsync(d_first, first.data(), sizeof(int32_t) * (nhv + 1), cudaMemcpyHostToDevice, s));
    if (ns > 0) {
        TRY_CUDA(c, cudaMemcpyAsync(d_var, var.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
        TRY_CUDA(c, cudaMemcpyAsync(d_beg, beg.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
    }
    TRY_CUDA(c, cudaStreamSynchronize(s));
    cv.n_cseg = ns;
    cv.cseg_first = d_first;
    cv.cseg_var = d_var;
    cv.cseg_beg = d_beg;
    return MWU_OK;
}

template <class T>
static int alloc_problem(mwu_ctx *c, Problem<T> &p, const SideBuild sb[2], int32_t *heavy_var, int32_t n_heavy_var,
                         int32_t *med_var, int32_t n_med_var, int G_var, int var_bps, int row_bps, int upd_bps) {
    p.n = c->n;
    p.x = c->ar.alloc<T>(c->n);
    p.d = c->ar.alloc<T>(c->n);
    p.g = c->ar.alloc<T>(c->n);
    p.h = c->ar.alloc<T>(c->n);
    if (!p.x || !p.d || !p.g || !p.h) return fail(c, MWU_ERR_OOM, "allocating variable vectors");
    for (int s = 0; s < 2; ++s) {
        Side<T> &sd = p.side[s];
        sd.rv = sb[s].rv;
        sd.cv = sb[s].cv;
        sd.sign = sb[s].sign;
        sd.m = sb[s].m;
        sd.seg_part = nullptr;
        if (!sb[s].dense) {
            sd.v = c->ar.alloc<T>(sd.m);
            sd.dv = c->ar.alloc<T>(sd.m);
            if (!sd.v || !sd.dv) return fail(c, MWU_ERR_OOM, "allocating constraint vectors");
            if (sd.rv.n_seg > 0) {
                sd.seg_part = c->ar.alloc<T>(sd.rv.n_seg);
                if (!sd.seg_part) return fail(c, MWU_ERR_OOM, "allocating segment partials");
            }
        } else {
            sd.v = sd.dv = nullptr;
        }
    }
    p.st = c->st_dev;
    p.grid_var = std::max(1, c->n_sms * var_bps);
    p.grid_row = std::max(2, c->n_sms * row_bps);
    p.grid_upd = std::max(2, c->n_sms * std::min(upd_bps, row_bps));
    p.grid_spmv = std::max(2, c->n_sms * std::min(8, spmv_blocks_per_sm<T>()));
    p.grid_newton = std::max(2, c->n_sms * std::min(8, newton_blocks_per_sm<T>()));
    p.grid_tiled = std::max(1, c->n_sms * tiled_blocks_per_sm<T>());
    p.cond_on = 0;
    p.cond = 0;
    p.cond_kc = 0;
    size_t recs = (size_t)std::max(std::max(p.grid_var, p.grid_newton), std::max(p.grid_row, p.grid_upd)) + 8;
    p.part_var = c->ar.alloc<double>((int64_t)(recs * REC));
    p.part_row = c->ar.alloc<double>((int64_t)(recs * REC));
    if (!p.part_var || !p.part_row) return fail(c, MWU_ERR_OOM, "allocating partial buffers");
    p.G_var = G_var;
    p.heavy_var = heavy_var;
    p.n_heavy_var = n_heavy_var;
    p.med_var = med_var;
    p.n_med_var = n_med_var;
    p.hacc = nullptr;
    p.cseg_part = nullptr;
    if (p.side[1].cv.kind == CK_SPLIT2 && p.side[1].cv.n_cseg > 0) {
        p.cseg_part = c->ar.alloc<T>(p.side[1].cv.n_cseg);
        if (!p.cseg_part) return fail(c, MWU_ERR_OOM, "allocating column segment partials");
    }
    p.x_eager = 0;
    for (int s = 0; s < 2; ++s)
        if (p.side[s].cv.kind == CK_SPLIT2) {
            p.side[s].cv.xsrc = p.x;
            p.x_eager = 1;
        }
    p.dv_scatter = (c->opt.dv_scatter && sb[1].rv.kind == RK_CSR && sb[1].cv.kind == CK_CSR) ? 2 : 0;
    if (c->opt.h_scatter && (sb[1].rv.kind == RK_FIXED2 || sb[1].rv.kind == RK_CSR) && sb[1].cv.kind == CK_CSR) {
        p.hacc = c->ar.alloc<T>(c->n);
        if (!p.hacc) return fail(c, MWU_ERR_OOM, "allocating the scatter sums");
        if (cudaMemsetAsync(p.hacc, 0, sizeof(T) * (size_t)c->n, c->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, MWU_ERR_CUDA, "clearing the scatter sums");
        }
    }
    return MWU_OK;
}

int mwu_create(int32_t kind, const mwu_matrix *P, const mwu_matrix *C, const float *objective_c,
               const mwu_options *opt, mwu_ctx **out) {
    if (!out) return fail(nullptr, MWU_ERR_INVALID, "out is NULL");
    *out = nullptr;
    mwu_options o;
    if (opt) o = *opt;
    else mwu_default_options(&o);
    if (!(o.eps > 0.0 && o.eps < 1.0)) return fail(nullptr, MWU_ERR_INVALID, "eps must lie in (0,1)");
    if (o.max_iter < 0 || o.K < 1 || o.K > KMAX) return fail(nullptr, MWU_ERR_INVALID, "max_iter < 0 or K not in 1..8");
    if (!(o.eta_factor > 0.0)) return fail(nullptr, MWU_ERR_INVALID, "eta_factor must be > 0");
    if (o.group != 0 && (o.group < 1 || o.group > 32 || (o.group & (o.group - 1))))
        return fail(nullptr, MWU_ERR_INVALID, "group must be 0 or a power of two <= 32");
    if (kind < MWU_PACKING || kind > MWU_DENSEST) return fail(nullptr, MWU_ERR_INVALID, "unknown problem kind");
    if (o.precision != MWU_PREC_F32_R64 && o.precision != MWU_PREC_FP64)
        return fail(nullptr, MWU_ERR_INVALID, "unknown precision");
    if (o.step < MWU_STEP_KARY || o.step > MWU_STEP_NEWTON) return fail(nullptr, MWU_ERR_INVALID, "unknown step mode");
    if (o.max_newton < 0) return fail(nullptr, MWU_ERR_INVALID, "max_newton must be >= 0");
    if (o.drop_covered < 0 || o.drop_covered > 2) return fail(nullptr, MWU_ERR_INVALID, "drop_covered must be 0, 1 or 2");

    mwu_ctx *c = new mwu_ctx();
    c->kind = kind;
    c->fp64 = o.precision == MWU_PREC_FP64;
    if (const char *tr = std::getenv("MWU_TRACE")) c->trace = tr[0] == '1';
    if (const char *g = std::getenv("MWU_SEARCH_GUARD")) c->guard_limit = std::atoi(g);
    if (c->fp64 || o.step == MWU_STEP_BINARY) o.K = 1;
    if (o.max_passes <= 0) o.max_passes = (c->fp64 || o.K == 1) ? 64 : (o.step == MWU_STEP_NEWTON ? 16 : 6);
    if (o.max_newton == 0) o.max_newton = 8;
    if (!(o.newton_tol > 0.0)) o.newton_tol = o.eps / 20.0;
    if (o.outer_tol <= 0.0) o.outer_tol = o.eps;
    if (o.max_probes <= 0) o.max_probes = 64;
    if (o.check_every <= 0) o.check_every = 8;
    if (o.grad_tol < 0.0) o.grad_tol = c->fp64 ? 0.0 : std::ldexp(1.0, -16);
    if (o.grad_tol >= 1.0) { c->err = "grad_tol must be < 1"; g_create_error = c->err; delete c; return MWU_ERR_INVALID; }
    if (o.stop_rule != 0 && o.stop_rule != 1) { c->err = "stop_rule must be 0 or 1"; g_create_error = c->err; delete c; return MWU_ERR_INVALID; }
    c->opt = o;
    auto bail = [&](int rc) {
        g_create_error = c->err;
        mwu_destroy(c);   // frees the arena, the stream and the pinned state
        return rc;
    };
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        // a blocking stream: its work is ordered after what the caller queued on
        // the legacy default stream, so device inputs written there before the
        // call are complete when the context reads them (a non-blocking stream
        // could copy an edge list that is still being written)
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault) != cudaSuccess) {
            cudaGetLastError();
            c->err = "cannot create a CUDA stream (no device?)";
            return bail(MWU_ERR_CUDA);
        }
        c->own_stream = true;
    }
    c->ar.set_stream(c->stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        c->err = "no CUDA device";
        return bail(MWU_ERR_CUDA);
    }
    int *d_err = c->ar.alloc<int>(4);
    if (!d_err || cudaMemsetAsync(d_err, 0, 4 * sizeof(int), c->stream) != cudaSuccess) {
        c->err = "allocating error flag";
        return bail(MWU_ERR_OOM);
    }
    SideBuild sb[2];
    int rc = MWU_OK;
    switch (kind) {
    case MWU_PACKING:
        if ((rc = build_side(c, P, +1, sb[0], d_err)) != MWU_OK) return bail(rc);
        c->n = sb[0].nvar;
        break;
    case MWU_COVERING:
        if ((rc = build_side(c, C, -1, sb[1], d_err)) != MWU_OK) return bail(rc);
        c->n = sb[1].nvar;
        break;
    case MWU_MIXED:
        if ((rc = build_side(c, P, +1, sb[0], d_err)) != MWU_OK) return bail(rc);
        if ((rc = build_side(c, C, -1, sb[1], d_err)) != MWU_OK) return bail(rc);
        if (sb[0].nvar != sb[1].nvar) { c->err = "P and C disagree on the number of variables"; return bail(MWU_ERR_INVALID); }
        c->n = sb[0].nvar;
        break;
    case MWU_DENSEST:
        if (!P || !C || P->kind != MWU_MAT_PAIR || C->kind != MWU_MAT_INTERWEAVE) {
            c->err = "DENSEST needs P = MWU_MAT_PAIR and C = MWU_MAT_INTERWEAVE";
            return bail(MWU_ERR_INVALID);
        }
        if (P->n_edges != C->n_edges) { c->err = "P and C edge counts differ"; return bail(MWU_ERR_INVALID); }
        if ((rc = build_side(c, P, +1, sb[0], d_err)) != MWU_OK) return bail(rc);
        if ((rc = build_side(c, C, -1, sb[1], d_err)) != MWU_OK) return bail(rc);
        c->n = sb[0].nvar;
        break;
    }
    if (c->n <= 0) { c->err = "no variables"; return bail(MWU_ERR_INVALID); }
    if (c->n >= (int64_t)INT32_MAX) { c->err = "variable count exceeds int32 indexing"; return bail(MWU_ERR_INVALID); }
    if (kind == MWU_PACKING || kind == MWU_COVERING) {
        const float *cd = nullptr;
        if (objective_c) {
            cd = copy_in_f(c, objective_c, c->n);
            if (!cd) { c->err = "copying objective"; return bail(MWU_ERR_OOM); }
            if (validate_nonneg(cd, c->n, 8, d_err, c->stream) != cudaSuccess) { c->err = "validate objective"; return bail(MWU_ERR_CUDA); }
            if ((rc = check_err_flag(c, d_err)) != MWU_OK) return bail(rc);
        }
        c->objective = cd;
        if (kind == MWU_PACKING) dense_side(sb[1], cd, -1);
        else dense_side(sb[0], cd, +1);
    }
    c->mP = sb[0].m;
    c->mC = sb[1].m;
    // variables of CSR column views by column length: lanes per light variable
    // from the 75th percentile of the lengths (power-law graphs have a mean
    // far above the typical column), G_var lanes covering four loads each;
    // light columns up to 16 G_var entries, medium up to HEAVY_LEN (a warp
    // each), heavy beyond (a block each)
    int G_var = 1;
    int32_t *hv = nullptr, nhv = 0, *mv = nullptr, nmv = 0;
    int32_t *tv = nullptr, ntv = 0, *lv = nullptr, nlv = -1;
    auto col_lengths = [&](const SideBuild &b) -> const int32_t * {
        return (b.cv.kind == CK_CSR || b.cv.kind == CK_SPLIT2) ? b.cv.ptr : nullptr;
    };
    const int32_t *cp0 = col_lengths(sb[0]);
    const int32_t *cp1 = col_lengths(sb[1]);
    if (cp0 || cp1) {
        int lq = 1;
        cudaError_t e = length_quantile2(c->ar, cp0, cp1, c->n, 0.75, &lq, c->stream);
        if (e != cudaSuccess) return bail(fail_cuda(c, e, "column length quantile"));
        G_var = c->opt.group > 0 ? c->opt.group : std::max(1, std::min(32, pow2_ceil((lq + 3) / 4)));
        const int light = std::min(16 * G_var, HEAVY_LEN);
        for (int s = 0; s < 2; ++s)
            if (sb[s].cv.kind == CK_CSR) { sb[s].cv.G = G_var; sb[s].cv.heavy_len = light; }
            else if (sb[s].cv.kind == CK_SPLIT2) { sb[s].cv.G = G_var; sb[s].cv.heavy_len = std::min(light, SPLIT_HEAVY); }
        // a split view sends every column above SPLIT_HEAVY entries through the
        // balanced segment pre-pass
        const int heavy = (sb[1].cv.kind == CK_SPLIT2 && !cp0) ? SPLIT_HEAVY : HEAVY_LEN;
        e = heavy_list2(c->ar, cp0, heavy, cp1, heavy, c->n, &hv, &nhv, c->stream);
        if (e == cudaSuccess) e = range_list2(c->ar, cp0, cp1, c->n, light, std::max(light, heavy), &mv, &nmv, c->stream);
        if (e != cudaSuccess) return bail(fail_cuda(c, e, "variable length classes"));
        if (sb[1].cv.kind == CK_SPLIT2 && nhv > 0 && (rc = split_segments(c, sb[1].cv, hv, nhv)) != MWU_OK)
            return bail(rc);
        if (sb[1].cv.kind == CK_SPLIT2 && !cp0) {   // split view: tiny and light variable lists
            const int lt = std::min(light, SPLIT_HEAVY);
            e = range_list2(c->ar, nullptr, cp1, c->n, -1, SPLIT_TINY, &tv, &ntv, c->stream);
            if (e == cudaSuccess) e = range_list2(c->ar, nullptr, cp1, c->n, SPLIT_TINY, lt, &lv, &nlv, c->stream);
            if (e != cudaSuccess) return bail(fail_cuda(c, e, "variable length classes"));
        }
    }
    // device state
    c->st_dev = c->ar.alloc<DevState>(1);
    if (!c->st_dev || cudaMallocHost((void **)&c->st_host, sizeof(DevState)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "allocating state";
        return bail(MWU_ERR_OOM);
    }
    std::memset(c->st_host, 0, sizeof(DevState));
    if (cudaMemsetAsync(c->st_dev, 0, sizeof(DevState), c->stream) != cudaSuccess) {
        cudaGetLastError();
        c->err = "clearing state";
        return bail(MWU_ERR_CUDA);
    }
    int vb = 1, rb = 1, ub = 1;
    if (c->fp64) {
        sweep_blocks_per_sm<double>(&vb, &rb, &ub);
        rc = alloc_problem(c, c->pd, sb, hv, nhv, mv, nmv, G_var, vb, rb, ub);
        c->pd.n_tiny_var = ntv; c->pd.tiny_var = tv; c->pd.n_light_var = nlv; c->pd.light_var = lv;
    } else {
        sweep_blocks_per_sm<float>(&vb, &rb, &ub);
        rc = alloc_problem(c, c->pf, sb, hv, nhv, mv, nmv, G_var, vb, rb, ub);
        c->pf.n_tiny_var = ntv; c->pf.tiny_var = tv; c->pf.n_light_var = nlv; c->pf.light_var = lv;
    }
    if (rc != MWU_OK) return bail(rc);
    // active-row compaction: drop_covered = 1 on a covering side of edge rows
    // in the split view (vertex cover); two buffer sets of pairs, z and row
    // numbers, one dz, the tile offsets
    {
        const Side<float> &s1f = c->pf.side[1];
        const Side<double> &s1d = c->pd.side[1];
        const int32_t ck = c->fp64 ? s1d.cv.kind : s1f.cv.kind, rk = c->fp64 ? s1d.rv.kind : s1f.rv.kind;
        const int64_t m1 = c->fp64 ? s1d.m : s1f.m;
        if (o.drop_covered == 1 && ck == CK_SPLIT2 && rk == RK_FIXED2 && !o.h_scatter && m1 > 0) {
            const size_t ts = c->fp64 ? sizeof(double) : sizeof(float);
            bool ok = true;
            for (int b = 0; b < 2; ++b) {
                c->cmp_pairs[b] = c->ar.alloc<int32_t>(2 * m1);
                c->cmp_orig[b] = c->ar.alloc<int32_t>(m1);
                c->cmp_v[b] = c->ar.raw((size_t)m1 * ts);
                ok = ok && c->cmp_pairs[b] && c->cmp_orig[b] && c->cmp_v[b];
            }
            c->cmp_dv = c->ar.raw((size_t)m1 * ts);
            c->cmp_tile = c->ar.alloc<int32_t>(cmp_tiles(m1) + 1);
            c->cmp_total = c->ar.alloc<int64_t>(1);
            if (!ok || !c->cmp_dv || !c->cmp_tile || !c->cmp_total) {
                c->err = "allocating the compaction buffers";
                return bail(MWU_ERR_OOM);
            }
            c->cmp_ok = true;
            c->cmp_full_f = s1f;
            c->cmp_full_d = s1d;
        }
    }
    c->x_best = c->ar.raw((size_t)c->n * (c->fp64 ? sizeof(double) : sizeof(float)));
    if (!c->x_best) { c->err = "allocating best x"; return bail(MWU_ERR_OOM); }
    c->ar.release_tmp();
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        fail_cuda(c, cudaGetLastError(), "mwu_create");
        return bail(MWU_ERR_CUDA);
    }
    // initial target: 1 (MIXED) or the automatic upper end
    rc = mwu_set_target(c, 1.0);
    if (rc < 0) return bail(rc);
    *out = c;
    return MWU_OK;
}

void mwu_destroy(mwu_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gexec_chunk) cudaGraphExecDestroy(c->gexec_chunk);
    if (c->gexec_one) cudaGraphExecDestroy(c->gexec_one);
    if (c->gexec_chunk_c) cudaGraphExecDestroy(c->gexec_chunk_c);
    if (c->gexec_one_c) cudaGraphExecDestroy(c->gexec_one_c);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_one) cudaEventDestroy(e);
    if (c->st_host) cudaFreeHost(c->st_host);
    c->ar.free_all();
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->body_stream) cudaStreamDestroy(c->body_stream);
    if (c->kc_stream) cudaStreamDestroy(c->kc_stream);
    if (c->batch_graph) cudaGraphExecDestroy(c->batch_graph);
    delete c;
}

// ------------------------------------------------------------ state I/O
static int pull_state(mwu_ctx *c) {
    TRY_CUDA(c, cudaMemcpyAsync(c->st_host, c->st_dev, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    return MWU_OK;
}
static int push_state(mwu_ctx *c) {
    TRY_CUDA(c, cudaMemcpyAsync(c->st_dev, c->st_host, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    return MWU_OK;
}

static void reset_probe_fields(DevState &h) {
    h.status = ST_RUNNING;
    h.reason = RS_NONE;
    h.iter = 0;
    h.numeric_bad = 0;
    h.pending = 0;
    h.alpha_acc = 0.0;
    h.alpha_prev = 0.0;
    h.phase = PH_DONE;
    h.passes = 0;
    h.last_passes = 0;
    h.evals = 0;
    h.total_passes = 0;
    h.n_pos = 0;
    for (int k = 0; k < 8; ++k) h.counter[k] = 0;
}

static int probe_status(const DevState &h) {
    switch (h.status) {
    case ST_FEASIBLE: return MWU_FEASIBLE;
    case ST_INFEASIBLE: return MWU_INFEASIBLE;
    case ST_MAX_ITER: return MWU_MAX_ITER;
    case ST_RUNNING: return MWU_RUNNING;
    case ST_TIMEOUT: return MWU_ERR_TIMEOUT;
    default: return MWU_ERR_NUMERIC;
    }
}

int mwu_set_target(mwu_ctx *c, double target) {
    if (!c) return MWU_ERR_INVALID;
    if (!(target > 0.0) || !std::isfinite(target)) return fail(c, MWU_ERR_INVALID, "target must be positive and finite");
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    DevState &h = *c->st_host;
    const mwu_options &o = c->opt;
    c->target = target;
    h.eps = o.eps;
    h.eta = o.eta_factor * std::log((double)(c->mP + c->mC)) / o.eps;
    h.inv_eta = 1.0 / h.eta;
    h.c_d = (o.double_single && (c->mP == 1 || c->mC == 1)) ? 1.0 / h.eta : 1.0 / (2.0 * h.eta);
    h.target = target;
    h.scale[0] = h.scale[1] = 1.0;
    if (c->kind == MWU_PACKING) h.scale[1] = 1.0 / target;
    else if (c->kind == MWU_COVERING || c->kind == MWU_DENSEST) h.scale[0] = 1.0 / target;
    h.max_iter = o.max_iter;
    h.K = o.K;
    h.max_passes = o.max_passes;
    h.guard_limit = c->guard_limit > 0 ? c->guard_limit : o.max_passes + 4;
    h.warm_start = o.warm_start;
    h.step_mode = o.step == MWU_STEP_STANDARD ? 2 : (o.step == MWU_STEP_BINARY ? 1 : (o.step == MWU_STEP_NEWTON ? 3 : 0));
    h.max_newton = o.max_newton;
    h.newton_tol = o.newton_tol;
    h.act_hi = o.drop_covered ? 1.0 : (double)INFINITY;
    h.kpass = o.K;
    h.deriv = 0;
    h.stop_rule = o.stop_rule;
    h.grad_tol = o.grad_tol;
    h.ratio_stop = o.stop_rule == 1 ? 1.0 + o.eps : 0.0;
    reset_probe_fields(h);
    if ((rc = push_state(c)) != MWU_OK) return rc;
    c->have_direction = false;
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_x_init(p, c->stream); }));
    c->launches += 2;
    if ((rc = pull_state(c)) != MWU_OK) return rc;
    return probe_status(h) == MWU_ERR_NUMERIC ? fail(c, MWU_ERR_NUMERIC, "NaN/Inf in the initial reductions") : MWU_OK;
}

int mwu_set_x(mwu_ctx *c, const void *x, int32_t x_is_fp64) {
    if (!c || !x) return MWU_ERR_INVALID;
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    reset_probe_fields(*c->st_host);
    if ((rc = push_state(c)) != MWU_OK) return rc;
    // stage a copy on the device when x is host memory
    cudaPointerAttributes at{};
    const void *src = x;
    void *tmp = nullptr;
    if (cudaPointerGetAttributes(&at, x) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        size_t nb = (size_t)c->n * (x_is_fp64 ? 8 : 4);
        TRY_CUDA(c, cudaMalloc(&tmp, nb));
        cudaError_t e = cudaMemcpyAsync(tmp, x, nb, cudaMemcpyDefault, c->stream);
        if (e != cudaSuccess) { cudaFree(tmp); return fail_cuda(c, e, "copy x"); }
        src = tmp;
    }
    cudaError_t e = with_prob(c, [&](auto &p) { return launch_x_set(p, src, x_is_fp64, c->stream); });
    if (tmp) { cudaStreamSynchronize(c->stream); cudaFree(tmp); }
    if (e != cudaSuccess) return fail_cuda(c, e, "launch_x_set");
    c->have_direction = false;
    if ((rc = pull_state(c)) != MWU_OK) return rc;
    return probe_status(*c->st_host) == MWU_ERR_NUMERIC ? fail(c, MWU_ERR_NUMERIC, "NaN/Inf in the reductions of Px, Cx")
                                                         : MWU_OK;
}

// a6: dv = A d for both sides.  The covering side's dz is already written by
// the edge-pair direction kernel (densest), or comes by scatter over the
// columns of the moving variables (option dv_scatter); the rest by the SpMV.
template <class Prob>
static cudaError_t spmv_direction(const Prob &p, int keep_gh, cudaStream_t s) {
    bool skip_c = dir_fuses_dz(p, keep_gh);
    if (!skip_c && (p.dv_scatter & 2)) {
        cudaError_t e = launch_spmv_scatter(p, 1, s);
        if (e != cudaSuccess) return e;
        skip_c = true;
    }
    return launch_spmv(p, s, skip_c ? 1 : 0);
}

// Copy n entries of src (host or device memory, float32 or float64 per
// src_fp64) into the context's vector dst of type T, converting on the device.
template <class T>
static int load_vec(mwu_ctx *c, T *dst, const void *src, int64_t n, int32_t src_fp64) {
    cudaPointerAttributes at{};
    const void *from = src;
    void *tmp = nullptr;
    const size_t nb = (size_t)n * (src_fp64 ? 8 : 4);
    if (cudaPointerGetAttributes(&at, src) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        TRY_CUDA(c, cudaMalloc(&tmp, nb));
        cudaError_t e = cudaMemcpyAsync(tmp, src, nb, cudaMemcpyDefault, c->stream);
        if (e != cudaSuccess) { cudaFree(tmp); return fail_cuda(c, e, "copy vector in"); }
        from = tmp;
    }
    cudaError_t e = src_fp64 ? launch_convert_in<T>((const double *)from, dst, n, c->stream)
                             : launch_convert_in<T>((const float *)from, dst, n, c->stream);
    // every constraint value and direction product of the LP is finite and >= 0
    int *bad = nullptr, h = 0;
    if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = launch_check_nonneg<T>(dst, n, bad, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    if (tmp) cudaFree(tmp);
    if (bad) cudaFree(bad);
    if (e != cudaSuccess) return fail_cuda(c, e, "convert vector in");
    if (h) return fail(c, MWU_ERR_INVALID, "loaded vector holds a negative, NaN or infinite value");
    return MWU_OK;
}

// One entry of src (host or device) as a double: the value of a side that is
// the single objective row.
static int load_scalar(mwu_ctx *c, const void *src, int32_t src_fp64, double *out) {
    if (src_fp64) {
        TRY_CUDA(c, cudaMemcpy(out, src, 8, cudaMemcpyDefault));
    } else {
        float f = 0.0f;
        TRY_CUDA(c, cudaMemcpy(&f, src, 4, cudaMemcpyDefault));
        *out = (double)f;
    }
    return std::isfinite(*out) ? MWU_OK : fail(c, MWU_ERR_INVALID, "non-finite value loaded");
}

int mwu_set_state(mwu_ctx *c, const void *y, const void *z, const void *dy, const void *dz, int32_t is_fp64) {
    if (!c) return MWU_ERR_INVALID;
    if (!y && !z && !dy && !dz) return MWU_OK;
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    DevState &h = *c->st_host;
    const void *vals[2] = {y, z}, *dirs[2] = {dy, dz};
    const bool rows = y || z;
    if (rows) reset_probe_fields(h);
    auto side_of = [&](auto &p, int s) -> auto & { return p.side[s]; };
    for (int s = 0; s < 2; ++s) {
        const bool dense = c->fp64 ? side_of(c->pd, s).rv.kind == RK_DENSE1 : side_of(c->pf, s).rv.kind == RK_DENSE1;
        const int64_t m = c->fp64 ? side_of(c->pd, s).m : side_of(c->pf, s).m;
        for (int w = 0; w < 2; ++w) {
            const void *src = w == 0 ? vals[s] : dirs[s];
            if (!src) continue;
            if (dense) {
                double v = 0.0;
                if ((rc = load_scalar(c, src, is_fp64, &v)) != MWU_OK) return rc;
                (w == 0 ? h.dense_v : h.dense_dv)[s] = v;
                continue;
            }
            if (c->fp64) {
                auto &sd = side_of(c->pd, s);
                rc = load_vec<double>(c, w == 0 ? sd.v : sd.dv, src, m, is_fp64);
            } else {
                auto &sd = side_of(c->pf, s);
                rc = load_vec<float>(c, w == 0 ? sd.v : sd.dv, src, m, is_fp64);
            }
            if (rc != MWU_OK) return rc;
        }
    }
    if ((rc = push_state(c)) != MWU_OK) return rc;
    if (rows) {
        TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_rows_reduce(p, c->stream); }));
        c->launches += 1;
    }
    if (dy || dz) c->have_direction = true;
    else if (rows) c->have_direction = false;
    if ((rc = pull_state(c)) != MWU_OK) return rc;
    return probe_status(h) == MWU_ERR_NUMERIC ? fail(c, MWU_ERR_NUMERIC, "NaN/Inf in the reductions of y, z")
                                              : MWU_OK;
}

int mwu_set_direction(mwu_ctx *c, const void *d, int32_t is_fp64) {
    if (!c || !d) return MWU_ERR_INVALID;
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    if (c->st_host->status != ST_RUNNING) return fail(c, MWU_ERR_STATE, "probe not running (set a target or x first)");
    if (c->fp64) rc = load_vec<double>(c, c->pd.d, d, c->n, is_fp64);
    else rc = load_vec<float>(c, c->pf.d, d, c->n, is_fp64);
    if (rc != MWU_OK) return rc;
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_dense_dir(p, c->stream); }));
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return spmv_direction(p, 1, c->stream); }));
    if ((rc = pull_state(c)) != MWU_OK) return rc;
    c->have_direction = true;
    return MWU_OK;
}


// ------------------------------------------------------------ iterations
// kernels of one iteration; ev (6 events or nullptr) brackets the kernel classes.  The
// events are recorded as external event nodes when the sequence is captured.
// kernels an eager iteration launches: direction, SpMV, update and max_passes
// turns of the search (two kernels per turn with Newton's method)
// kernels an iteration launches besides direction, SpMV and update: the h
// scatter, the x step before a rebuilding update, the split view's segment
// pre-pass and the long-row segment fix-up after the SpMV
static int extra_kernels(const mwu_ctx *c) {
    auto count = [](const auto &p) {
        return (p.hacc != nullptr) + p.x_eager + (p.side[1].cv.n_cseg > 0) +
               (p.side[0].rv.n_long + p.side[1].rv.n_long > 0);
    };
    return c->fp64 ? count(c->pd) : count(c->pf);
}
static int kernels_per_iteration(const mwu_ctx *c) {
    return 3 + extra_kernels(c) + (c->opt.step == MWU_STEP_NEWTON ? 2 : 1) * c->opt.max_passes;
}
constexpr int EV_PER_IT = 5;

// The step-size search of one iteration.  Captured (graph): a conditional WHILE
// node, opened by the direction kernel, whose body is the one-candidate pass
// kernel (Newton and backoff passes) followed by an IF node around the
// K-candidate pass kernel; the first kernel sets the IF condition, and every
// body turn ends by setting the loop condition, so the loop runs the passes the
// search needs and no turn launches a kernel that has nothing to do.  Eager:
// max_passes turns of the same kernels, which return at once outside their
// phases or once the search has ended.
template <class Prob>
static cudaError_t enqueue_search(mwu_ctx *c, Prob &p, bool loop) {
    cudaError_t e;
    if (!loop) {
        for (int k = 0; k < c->opt.max_passes; ++k) {
            if (c->opt.step == MWU_STEP_NEWTON && (e = launch_cand_newton(p, c->stream)) != cudaSuccess) return e;
            if ((e = launch_cand(p, 0, c->stream)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess) return e;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = p.cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return e;
    if (!c->body_stream && (e = cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return e;
    if (!c->kc_stream && (e = cudaStreamCreateWithFlags(&c->kc_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return e;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaGraphConditionalHandleCreate(&p.cond_kc, body, 0u, 0u)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCaptureToGraph(c->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess)
        return e;
    cudaError_t e1 = launch_cand_newton(p, c->body_stream);
    cudaGraphNodeParams ip{};
    if (e1 == cudaSuccess) {
        cudaGraph_t bg = nullptr;
        const cudaGraphNode_t *bdeps = nullptr;
        size_t bnd = 0;
        e1 = cudaStreamGetCaptureInfo(c->body_stream, &cs, nullptr, &bg, &bdeps, nullptr, &bnd);
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = p.cond_kc;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode;
        if (e1 == cudaSuccess) e1 = cudaGraphAddNode(&inode, bg, bdeps, nullptr, bnd, &ip);
        if (e1 == cudaSuccess)
            e1 = cudaStreamUpdateCaptureDependencies(c->body_stream, &inode, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies);
    }
    if (e1 == cudaSuccess) {
        e1 = cudaStreamBeginCaptureToGraph(c->kc_stream, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed);
        if (e1 == cudaSuccess) {
            cudaError_t e3 = launch_cand(p, 0, c->kc_stream);
            cudaGraph_t kbody = nullptr;
            cudaError_t e4 = cudaStreamEndCapture(c->kc_stream, &kbody);
            e1 = e3 != cudaSuccess ? e3 : e4;
        }
    }
    cudaGraph_t bout = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->body_stream, &bout);
    return e1 != cudaSuccess ? e1 : e2;
}

// The direction kernels read the covering side through its column view, whose
// split form streams z by the full edge order: with compacted rows they get
// the full z (the update keeps it current for the active edges).
template <class P> static P dir_view(const P &p) {
    P q = p;
    if (q.side[1].orig) q.side[1].v = q.side[1].vfull;
    return q;
}

static cudaError_t enqueue_iteration(mwu_ctx *c, cudaEvent_t *ev, bool loop = false) {
    return with_prob(c, [&](auto &p0) -> cudaError_t {
        cudaError_t e;
        auto p = p0;   // this iteration's copy: carries the handle of its search loop
        if (loop) {
            cudaStreamCaptureStatus cs;
            cudaGraph_t g = nullptr;
            if ((e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr)) != cudaSuccess)
                return e;
            if ((e = cudaGraphConditionalHandleCreate(&p.cond, g, 0u, 0u)) != cudaSuccess) return e;
            p.cond_on = 1;
        }
        if (ev && (e = cudaEventRecordWithFlags(ev[0], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
        if ((e = launch_dir(dir_view(p), 0, c->stream)) != cudaSuccess) return e;
        if (ev && (e = cudaEventRecordWithFlags(ev[1], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
        if ((e = spmv_direction(p, 0, c->stream)) != cudaSuccess) return e;
        if (ev && (e = cudaEventRecordWithFlags(ev[2], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
        if ((e = enqueue_search(c, p, loop)) != cudaSuccess) return e;
        if (ev && (e = cudaEventRecordWithFlags(ev[3], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
        if ((e = launch_update(p, c->stream)) != cudaSuccess) return e;
        if (ev && (e = cudaEventRecordWithFlags(ev[4], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
        return cudaSuccess;
    });
}

static int make_events(mwu_ctx *c, std::vector<cudaEvent_t> &ev, int n) {
    while ((int)ev.size() < n) {
        cudaEvent_t e;
        TRY_CUDA(c, cudaEventCreate(&e));
        ev.push_back(e);
    }
    return MWU_OK;
}

static int capture(mwu_ctx *c, int iters, std::vector<cudaEvent_t> &ev, cudaGraphExec_t *out) {
    int rc;
    if (c->opt.timing && (rc = make_events(c, ev, EV_PER_IT * iters)) != MWU_OK) return rc;
    cudaGraph_t g = nullptr;
    TRY_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < iters && e == cudaSuccess; ++k)
        e = enqueue_iteration(c, c->opt.timing ? &ev[EV_PER_IT * k] : nullptr, true);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return fail_cuda(c, e, "capture iteration"); }
    if (e2 != cudaSuccess) return fail_cuda(c, e2, "end capture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { *out = nullptr; return fail_cuda(c, e, "instantiate iteration graph"); }
    return MWU_OK;
}

static int ensure_graphs(mwu_ctx *c) {
    int rc;
    cudaGraphExec_t &gc = c->cmp_on ? c->gexec_chunk_c : c->gexec_chunk;
    cudaGraphExec_t &g1 = c->cmp_on ? c->gexec_one_c : c->gexec_one;
    if (!gc && (rc = capture(c, c->opt.check_every, c->ev, &gc)) != MWU_OK) return rc;
    if (!g1 && (rc = capture(c, 1, c->ev_one, &g1)) != MWU_OK) return rc;
    return MWU_OK;
}

// ------------------------------------------------------------ active-row compaction
// Between graph launches (or iterations of the plain form) of one mwu_iterate
// call: count the unsatisfied covering rows (z < act_hi) of the current rows
// and, once they are at most CMP_KEEP of them, compact the edge pairs, z and
// the original row numbers into the other buffer set.  x only grows within a
// probe, so a dropped row stays satisfied.
constexpr double CMP_KEEP = 0.7;

template <class T> static int compact_rows(mwu_ctx *c, Problem<T> &p, const Side<T> &full) {
    Side<T> &sd = p.side[1];
    const int64_t m = sd.m;
    if (m <= 0) return MWU_OK;
    const double hi = c->st_host->act_hi;
    TRY_CUDA(c, launch_cmp_count<T>(sd.v, m, hi, c->cmp_tile, c->cmp_total, c->stream));
    int64_t total = 0;
    TRY_CUDA(c, cudaMemcpyAsync(&total, c->cmp_total, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    c->launches += 2;
    if (total <= 0 || (double)total > CMP_KEEP * (double)m) return MWU_OK;
    const int nb = c->cmp_on ? 1 - c->cmp_buf : 0;
    TRY_CUDA(c, launch_cmp_scatter<T>(sd.rv.idx, sd.v, sd.orig, m, hi, c->cmp_tile, c->cmp_pairs[nb],
                                      (T *)c->cmp_v[nb], c->cmp_orig[nb], c->stream));
    c->launches += 1;
    sd.rv.idx = c->cmp_pairs[nb];
    sd.rv.rows = total;
    sd.rv.nnz = 2 * total;
    sd.m = total;
    sd.v = (T *)c->cmp_v[nb];
    sd.dv = (T *)c->cmp_dv;
    sd.orig = c->cmp_orig[nb];
    sd.vfull = full.v;
    c->cmp_buf = nb;
    c->cmp_on = true;
    c->tim.compactions += 1;
    if (c->gexec_chunk_c) { cudaGraphExecDestroy(c->gexec_chunk_c); c->gexec_chunk_c = nullptr; }
    if (c->gexec_one_c) { cudaGraphExecDestroy(c->gexec_one_c); c->gexec_one_c = nullptr; }
    if (c->trace)
        std::fprintf(stderr, "[mwu] compaction: %lld of %lld covering rows active (iteration %d)\n", (long long)total,
                     (long long)m, c->st_host->iter);
    return MWU_OK;
}

static int maybe_compact(mwu_ctx *c) {
    if (!c->cmp_ok || c->st_host->status != ST_RUNNING) return MWU_OK;
    return c->fp64 ? compact_rows(c, c->pd, c->cmp_full_d) : compact_rows(c, c->pf, c->cmp_full_f);
}

// Back to the full rows: z = x_u + x_v over every edge (the rows dropped
// earlier hold their value at drop time), and a probe that stopped on the
// bound act_hi for the dropped rows' minimum re-runs the stopping test on the
// exact min z over every row.
template <class T> static int expand_rows(mwu_ctx *c, Problem<T> &p, const Side<T> &full) {
    p.side[1] = full;
    c->cmp_on = false;
    TRY_CUDA(c, launch_cmp_refresh<T>(p, c->stream));
    c->launches += 1;
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    DevState &h = *c->st_host;
    if (h.reason == RS_RATIO || h.reason == RS_COVERED || h.reason == RS_PACKING) {
        h.status = ST_RUNNING;
        h.reason = RS_NONE;
        TRY_CUDA(c, cudaMemcpyAsync(&c->st_dev->status, &h.status, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        TRY_CUDA(c, cudaMemcpyAsync(&c->st_dev->reason, &h.reason, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
        TRY_CUDA(c, launch_rows_reduce<T>(p, c->stream));
        c->launches += 1;
        if ((rc = pull_state(c)) != MWU_OK) return rc;
    }
    return MWU_OK;
}

static int cmp_expand(mwu_ctx *c) {
    if (!c->cmp_on) return MWU_OK;
    return c->fp64 ? expand_rows(c, c->pd, c->cmp_full_d) : expand_rows(c, c->pf, c->cmp_full_f);
}

// add the event times of the first `real` iterations recorded in ev
static int accumulate_timing(mwu_ctx *c, const std::vector<cudaEvent_t> &ev, int real) {
    for (int k = 0; k < real; ++k) {
        float t[EV_PER_IT - 1];
        for (int j = 0; j < EV_PER_IT - 1; ++j)
            TRY_CUDA(c, cudaEventElapsedTime(&t[j], ev[EV_PER_IT * k + j], ev[EV_PER_IT * k + j + 1]));
        c->tim.dir_ms += t[0];
        c->tim.spmv_ms += t[1];
        c->tim.cand_ms += t[2];
        c->tim.update_ms += t[3];
        c->tim.iters += 1;
    }
    return MWU_OK;
}

static void fill_stats(mwu_ctx *c, mwu_iter_stats *s) {
    if (!s) return;
    const DevState &h = *c->st_host;
    s->status = probe_status(h);
    s->reason = h.reason;
    s->iters = h.iter;
    s->last_passes = h.last_passes;
    s->evals = h.evals;
    s->passes = h.total_passes;
    s->alpha = h.alpha_prev;
    s->ymax = h.ymax;
    s->zmin = h.zmin;
}

static int iterate_loop(mwu_ctx *c, int32_t n_iters) {
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    c->have_direction = false;
    const bool graph = !c->fp64 && c->opt.use_graph;
    const int kpi = kernels_per_iteration(c);
    int done = 0;
    while (done < n_iters && c->st_host->status == ST_RUNNING) {
        const int iter0 = c->st_host->iter;
        const int64_t passes0 = c->st_host->total_passes;
        const int64_t loop0 = c->st_host->loop_launches;
        if (c->fp64) {
            // plain form: host-driven search, one readback per candidate pass
            std::vector<cudaEvent_t> &ev = c->ev_one;
            if (c->opt.timing && (rc = make_events(c, ev, EV_PER_IT)) != MWU_OK) return rc;
            if (c->opt.timing) TRY_CUDA(c, cudaEventRecord(ev[0], c->stream));
            TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_dir(dir_view(p), 0, c->stream); }));
            if (c->opt.timing) TRY_CUDA(c, cudaEventRecord(ev[1], c->stream));
            TRY_CUDA(c, with_prob(c, [&](auto &p) { return spmv_direction(p, 0, c->stream); }));
            if (c->opt.timing) TRY_CUDA(c, cudaEventRecord(ev[2], c->stream));
            TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_cand(p, 0, c->stream); }));
            c->launches += 3;
            if ((rc = pull_state(c)) != MWU_OK) return rc;
            int guard = 0;
            const int limit = c->guard_limit > 0 ? c->guard_limit : c->opt.max_passes + 4;
            while (c->st_host->status == ST_RUNNING && c->st_host->phase != PH_DONE) {
                if (guard++ >= limit)
                    return fail(c, MWU_ERR_TIMEOUT, "the step search exceeded its bound on candidate passes");
                const bool cover = c->st_host->phase == PH_COVER;
                TRY_CUDA(c, with_prob(c, [&](auto &p) {
                    return cover ? launch_cand_newton(p, c->stream) : launch_cand(p, 0, c->stream);
                }));
                c->launches += 1;
                if ((rc = pull_state(c)) != MWU_OK) return rc;
            }
            if (c->opt.timing) TRY_CUDA(c, cudaEventRecord(ev[3], c->stream));
            TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_update(p, c->stream); }));
            if (c->opt.timing) TRY_CUDA(c, cudaEventRecord(ev[4], c->stream));
            c->launches += 1 + extra_kernels(c);
            if ((rc = pull_state(c)) != MWU_OK) return rc;
            if (c->opt.timing && (rc = accumulate_timing(c, ev, c->st_host->iter - iter0)) != MWU_OK) return rc;
            done += 1;
        } else if (graph) {
            if ((rc = ensure_graphs(c)) != MWU_OK) return rc;
            bool chunk = n_iters - done >= c->opt.check_every;
            int n = chunk ? c->opt.check_every : 1;
            cudaGraphExec_t gx = chunk ? (c->cmp_on ? c->gexec_chunk_c : c->gexec_chunk)
                                       : (c->cmp_on ? c->gexec_one_c : c->gexec_one);
            TRY_CUDA(c, cudaGraphLaunch(gx, c->stream));
            if ((rc = pull_state(c)) != MWU_OK) return rc;
            // direction, SpMV and update per captured iteration, plus the kernels
            // the search loops ran (counted on the device)
            c->launches += (int64_t)n * (3 + extra_kernels(c)) + (c->st_host->loop_launches - loop0);
            if (c->opt.timing &&
                (rc = accumulate_timing(c, chunk ? c->ev : c->ev_one, c->st_host->iter - iter0)) != MWU_OK)
                return rc;
            done += n;
        } else {
            int n = std::min(c->opt.check_every, n_iters - done);
            for (int k = 0; k < n; ++k) TRY_CUDA(c, enqueue_iteration(c, nullptr));
            c->launches += (int64_t)n * kpi;
            if ((rc = pull_state(c)) != MWU_OK) return rc;
            done += n;
        }
        c->tim.cand_passes += c->st_host->total_passes - passes0;
        if ((rc = maybe_compact(c)) != MWU_OK) return rc;
    }
    return MWU_OK;
}

int mwu_iterate(mwu_ctx *c, int32_t n_iters, mwu_iter_stats *stats) {
    if (!c || n_iters < 0) return MWU_ERR_INVALID;
    int rc = iterate_loop(c, n_iters);
    const int rc2 = cmp_expand(c);   // the full rows again (exact z, the stopping test re-decided)
    if (rc != MWU_OK) return rc;
    if (rc2 != MWU_OK) return rc2;
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_flush(p, c->stream); }));
    c->launches += 1;
    if ((rc = pull_state(c)) != MWU_OK) return rc;
    fill_stats(c, stats);
    int st = probe_status(*c->st_host);
    if (st == MWU_ERR_NUMERIC) return fail(c, MWU_ERR_NUMERIC, "NaN/Inf in a reduction");
    if (st == MWU_ERR_TIMEOUT) return fail(c, MWU_ERR_TIMEOUT, "the device-side step search exceeded its bound on turns");
    return st;
}

int mwu_get_timing(mwu_ctx *c, mwu_timing *out, int32_t reset) {
    if (!c) return MWU_ERR_INVALID;
    mwu_timing t = c->tim;
    if (out) *out = t;
    if (reset) c->tim = mwu_timing{};
    return MWU_OK;
}

int mwu_spmv_tiles(mwu_ctx *c, int32_t *tiles_p, int32_t *tiles_c) {
    if (!c || c->kind < 0) return MWU_ERR_INVALID;
    int32_t t[2];
    for (int s = 0; s < 2; ++s) t[s] = c->fp64 ? c->pd.side[s].rv.n_tiles : c->pf.side[s].rv.n_tiles;
    if (tiles_p) *tiles_p = t[0];
    if (tiles_c) *tiles_c = t[1];
    return MWU_OK;
}

int mwu_direction(mwu_ctx *c, int64_t *n_positive) {
    if (!c) return MWU_ERR_INVALID;
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    if (c->st_host->status != ST_RUNNING) return fail(c, MWU_ERR_STATE, "probe not running (set a target or x first)");
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_dir(p, 1, c->stream); }));
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return spmv_direction(p, 1, c->stream); }));
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_cand(p, 1, c->stream); }));
    if ((rc = pull_state(c)) != MWU_OK) return rc;
    if (n_positive) *n_positive = c->st_host->n_pos;
    c->have_direction = true;
    int st = probe_status(*c->st_host);
    if (st == MWU_ERR_NUMERIC) return fail(c, MWU_ERR_NUMERIC, "NaN/Inf in a reduction");
    if (st == MWU_ERR_TIMEOUT) return fail(c, MWU_ERR_TIMEOUT, "the device-side step search exceeded its bound on turns");
    return st == MWU_RUNNING ? MWU_OK : st;
}

int mwu_eval_candidates(mwu_ctx *c, const double *alphas, int32_t K, double *psi, double *phi, double *zmin) {
    if (!c || !alphas || K < 1 || K > KMAX) return MWU_ERR_INVALID;
    if (!c->have_direction) return fail(c, MWU_ERR_STATE, "call mwu_direction first");
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    DevState saved = *c->st_host;
    DevState &h = *c->st_host;
    h.K = K;
    h.kpass = K;
    h.deriv = 0;
    for (int k = 0; k < K; ++k) h.alpha[k] = alphas[k];
    if ((rc = push_state(c)) != MWU_OK) return rc;
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_cand(p, 1, c->stream); }));
    if ((rc = pull_state(c)) != MWU_OK) return rc;
    for (int k = 0; k < K; ++k) {
        if (psi) psi[k] = h.psi[k];
        if (phi) phi[k] = h.phi[k];
        if (zmin) zmin[k] = h.zmink[k];
    }
    int bad = h.status == ST_NUMERIC;
    // restore the search state of the direction
    saved.psi[0] = h.psi[0];
    *c->st_host = saved;
    if ((rc = push_state(c)) != MWU_OK) return rc;
    TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    return bad ? fail(c, MWU_ERR_NUMERIC, "NaN/Inf in a candidate") : MWU_OK;
}

int mwu_eval_newton(mwu_ctx *c, double alpha, double *out) {
    if (!c || !out || !(alpha >= 0.0)) return MWU_ERR_INVALID;
    if (!c->have_direction) return fail(c, MWU_ERR_STATE, "call mwu_direction first");
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    DevState saved = *c->st_host;
    DevState &h = *c->st_host;
    h.K = 1;
    h.kpass = 1;
    h.deriv = 1;
    h.alpha[0] = alpha;
    if ((rc = push_state(c)) != MWU_OK) return rc;
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_cand(p, 1, c->stream); }));
    if ((rc = pull_state(c)) != MWU_OK) return rc;
    out[0] = h.psi[0];
    out[1] = h.phi[0];
    out[2] = h.dpsi;
    out[3] = h.dphi;
    int bad = h.status == ST_NUMERIC;
    *c->st_host = saved;
    if ((rc = push_state(c)) != MWU_OK) return rc;
    TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    return bad ? fail(c, MWU_ERR_NUMERIC, "NaN/Inf in a candidate") : MWU_OK;
}

int mwu_search(mwu_ctx *c, double *alpha, int64_t *evals) {
    if (!c) return MWU_ERR_INVALID;
    if (!c->have_direction) return fail(c, MWU_ERR_STATE, "call mwu_direction first");
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    int guard = 0;
    while (c->st_host->status == ST_RUNNING && c->st_host->phase != PH_DONE && guard++ < 256) {
        const bool cover = c->st_host->phase == PH_COVER;   // the covering-step pass
        TRY_CUDA(c, with_prob(c, [&](auto &p) {
            return cover ? launch_cand_newton(p, c->stream) : launch_cand(p, 0, c->stream);
        }));
        if ((rc = pull_state(c)) != MWU_OK) return rc;
    }
    if (alpha) *alpha = c->st_host->status == ST_RUNNING ? c->st_host->alpha_acc : 0.0;
    if (evals) *evals = c->st_host->evals;
    int st = probe_status(*c->st_host);
    if (st == MWU_ERR_NUMERIC) return fail(c, MWU_ERR_NUMERIC, "NaN/Inf in a candidate");
    return st == MWU_RUNNING ? MWU_OK : st;
}

// ------------------------------------------------------------ read back
int mwu_get_scalars(mwu_ctx *c, mwu_scalars *o) {
    if (!c || !o) return MWU_ERR_INVALID;
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    const DevState &h = *c->st_host;
    o->eta = h.eta;
    o->c_d = h.c_d;
    o->eps = h.eps;
    o->target = h.target;
    o->s_p = h.s[0];
    o->S_p = h.S[0];
    o->s_c = h.s[1];
    o->S_c = h.S[1];
    o->ymax = h.ymax;
    o->zmin = h.zmin;
    o->alpha = h.alpha_acc > 0 ? h.alpha_acc : h.alpha_prev;
    o->n_positive = h.n_pos;
    o->n = c->n;
    o->m_P = c->mP;
    o->m_C = c->mC;
    o->K = h.K;
    o->iters = h.iter;
    return MWU_OK;
}

int mwu_get_vector(mwu_ctx *c, int32_t which, void *dst, int64_t n, int32_t as_fp64) {
    if (!c || !dst) return MWU_ERR_INVALID;
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    const void *src = nullptr;
    int64_t len = 0;
    int side = -1;
    bool dv = false;
    switch (which) {
    case MWU_VEC_X: len = c->n; break;
    case MWU_VEC_D: len = c->n; break;
    case MWU_VEC_G: len = c->n; break;
    case MWU_VEC_H: len = c->n; break;
    case MWU_VEC_Y: side = 0; break;
    case MWU_VEC_Z: side = 1; break;
    case MWU_VEC_DY: side = 0; dv = true; break;
    case MWU_VEC_DZ: side = 1; dv = true; break;
    default: return fail(c, MWU_ERR_INVALID, "unknown vector id");
    }
    auto pick = [&](auto &p) {
        using T = std::remove_pointer_t<decltype(p.x)>;
        const T *s = nullptr;
        if (side < 0) s = which == MWU_VEC_X ? p.x : which == MWU_VEC_D ? p.d : which == MWU_VEC_G ? p.g : p.h;
        else { s = dv ? p.side[side].dv : p.side[side].v; len = p.side[side].m; }
        return (const void *)s;
    };
    src = c->fp64 ? pick(c->pd) : pick(c->pf);
    if (n != len) return fail(c, MWU_ERR_INVALID, "length mismatch");
    if (side >= 0 && !src) {   // the single objective row: a scalar held in the state
        double v = dv ? c->st_host->dense_dv[side] : c->st_host->dense_v[side];
        if (as_fp64) { double t = v; TRY_CUDA(c, cudaMemcpy(dst, &t, 8, cudaMemcpyDefault)); }
        else { float t = (float)v; TRY_CUDA(c, cudaMemcpy(dst, &t, 4, cudaMemcpyDefault)); }
        return MWU_OK;
    }
    bool same = (as_fp64 != 0) == c->fp64;
    cudaPointerAttributes at{};
    bool dst_dev = cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    size_t nb = (size_t)len * (as_fp64 ? 8 : 4);
    if (same) {
        TRY_CUDA(c, cudaMemcpyAsync(dst, src, nb, cudaMemcpyDefault, c->stream));
    } else if (dst_dev) {
        if (c->fp64) TRY_CUDA(c, launch_copy_vec<double>((const double *)src, dst, len, as_fp64, c->stream));
        else TRY_CUDA(c, launch_copy_vec<float>((const float *)src, dst, len, as_fp64, c->stream));
    } else {
        void *tmp = nullptr;
        TRY_CUDA(c, cudaMalloc(&tmp, nb));
        cudaError_t e = c->fp64 ? launch_copy_vec<double>((const double *)src, tmp, len, as_fp64, c->stream)
                                : launch_copy_vec<float>((const float *)src, tmp, len, as_fp64, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, nb, cudaMemcpyDefault, c->stream);
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return fail_cuda(c, e, "copy vector");
    }
    TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    return MWU_OK;
}

// ------------------------------------------------------------ certificate
// Recompute y = Px and z = Cx exactly from x and return the certified
// objective of the homogeneous LP (c^T x / max(Px), c^T x / min(Cx), or
// max(Oz)/min(Wz)); the probe's status is left unchanged.
static int certify(mwu_ctx *c, double *cert) {
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_x_set(p, p.x, c->fp64 ? 1 : 0, c->stream); }));
    c->launches += 2;
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    const DevState &h = *c->st_host;
    double M = c->target;
    switch (c->kind) {
    case MWU_PACKING: *cert = h.s[0] > 0 ? M * h.dense_v[1] / h.s[0] : 0.0; break;
    case MWU_COVERING: *cert = h.s[1] > 0 ? M * h.dense_v[0] / h.s[1] : INFINITY; break;
    case MWU_DENSEST: *cert = h.s[1] > 0 ? M * h.s[0] / h.s[1] : INFINITY; break;
    default: *cert = h.s[1] > 0 ? h.s[0] / h.s[1] : INFINITY; break;
    }
    return MWU_OK;
}

static int auto_bracket_compute(mwu_ctx *c, double *lo, double *hi);

// The automatic bracket depends on the matrices and the objective only, which
// a context keeps: it is computed by the first solve and reused.
static int auto_bracket(mwu_ctx *c, double *lo, double *hi) {
    if (!c->bracket_ok) {
        int rc = auto_bracket_compute(c, &c->bracket_lo, &c->bracket_hi);
        if (rc != MWU_OK) return rc;
        c->bracket_ok = true;
    }
    *lo = c->bracket_lo;
    *hi = c->bracket_hi;
    return MWU_OK;
}

static int auto_bracket_compute(mwu_ctx *c, double *lo, double *hi) {
    double a = 0, b = 0, dmax = 0;
    cudaStream_t s = c->stream;
    auto side_views = [&](int sd, RowView &rv, ColView &cv, int64_t &m) {
        if (c->fp64) { rv = c->pd.side[sd].rv; cv = c->pd.side[sd].cv; m = c->pd.side[sd].m; }
        else { rv = c->pf.side[sd].rv; cv = c->pf.side[sd].cv; m = c->pf.side[sd].m; }
    };
    RowView rv;
    ColView cv;
    int64_t m;
    switch (c->kind) {
    case MWU_PACKING:
        // hi = sum_i c_i max_j 1/a_ji (Sec. 2.2), lo = value of x_i = 1/(n max_j a_ji)
        side_views(0, rv, cv, m);
        TRY_CUDA(c, bracket_stats(c->ar, cv, c->n, c->objective, &a, &b, &dmax, s));
        *hi = a;
        *lo = b / (double)c->n;
        break;
    case MWU_COVERING:
        // hi = c^T x for x_i = 1/min_j a_ji (feasible), lo = max_j min_i c_i / a_ji
        side_views(1, rv, cv, m);
        TRY_CUDA(c, bracket_stats(c->ar, cv, c->n, c->objective, &a, &b, &dmax, s));
        *hi = a;
        TRY_CUDA(c, bracket_rowratio(c->ar, rv, m, c->objective, lo, s));
        break;
    case MWU_DENSEST: {
        // lo = |E| / |V| (density of the whole graph), hi = d_max / 2
        side_views(0, rv, cv, m);
        int64_t nv = m, E = c->n / 2;
        std::vector<int32_t> ptr(nv + 1);
        TRY_CUDA(c, cudaMemcpyAsync(ptr.data(), rv.ptr, sizeof(int32_t) * (nv + 1), cudaMemcpyDeviceToHost, s));
        TRY_CUDA(c, cudaStreamSynchronize(s));
        int32_t dm = 0;
        for (int64_t v = 0; v < nv; ++v) dm = std::max(dm, ptr[v + 1] - ptr[v]);
        *lo = (double)E / (double)nv;
        *hi = dm / 2.0;
        break;
    }
    default:
        *lo = *hi = 1.0;
    }
    c->ar.release_tmp();
    return MWU_OK;
}

int mwu_solve(mwu_ctx *c, double lo, double hi, mwu_result *res) {
    if (!c) return MWU_ERR_INVALID;
    auto t0 = std::chrono::steady_clock::now();
    mwu_result r{};
    int rc;
    const int64_t launches0 = c->launches;
    if (c->kind == MWU_MIXED) {
        if ((rc = mwu_set_target(c, 1.0)) != MWU_OK) return rc;
        mwu_iter_stats s{};
        rc = mwu_iterate(c, c->opt.max_iter, &s);
        if (rc < 0) return rc;
        double cert;
        if ((rc = certify(c, &cert)) != MWU_OK) return rc;
        r.status = s.status;
        r.objective = cert;
        r.probes = 1;
        r.iters = s.iters;
        r.evals = s.evals;
        r.passes = s.passes;
    } else {
        if (lo <= 0.0 || hi <= 0.0) {
            double alo = 0, ahi = 0;
            if ((rc = auto_bracket(c, &alo, &ahi)) != MWU_OK) return rc;
            if (lo <= 0.0) lo = alo;
            if (hi <= 0.0) hi = ahi;
        }
        if (!(lo > 0.0) || !(hi >= lo)) return fail(c, MWU_ERR_INVALID, "bad bracket");
        const bool maximize = c->kind == MWU_PACKING;
        double best = maximize ? lo : hi;
        bool have_best = false;
        int probes = 0;
        int64_t iters = 0, evals = 0, passes = 0;
        size_t xb = (size_t)c->n * (c->fp64 ? 8 : 4);
        while (hi > (1.0 + c->opt.outer_tol) * lo && probes < c->opt.max_probes) {
            double M = std::sqrt(lo * hi);
            if ((rc = mwu_set_target(c, M)) != MWU_OK) return rc;
            // The probe may also stop as soon as its certificate closes the search:
            // cert = M zmin/ymax >= hi/(1+tol) (max) or M ymax/zmin <= (1+tol) lo (min).
            {
                const double tol1 = 1.0 + c->opt.outer_tol;
                double rho = maximize ? tol1 * M / hi : tol1 * lo / M;
                DevState &h = *c->st_host;
                h.ratio_stop = std::max(h.ratio_stop, rho);
                TRY_CUDA(c, cudaMemcpyAsync(&c->st_dev->ratio_stop, &h.ratio_stop, sizeof(double),
                                            cudaMemcpyHostToDevice, c->stream));
            }
            mwu_iter_stats s{};
            rc = mwu_iterate(c, c->opt.max_iter, &s);
            if (rc < 0) return rc;
            double cert;
            if ((rc = certify(c, &cert)) != MWU_OK) return rc;
            ++probes;
            iters += s.iters;
            evals += s.evals;
            passes += s.passes;
            if (c->trace)
                std::fprintf(stderr, "[mwu] probe %d target=%.9g status=%d reason=%d iters=%d passes=%lld cert=%.9g "
                             "lo=%.9g hi=%.9g\n", probes, M, s.status, s.reason, s.iters, (long long)s.passes, cert,
                             lo, hi);
            bool better = maximize ? cert > best : cert < best;
            if (better || !have_best) {
                if (better) best = cert;
                have_best = true;
                const void *xs = c->fp64 ? (const void *)c->pd.x : (const void *)c->pf.x;
                TRY_CUDA(c, cudaMemcpyAsync(c->x_best, xs, xb, cudaMemcpyDeviceToDevice, c->stream));
            }
            if (maximize) {
                lo = std::max(lo, cert);
                if (s.status == MWU_FEASIBLE) lo = std::max(lo, M);
                else hi = std::min(hi, M);
            } else {
                hi = std::min(hi, cert);
                if (s.status == MWU_FEASIBLE) hi = std::min(hi, M);
                else lo = std::max(lo, M);
            }
        }
        if (have_best) {
            void *xs = c->fp64 ? (void *)c->pd.x : (void *)c->pf.x;
            TRY_CUDA(c, cudaMemcpyAsync(xs, c->x_best, xb, cudaMemcpyDeviceToDevice, c->stream));
        }
        TRY_CUDA(c, cudaStreamSynchronize(c->stream));
        r.status = MWU_OK;
        r.objective = best;
        r.lo = lo;
        r.hi = hi;
        r.probes = probes;
        r.iters = iters;
        r.evals = evals;
        r.passes = passes;
    }
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    r.launches = c->launches - launches0;
    if (res) *res = r;
    return MWU_OK;
}

// ------------------------------------------------------------ potential
// The potential takes every covering row, whatever drop_covered says: the
// dropping threshold is lifted for the evaluation and put back after it.
static int set_drop_threshold(mwu_ctx *c, double hi) {
    int rc = pull_state(c);
    if (rc != MWU_OK) return rc;
    c->st_host->act_hi = hi;
    return push_state(c);
}

static int potential_all_rows(mwu_ctx *c, const float *x, double *pot, float *grad_x, float *grad_obj,
                              float *grad_vals);

int mwu_potential(mwu_ctx *c, const float *x, double *pot, float *grad_x, float *grad_obj, float *grad_vals) {
    if (!c || !x) return MWU_ERR_INVALID;
    if (!c->opt.drop_covered) return potential_all_rows(c, x, pot, grad_x, grad_obj, grad_vals);
    int rc = set_drop_threshold(c, (double)INFINITY);
    if (rc != MWU_OK) return rc;
    rc = potential_all_rows(c, x, pot, grad_x, grad_obj, grad_vals);
    // back to the active rows: the sums of the state at x follow them again
    int rc2 = set_drop_threshold(c, 1.0);
    if (rc2 == MWU_OK) rc2 = mwu_set_x(c, x, 0);
    return rc != MWU_OK ? rc : rc2;
}

static int potential_all_rows(mwu_ctx *c, const float *x, double *pot, float *grad_x, float *grad_obj,
                              float *grad_vals) {
    int rc = mwu_set_x(c, x, 0);
    if (rc != MWU_OK) return rc;
    const DevState &h = *c->st_host;
    double smx = h.s[0] + std::log(h.S[0]) / h.eta;
    double smn = h.s[1] - std::log(h.S[1]) / h.eta;
    if (pot) *pot = smx - smn;
    float *gp = nullptr, *gc = nullptr;
    if (grad_vals) {
        bool pcsr = c->fp64 ? c->pd.side[0].rv.kind == RK_CSR : c->pf.side[0].rv.kind == RK_CSR;
        bool ccsr = c->fp64 ? c->pd.side[1].rv.kind == RK_CSR : c->pf.side[1].rv.kind == RK_CSR;
        if (pcsr) gp = grad_vals;
        if (ccsr) {
            int64_t off = 0;
            if (pcsr) {
                int32_t last = 0;
                const int32_t *pp = c->fp64 ? c->pd.side[0].rv.ptr : c->pf.side[0].rv.ptr;
                int64_t rows = c->fp64 ? c->pd.side[0].m : c->pf.side[0].m;
                TRY_CUDA(c, cudaMemcpy(&last, pp + rows, sizeof(int32_t), cudaMemcpyDeviceToHost));
                off = last;
            }
            gc = grad_vals + off;
        }
    }
    TRY_CUDA(c, with_prob(c, [&](auto &p) { return launch_potential_grads(p, x, grad_x, grad_obj, gp, gc, c->stream); }));
    TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_direction = false;
    return MWU_OK;
}

// ------------------------------------------------------------ value check
int mwu_check_values(mwu_ctx *c, const float *objective, const float *vals, int32_t *same) {
    if (!c || !same || c->is_batch) return MWU_ERR_INVALID;
    *same = 1;
    int *flag = nullptr;
    TRY_CUDA(c, cudaMalloc(&flag, sizeof(int)));
    std::vector<void *> staged;
    auto release = [&]() {
        cudaStreamSynchronize(c->stream);
        for (void *p : staged) cudaFree(p);
        cudaFree(flag);
    };
    auto device_view = [&](const float *src, int64_t n, const float **out) -> cudaError_t {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeDevice) {
            *out = src;
            return cudaSuccess;
        }
        cudaGetLastError();
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, 4 * (size_t)std::max<int64_t>(n, 1));
        if (e != cudaSuccess) return e;
        staged.push_back(p);
        *out = (const float *)p;
        return cudaMemcpyAsync(p, src, 4 * (size_t)n, cudaMemcpyDefault, c->stream);
    };
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), c->stream);
    if (e == cudaSuccess && objective && (c->kind == MWU_PACKING || c->kind == MWU_COVERING)) {
        const float *d = nullptr;
        e = device_view(objective, c->n, &d);
        if (e == cudaSuccess) e = launch_same_f32(c->objective, d, c->n, flag, c->stream);
    }
    if (e == cudaSuccess && vals) {
        int64_t off = 0;
        for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
            const RowView &rv = c->fp64 ? c->pd.side[s].rv : c->pf.side[s].rv;
            if (rv.kind != RK_CSR) continue;
            const float *d = nullptr;
            e = device_view(vals + off, rv.nnz, &d);
            if (e == cudaSuccess) e = launch_same_f32(rv.val, d, rv.nnz, flag, c->stream);
            off += rv.nnz;
        }
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    release();
    if (e != cudaSuccess) return fail_cuda(c, e, "mwu_check_values");
    *same = h ? 0 : 1;
    return MWU_OK;
}

// ------------------------------------------------------------ batch
// The instances are packed into one set of arrays (edges, capacities and the
// vertex -> incident-edge lists of each, built with the setup's stable radix
// sort) and solved by one persistent launch (k_batch_solve): a block per
// instance at a time, taken from a work queue in decreasing size.
int mwu_create_batch(int32_t count, const mwu_matrix *P, const mwu_options *opt, mwu_ctx **out) {
    if (!out || !P || count <= 0) return fail(nullptr, MWU_ERR_INVALID, "bad batch arguments");
    *out = nullptr;
    mwu_options o;
    if (opt) o = *opt;
    else mwu_default_options(&o);
    if (!(o.eps > 0.0 && o.eps < 1.0)) return fail(nullptr, MWU_ERR_INVALID, "eps must lie in (0,1)");
    if (o.batch_workers != 0 && o.batch_workers != 256 && o.batch_workers != 512 && o.batch_workers != 1024)
        return fail(nullptr, MWU_ERR_INVALID, "batch_workers must be 0 (autotuned), 256, 512 or 1024");
    if (o.batch_cluster == 0) o.batch_cluster = 1;
    if (o.batch_cluster != 1 && o.batch_cluster != 4 && o.batch_cluster != 8 && o.batch_cluster != 16)
        return fail(nullptr, MWU_ERR_INVALID, "batch_cluster must be 0, 1, 4, 8 or 16");
    if (o.batch_cluster_edges < 0) return fail(nullptr, MWU_ERR_INVALID, "batch_cluster_edges must be >= 0");
    if (o.batch_cluster > 1 && o.batch_workers == 1024)
        return fail(nullptr, MWU_ERR_INVALID, "batch_cluster > 1 needs batch_workers 0, 256 or 512");
    int64_t Et = 0, Nt = 0;
    for (int k = 0; k < count; ++k) {
        if (P[k].kind != MWU_MAT_INCIDENCE || !P[k].edges || P[k].n_edges <= 0 || P[k].n_vertices <= 0)
            return fail(nullptr, MWU_ERR_INVALID, "batch instance " + std::to_string(k) +
                                                  ": PACKING over a non-empty MWU_MAT_INCIDENCE edge list required");
        if (2 * P[k].n_edges >= (int64_t)INT32_MAX) return fail(nullptr, MWU_ERR_INVALID, "instance too large");
        Et += P[k].n_edges;
        Nt += P[k].n_vertices;
    }
    mwu_ctx *c = new mwu_ctx();
    c->kind = -1;
    c->is_batch = true;
    if (o.step != MWU_STEP_KARY && o.step != MWU_STEP_NEWTON)
        return fail(nullptr, MWU_ERR_INVALID, "batch: step must be MWU_STEP_KARY or MWU_STEP_NEWTON");
    if (o.max_passes <= 0) o.max_passes = o.step == MWU_STEP_NEWTON ? 16 : 6;
    if (o.max_newton <= 0) o.max_newton = 8;
    if (!(o.newton_tol > 0.0)) o.newton_tol = o.eps / 20.0;
    if (o.outer_tol <= 0.0) o.outer_tol = o.eps;
    if (o.max_probes <= 0) o.max_probes = 64;
    if (o.grad_tol < 0.0) o.grad_tol = std::ldexp(1.0, -16);
    if (o.K < 1 || o.K > KMAX) o.K = KMAX;
    c->opt = o;
    auto bail = [&](int rc) {
        g_create_error = c->err;
        mwu_destroy(c);
        return rc;
    };
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault) != cudaSuccess) {
        cudaGetLastError();
        c->err = "cannot create a CUDA stream (no device?)";
        return bail(MWU_ERR_CUDA);
    }
    c->own_stream = true;
    c->ar.set_stream(c->stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        c->err = "no CUDA device";
        return bail(MWU_ERR_CUDA);
    }
    cudaStream_t s = c->stream;
    std::vector<int64_t> eoff(count + 1, 0), voff(count + 1, 0);
    for (int k = 0; k < count; ++k) {
        eoff[k + 1] = eoff[k] + P[k].n_edges;
        voff[k + 1] = voff[k] + P[k].n_vertices;
        c->batch_e.push_back(P[k].n_edges);
    }
    c->batch_count = count;
    c->batch_edges = Et;
    int32_t *edges = c->ar.alloc<int32_t>(2 * Et), *vptr = c->ar.alloc<int32_t>(Nt + count), *eids = c->ar.alloc<int32_t>(2 * Et);
    float *bound = c->ar.alloc<float>(Nt);
    int64_t *d_eoff = c->ar.alloc<int64_t>(count + 1), *d_voff = c->ar.alloc<int64_t>(count + 1);
    int32_t *d_order = c->ar.alloc<int32_t>(count);
    int *d_err = c->ar.alloc<int>(4);
    if (!edges || !vptr || !eids || !bound || !d_eoff || !d_voff || !d_order || !d_err) {
        c->err = "allocating the packed batch";
        return bail(MWU_ERR_OOM);
    }
    if (cudaMemsetAsync(d_err, 0, 4 * sizeof(int), s) != cudaSuccess) { c->err = "clearing flags"; return bail(MWU_ERR_CUDA); }
    std::vector<float> ones;
    for (int k = 0; k < count; ++k) {
        const int64_t E = P[k].n_edges, n = P[k].n_vertices;
        int32_t *ek = edges + 2 * eoff[k];
        if (cudaMemcpyAsync(ek, P[k].edges, 8 * (size_t)E, cudaMemcpyDefault, s) != cudaSuccess ||
            validate_edges(ek, E, (int32_t)n, d_err, s) != cudaSuccess) {
            cudaGetLastError();
            c->err = "copying instance " + std::to_string(k);
            return bail(MWU_ERR_CUDA);
        }
        int32_t *vp = nullptr, *sl = nullptr, *el = nullptr;
        cudaError_t e = build_vertex_slots(c->ar, ek, E, (int32_t)n, &vp, &sl, s);
        if (e == cudaSuccess) e = slots_to_edges(c->ar, sl, 2 * E, &el, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vptr + voff[k] + k, vp, 4 * (size_t)(n + 1), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(eids + 2 * eoff[k], el, 8 * (size_t)E, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) {
            if (P[k].row_bound) {
                e = cudaMemcpyAsync(bound + voff[k], P[k].row_bound, 4 * (size_t)n, cudaMemcpyDefault, s);
            } else {
                ones.assign((size_t)n, 1.0f);
                e = cudaMemcpyAsync(bound + voff[k], ones.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            }
        }
        if (e != cudaSuccess) return bail(fail_cuda(c, e, "packing a batch instance"));
        c->ar.release_tmp();
    }
    if (validate_positive(bound, Nt, 7, d_err, s) != cudaSuccess) { c->err = "validating bounds"; return bail(MWU_ERR_CUDA); }
    int rc = check_err_flag(c, d_err);
    if (rc != MWU_OK) return bail(rc);
    std::vector<int32_t> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return P[a].n_edges > P[b].n_edges; });
    c->batch_order = order;
    TRY_CUDA(c, cudaMemcpyAsync(d_eoff, eoff.data(), 8 * (size_t)(count + 1), cudaMemcpyHostToDevice, s));
    TRY_CUDA(c, cudaMemcpyAsync(d_voff, voff.data(), 8 * (size_t)(count + 1), cudaMemcpyHostToDevice, s));
    TRY_CUDA(c, cudaMemcpyAsync(d_order, order.data(), 4 * (size_t)count, cudaMemcpyHostToDevice, s));
    BatchDesc &B = c->bd;
    B.count = count;
    B.order = d_order;
    B.eoff = d_eoff;
    B.voff = d_voff;
    B.edges = edges;
    B.bound = bound;
    B.vptr = vptr;
    B.eids = eids;
    B.x = c->ar.alloc<float>(Et);
    B.d = c->ar.alloc<float>(Et);
    B.y = c->ar.alloc<float>(Nt);
    B.dy = c->ar.alloc<float>(Nt);
    B.obj = c->ar.alloc<double>(count);
    B.iters = c->ar.alloc<int64_t>(count);
    B.evals = c->ar.alloc<int64_t>(count);
    B.passes = c->ar.alloc<int64_t>(count);
    B.probes = c->ar.alloc<int32_t>(count);
    B.queue = c->ar.alloc<unsigned int>(2);
    B.t_beg = c->ar.alloc<int64_t>(count);
    B.t_end = c->ar.alloc<int64_t>(count);
    if (!B.x || !B.d || !B.y || !B.dy || !B.obj || !B.iters || !B.evals || !B.passes || !B.probes || !B.queue ||
        !B.t_beg || !B.t_end) {
        c->err = "allocating the batch work vectors";
        return bail(MWU_ERR_OOM);
    }
    B.eps = o.eps;
    B.eta_factor = o.eta_factor;
    B.outer_tol = o.outer_tol;
    B.grad_tol = o.grad_tol;
    B.max_iter = o.max_iter;
    B.max_probes = o.max_probes;
    B.max_passes = o.max_passes;
    B.K = o.K;
    B.warm_start = o.warm_start;
    B.step_mode = o.step == MWU_STEP_NEWTON ? 3 : 0;
    B.max_newton = o.max_newton;
    B.newton_tol = o.newton_tol;
    c->batch_nt = o.batch_workers;   // 0: tuned on the first solve
    c->batch_cl = o.batch_cluster;
    TRY_CUDA(c, cudaStreamSynchronize(s));
    *out = c;
    return MWU_OK;
}

// The autotuner's configurations (threads per block, blocks per cluster), in
// the order of mwu_batch_tuning's timings.
static const int kTuneNT[MWU_BATCH_TUNE_CONFIGS] = {256, 512, 1024, 256, 512, 256, 512, 256, 512};
static const int kTuneCL[MWU_BATCH_TUNE_CONFIGS] = {1, 1, 1, 4, 4, 8, 8, 16, 16};

// Instances solved by whole clusters: the prefix of the order with at least
// batch_cluster_edges edges (0: 2 x threads x cluster).
static int batch_n_cluster(const mwu_ctx *c, int nt, int cl) {
    if (cl <= 1) return 0;
    const int64_t thr = c->opt.batch_cluster_edges > 0 ? (int64_t)c->opt.batch_cluster_edges : 2LL * nt * cl;
    int k = 0;
    while (k < c->batch_count && c->batch_e[c->batch_order[k]] >= thr) ++k;
    return k;
}

// The persistent grid: every block resident, no more than the work needs.
static int batch_blocks_for(mwu_ctx *c, int nt, int cl) {
    const int res = batch_blocks(nt, cl, c->n_sms);
    if (res <= 0) return 0;
    const int nc = batch_n_cluster(c, nt, cl);
    const int64_t need = (int64_t)nc * cl + (c->batch_count - nc);
    const int64_t b = std::min<int64_t>(res, (need + cl - 1) / cl * cl);
    return (int)std::max<int64_t>(cl, b);
}

static cudaError_t batch_launch(mwu_ctx *c, int nt, int cl) {
    const int blocks = batch_blocks_for(c, nt, cl);
    if (blocks <= 0) return cudaErrorInvalidConfiguration;
    return launch_batch_solve(c->bd, nt, cl, batch_n_cluster(c, nt, cl), blocks, c->stream);
}

// Autotuner: the whole batch solved once in each configuration (CUDA events),
// the fastest kept for the context (and its timings for mwu_batch_tuning).  A
// configuration the device cannot run (no resident cluster) is skipped.
static int batch_autotune(mwu_ctx *c) {
    cudaEvent_t a, b;
    TRY_CUDA(c, cudaEventCreate(&a));
    TRY_CUDA(c, cudaEventCreate(&b));
    int best = -1;
    for (int i = 0; i < MWU_BATCH_TUNE_CONFIGS; ++i) {
        c->tune_ms[i] = 0.0;
        if (batch_blocks_for(c, kTuneNT[i], kTuneCL[i]) <= 0) continue;
        cudaError_t e = cudaEventRecord(a, c->stream);
        if (e == cudaSuccess) e = batch_launch(c, kTuneNT[i], kTuneCL[i]);
        if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return fail_cuda(c, e, "batch autotune"); }
        c->tune_ms[i] = ms;
        if (best < 0 || ms < c->tune_ms[best]) best = i;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (best < 0) return fail(c, MWU_ERR_CUDA, "batch autotune: no configuration can run");
    c->batch_nt = kTuneNT[best];
    c->batch_cl = kTuneCL[best];
    return MWU_OK;
}

int mwu_solve_batch(mwu_ctx *c, double *objective, int64_t *iters, mwu_result *total) {
    if (!c || !c->is_batch) return MWU_ERR_INVALID;
    auto t0 = std::chrono::steady_clock::now();
    int rc;
    if (c->batch_nt == 0 && (rc = batch_autotune(c)) != MWU_OK) return rc;
    if (c->batch_graph_nt != c->batch_nt || c->batch_graph_cl != c->batch_cl) {
        if (c->batch_graph) { cudaGraphExecDestroy(c->batch_graph); c->batch_graph = nullptr; }
        c->batch_blocks = batch_blocks_for(c, c->batch_nt, c->batch_cl);
        if (c->batch_blocks <= 0) return fail(c, MWU_ERR_INVALID, "batch: no cluster of this size fits the device");
        cudaGraph_t g = nullptr;
        TRY_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = batch_launch(c, c->batch_nt, c->batch_cl);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return fail_cuda(c, e, "capture batch solve"); }
        if (e2 != cudaSuccess) return fail_cuda(c, e2, "end capture");
        e = cudaGraphInstantiate(&c->batch_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { c->batch_graph = nullptr; return fail_cuda(c, e, "instantiate batch graph"); }
        c->batch_graph_nt = c->batch_nt;
        c->batch_graph_cl = c->batch_cl;
    }
    TRY_CUDA(c, cudaGraphLaunch(c->batch_graph, c->stream));
    const int n = c->batch_count;
    std::vector<double> obj(n);
    std::vector<int64_t> it(n), ev(n), pa(n);
    std::vector<int32_t> pr(n);
    c->batch_t_beg.resize(n);
    c->batch_t_end.resize(n);
    TRY_CUDA(c, cudaMemcpyAsync(c->batch_t_beg.data(), c->bd.t_beg, 8 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaMemcpyAsync(c->batch_t_end.data(), c->bd.t_end, 8 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaMemcpyAsync(obj.data(), c->bd.obj, 8 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaMemcpyAsync(it.data(), c->bd.iters, 8 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaMemcpyAsync(ev.data(), c->bd.evals, 8 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaMemcpyAsync(pa.data(), c->bd.passes, 8 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaMemcpyAsync(pr.data(), c->bd.probes, 4 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    mwu_result tot{};
    bool bad = false;
    for (int k = 0; k < n; ++k) {
        if (objective) objective[k] = obj[k];
        if (iters) iters[k] = it[k];
        if (!std::isfinite(obj[k])) bad = true;
        tot.objective += obj[k];
        tot.probes += pr[k];
        tot.iters += it[k];
        tot.evals += ev[k];
        tot.passes += pa[k];
    }
    c->batch_last_passes = pa;
    c->batch_last_probes = pr;
    tot.launches = 1;
    tot.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (total) *total = tot;
    return bad ? fail(c, MWU_ERR_NUMERIC, "NaN/Inf in a batch instance") : MWU_OK;
}

int mwu_batch_tuning(mwu_ctx *c, int32_t *threads, int32_t *cluster, double *ms) {
    if (!c || !c->is_batch) return MWU_ERR_INVALID;
    if (threads) *threads = c->batch_nt;
    if (cluster) *cluster = c->batch_nt ? c->batch_cl : 0;
    if (ms) for (int i = 0; i < MWU_BATCH_TUNE_CONFIGS; ++i) ms[i] = c->tune_ms[i];
    return MWU_OK;
}

int mwu_batch_timeline(mwu_ctx *c, double *start_ms, double *end_ms) {
    if (!c || !c->is_batch) return MWU_ERR_INVALID;
    if (c->batch_t_beg.empty()) return fail(c, MWU_ERR_STATE, "no batch solve yet");
    const int64_t t0 = *std::min_element(c->batch_t_beg.begin(), c->batch_t_beg.end());
    for (int k = 0; k < c->batch_count; ++k) {
        if (start_ms) start_ms[k] = 1e-6 * (double)(c->batch_t_beg[k] - t0);
        if (end_ms) end_ms[k] = 1e-6 * (double)(c->batch_t_end[k] - t0);
    }
    return MWU_OK;
}

int mwu_batch_stats(mwu_ctx *c, int64_t *passes, int32_t *probes) {
    if (!c || !c->is_batch) return MWU_ERR_INVALID;
    if (c->batch_last_passes.empty()) return fail(c, MWU_ERR_STATE, "no batch solve yet");
    for (int k = 0; k < c->batch_count; ++k) {
        if (passes) passes[k] = c->batch_last_passes[k];
        if (probes) probes[k] = c->batch_last_probes[k];
    }
    return MWU_OK;
}
