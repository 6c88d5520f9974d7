// Hot-path kernels of one MWU iteration (Alg. 2 with the step-size search of
// Alg. 3 / Sec. 4.2), for T = float (FP32 vectors, FP64 reductions) and
// T = double (plain FP64 form).
//
// Kernel sequence of one iteration (all on one stream, no host round trip):
//   k_dir     per variable: x += alpha_prev d (deferred update of the previous
//             iteration), g = P^T w_p, h = C^T w_c with the weights computed
//             in flight from y, z and the LSE shifts, d = c_d max(0,1-g/h) x,
//             counts of d > 0, dense-row dots.  Last block: d = 0 test, search init.
//   k_cand    per constraint row: (first pass) dv = A d, then K step candidates
//             accumulated with online shifts.  Last block: merge, Psi_k / Phi_k
//             in FP64, next candidates or the accepted alpha.
//   k_update  per constraint row: v += alpha dv with online LSE of the new v.
//             Last block: shifts and sums for the next iteration, stop test.
//
// Reductions: each thread accumulates in T, warps merge with shuffles, blocks
// write one FP64 record, and the last block to finish (threadfence + atomic
// ticket) merges the records in a fixed order.
#include "mwu_internal.cuh"
#include "mwu.h"

#include <cfloat>
#include <cmath>
#include <cstdio>
#include <string>

namespace mwu {

// ---------------------------------------------------------------- math
__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }

// u = 1 - e^{-b} for b >= 0 (the candidate factor of the T sums).  FP32: the
// Taylor series b - b^2/2! + ... - b^8/8! in Horner form for b <= 1/4, whose
// truncation error is below b^9/9! < 1e-10 b; 1 - e^{-b} from the fast
// exponential above, where u >= 0.22 keeps the cancellation below 2^-21
// relative.  FP64: -expm1(-b).
__device__ __forceinline__ float one_minus_exp_neg(float b) {
    b = fmaxf(b, 0.0f);
    float t = 1.0f - b * (1.0f / 8.0f);
    t = 1.0f - b * (1.0f / 7.0f) * t;
    t = 1.0f - b * (1.0f / 6.0f) * t;
    t = 1.0f - b * (1.0f / 5.0f) * t;
    t = 1.0f - b * (1.0f / 4.0f) * t;
    t = 1.0f - b * (1.0f / 3.0f) * t;
    t = 1.0f - b * 0.5f * t;
    const float series = b * t;
    return b <= 0.25f ? series : 1.0f - __expf(-b);
}
__device__ __forceinline__ double one_minus_exp_neg(double b) { return -expm1(-b); }
template <class T> __device__ __forceinline__ T exp_T(double x) { return t_exp((T)x); }
__device__ __forceinline__ float t_log(float x) { return logf(x); }
__device__ __forceinline__ double t_log(double x) { return log(x); }
__device__ __forceinline__ float t_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double t_log1p(double x) { return log1p(x); }
template <class T> __device__ __forceinline__ T t_inf();
template <> __device__ __forceinline__ float t_inf<float>() { return INFINITY; }
template <> __device__ __forceinline__ double t_inf<double>() { return (double)INFINITY; }

template <class T> __device__ __forceinline__ T shfl_x(T v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }

template <class T> __device__ __forceinline__ T group_sum(T v, int G) {
    for (int off = G >> 1; off > 0; off >>= 1) v += shfl_x(v, off);
    return v;
}
template <class T> __device__ __forceinline__ T group_max(T v, int G) {
    for (int off = G >> 1; off > 0; off >>= 1) v = fmax(v, shfl_x(v, off));
    return v;
}

// Block-wide sum (all threads get the result).  smem: >= 32 T.
template <class T> __device__ T block_sum(T v, T *smem) {
    v = group_sum(v, 32);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem[w] = v;
    __syncthreads();
    T r = (threadIdx.x < (blockDim.x >> 5)) ? smem[threadIdx.x] : T(0);
    if (w == 0) r = group_sum(r, 32);
    if (threadIdx.x == 0) smem[0] = r;
    __syncthreads();
    r = smem[0];
    __syncthreads();
    return r;
}
template <class T> __device__ T block_max(T v, T *smem) {
    v = group_max(v, 32);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) smem[w] = v;
    __syncthreads();
    T r = (threadIdx.x < (blockDim.x >> 5)) ? smem[threadIdx.x] : -t_inf<T>();
    if (w == 0) r = group_max(r, 32);
    if (threadIdx.x == 0) smem[0] = r;
    __syncthreads();
    r = smem[0];
    __syncthreads();
    return r;
}

// Online log-sum-exp pair: sum_i exp(sgn*eta*(v_i - s)) with s the running
// max (sgn = +1) or min (sgn = -1).  S == 0 means empty.
template <class T> struct Lse { T s; T S; };

template <class T> __device__ __forceinline__ void lse_push(Lse<T> &a, T v, T eta_sgn, int sgn) {
    if (a.S == T(0)) { a.s = v; a.S = T(1); return; }
    bool up = sgn > 0 ? (v > a.s) : (v < a.s);
    if (up) { a.S = a.S * t_exp(eta_sgn * (a.s - v)) + T(1); a.s = v; }
    else    { a.S += t_exp(eta_sgn * (v - a.s)); }
}
template <class T, class U> __device__ __forceinline__ void lse_merge(Lse<U> &a, U bs, U bS, U eta_sgn, int sgn) {
    if (bS == U(0)) return;
    if (a.S == U(0)) { a.s = bs; a.S = bS; return; }
    U s = sgn > 0 ? fmax(a.s, bs) : fmin(a.s, bs);
    // rescale factors in T precision (FP32 for the fast form), accumulation in U
    U fa = (U)t_exp((T)(eta_sgn * (a.s - s)));
    U fb = (U)t_exp((T)(eta_sgn * (bs - s)));
    a.S = a.S * fa + bS * fb;
    a.s = s;
}

// ---------------------------------------------------------------- record merges
// Per-block records of shifted sums (log-sum-exp sums of Sec. 2.2, candidate
// sums of Sec. 4.1) are merged by one warp per quantity in the last block: the
// common shift M = max_i m_i first, then each sum scaled by e^{c (m_i - M)}
// (or added as it is), accumulated per lane in compensated FP32 (Kahan) and
// combined across the 32 lanes in FP64.  GB300 issues FP64 at a small fraction
// of the FP32 rate, so FP64 is kept to the five steps of the lane tree.  The
// records hold T values (FP32 in the fast form, FP64 in the plain form).
template <class T> __host__ __device__ constexpr int rec_len() { return REC * (int)(sizeof(double) / sizeof(T)); }
template <class T> __device__ __forceinline__ T *rec_of(const double *part, int b) {
    return reinterpret_cast<T *>(const_cast<double *>(part)) + (size_t)b * rec_len<T>();
}

template <class T> __device__ __forceinline__ void kahan_add(T &sum, T &comp, T x) {
    const T y = x - comp;
    const T t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Merges, for each quantity q < nq, the block records b in [b0, b1) given by
// range(q, b0, b1).  get(q, b, m, r, v) reads record b's shift m, its NV sums r
// and (HASMIN) a value v whose minimum is wanted; bit j of scaled(q) marks the
// sums that carry the factor e^{c (m - M)}; records with r[0] = 0 are empty.
// The 8 warps share the quantities (several warps per quantity when nq < 8),
// each lane takes a strided subset of records with the loads unrolled, and
// emit(q, M, tot, vmin) runs once per quantity with the FP64 totals.  Every
// thread of the block must call it (it synchronises).
template <class T, int NV, bool HASMIN, class Range, class Scaled, class Get, class Emit>
__device__ void block_merge_shifted(int nq, T c, Range range, Scaled scaled, Get get, Emit emit) {
    constexpr int NW = BLOCK / 32;
    __shared__ T sm_M[NW], sm_min[NW];
    __shared__ double sm_S[NW][NV];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r0 = 0; r0 < nq; r0 += NW) {
        const int nr = min(NW, nq - r0);
        const int nwc = NW / nr;                       // warps per quantity in this round
        const int qi = w / nwc, sub = w % nwc;
        const bool act = qi < nr;
        const int q = r0 + qi;
        int b0 = 0, b1 = 0;
        if (act) range(q, b0, b1);
        const int first = b0 + sub * 32 + lane, stride = 32 * nwc;
        T M = -t_inf<T>(), vmin = t_inf<T>();
#pragma unroll 4
        for (int b = first; b < b1; b += stride) {
            T m, r[NV], v;
            get(q, b, m, r, v);
            if (r[0] != T(0)) M = fmax(M, m);
            if (HASMIN) vmin = fmin(vmin, v);
        }
        for (int off = 16; off > 0; off >>= 1) {
            M = fmax(M, shfl_x(M, off));
            if (HASMIN) vmin = fmin(vmin, shfl_x(vmin, off));
        }
        if (lane == 0) { sm_M[w] = M; sm_min[w] = vmin; }
        __syncthreads();
        if (act) {
            M = sm_M[qi * nwc];
            vmin = sm_min[qi * nwc];
            for (int j = 1; j < nwc; ++j) {
                M = fmax(M, sm_M[qi * nwc + j]);
                vmin = fmin(vmin, sm_min[qi * nwc + j]);
            }
        }
        T sum[NV], comp[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) { sum[j] = T(0); comp[j] = T(0); }
        const unsigned sc = act ? scaled(q) : 0u;
#pragma unroll 4
        for (int b = first; b < b1; b += stride) {
            T m, r[NV], v;
            get(q, b, m, r, v);
            const T f = (r[0] != T(0)) ? t_exp(c * (m - M)) : T(0);
#pragma unroll
            for (int j = 0; j < NV; ++j) kahan_add(sum[j], comp[j], ((sc >> j) & 1u) ? r[j] * f : r[j]);
        }
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double t = (double)sum[j] - (double)comp[j];
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            if (lane == 0) sm_S[w][j] = t;
        }
        __syncthreads();
        if (act && sub == 0 && lane == 0) {
            double tot[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                tot[j] = 0.0;
                for (int i = 0; i < nwc; ++i) tot[j] += sm_S[qi * nwc + i][j];
            }
            emit(q, M, tot, vmin);
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------- last block
__device__ __forceinline__ bool last_block_done(unsigned int *counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int ticket = atomicAdd(counter, 1u);
        am_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// ---------------------------------------------------------------- row weights
// w_j (unnormalised) = exp(sgn*eta*(v_j - s)) / rdiv_j, and 0 for a dropped
// row (v_j >= hi: a satisfied covering row when they are dropped)
template <class T> struct WeightFn {
    const T *v; const float *rdiv; T eta_sgn; T s; T hi;
    __device__ __forceinline__ T operator()(int64_t j) const {
        const T vj = v[j];
        if (!(vj < hi)) return T(0);
        T w = t_exp(eta_sgn * (vj - s));
        if (rdiv) w /= (T)rdiv[j];
        return w;
    }
    // the weight of a row whose value vj is recomputed rather than loaded (no row bound)
    __device__ __forceinline__ T of_value(T vj) const {
        if (!(vj < hi)) return T(0);
        return t_exp(eta_sgn * (vj - s));
    }
};

// Column of vertex i in the split view of an incidence transpose (CK_SPLIT2,
// built only for a covering side, whose scale is 1, without row bounds):
// the weights of the edges whose first endpoint is i, rows [b1, e1) of the
// stored z (a contiguous stream), plus those of the edges whose second
// endpoint is i, from z_e = x_i + x_u with their first endpoints u listed in
// idx2[q0, q1) (one gather of x each; the side keeps z = x_u + x_v exactly, and
// floating-point addition commutes, so both give the weight of the same z_e).
// Strided over `step` lanes starting at `lane`, four loads in flight.
template <class T, class F>
__device__ __forceinline__ T split_gather(const ColView &cv, int64_t i, int b1, int e1, int q0, int q1, int lane,
                                          int step, const F &w) {
    // z and the endpoint lists are streamed once (evict-first loads), so that
    // x, gathered at random, stays in L2.  Each round issues up to four z loads
    // and four endpoint loads together, then the four x gathers, so a short
    // column costs two dependent memory latencies, not one per entry.
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    const T *z = w.v;
    const T *xx = static_cast<const T *>(cv.xsrc);
    const T xi = __ldg(xx + i);
    for (int kz = b1 + lane, kx = q0 + lane; kz < e1 || kx < q1; kz += 4 * step, kx += 4 * step) {
        T zv[4];
        int ui[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int jz = kz + r * step, jx = kx + r * step;
            zv[r] = jz < e1 ? __ldcs(z + jz) : T(0);
            ui[r] = jx < q1 ? __ldcs(cv.idx2 + jx) : -1;
        }
        T xv[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) xv[r] = ui[r] >= 0 ? __ldg(xx + ui[r]) : T(0);
        T t[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            t[r] = (kz + r * step < e1) ? w.of_value(zv[r]) : T(0);
            if (ui[r] >= 0) t[r] += w.of_value(xi + xv[r]);
        }
        a0 += t[0]; a1 += t[1]; a2 += t[2]; a3 += t[3];
    }
    return (a0 + a1) + (a2 + a3);
}

// Column-view gather for variable i: sum_j A_ji w_j (without the side's scale).
// Simple kinds are computed by lane 0 of the group only.  Unless ALL, a CSR
// column longer than heavy_len gives 0 (the medium and heavy paths take it).
template <class T, bool ALL = false, class F>
__device__ __forceinline__ T col_gather(const ColView &cv, int64_t i, int lane, int G, const F &w, T dense_w) {
    T acc = T(0);
    switch (cv.kind) {
    case CK_CSR: {
        int beg = cv.ptr[i], end = cv.ptr[i + 1];
        if (!ALL && end - beg > cv.heavy_len) return T(0);
        // four independent gathers of v (and their exponentials) in flight per lane
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        int k = beg + lane;
        for (; k + 3 * G < end; k += 4 * G) {
            const int j0 = cv.idx[k], j1 = cv.idx[k + G], j2 = cv.idx[k + 2 * G], j3 = cv.idx[k + 3 * G];
            T t0 = w(j0), t1 = w(j1), t2 = w(j2), t3 = w(j3);
            if (cv.val) {
                t0 *= (T)cv.val[k]; t1 *= (T)cv.val[k + G]; t2 *= (T)cv.val[k + 2 * G]; t3 *= (T)cv.val[k + 3 * G];
            }
            a0 += t0; a1 += t1; a2 += t2; a3 += t3;
        }
        for (; k < end; k += G) {
            T t = w(cv.idx[k]);
            if (cv.val) t *= (T)cv.val[k];
            a0 += t;
        }
        acc = (a0 + a1) + (a2 + a3);
        break;
    }
    case CK_SPLIT2: {
        const int c0 = cv.ptr[i], c1 = cv.ptr[i + 1];
        if (!ALL && c1 - c0 > cv.heavy_len) return T(0);
        const int q0 = cv.ptr2[i], q1 = cv.ptr2[i + 1];
        acc = split_gather<T>(cv, i, c0 - q0, c1 - q1, q0, q1, lane, G, w);
        break;
    }
    case CK_FIXED2:
        if (lane == 0) { int2 e = reinterpret_cast<const int2 *>(cv.idx)[i]; acc = w(e.x) + w(e.y); }
        break;
    case CK_FIXED1:
        if (lane == 0) acc = w(cv.idx[i]);
        break;
    case CK_HALF1:
        if (lane == 0) acc = w(i >> 1);
        break;
    case CK_DENSE1:
        if (lane == 0) acc = (cv.cvec ? (T)cv.cvec[i] : T(1)) * dense_w;
        break;
    default:
        break;
    }
    return acc;
}

// Row-view product for row j: sum_k A_jk x_k (without scale and rdiv).
template <class T>
__device__ __forceinline__ T row_gather(const RowView &rv, int64_t j, int lane, int G, const T *x) {
    T acc = T(0);
    switch (rv.kind) {
    case RK_CSR: {
        int beg = rv.ptr[j], end = rv.ptr[j + 1];
        for (int k = beg + lane; k < end; k += G) {
            T t = x[rv.idx[k]];
            if (rv.val) t *= (T)rv.val[k];
            acc += t;
        }
        break;
    }
    case RK_FIXED2:
        if (lane == 0) { int2 e = reinterpret_cast<const int2 *>(rv.idx)[j]; acc = x[e.x] + x[e.y]; }
        break;
    case RK_PAIRSUM:
        if (lane == 0) acc = x[2 * j] + x[2 * j + 1];
        break;
    default:
        break;
    }
    return acc;
}

// Strided sum over [beg, end) with stride `step`, four independent loads in
// flight per lane: sum_k val[k] * x[idx[k]] (val == nullptr -> ones).
template <class T>
__device__ __forceinline__ T strided_gather(const int32_t *idx, const float *val, const T *x, int beg, int end,
                                            int step) {
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int k = beg;
    for (; k + 3 * step < end; k += 4 * step) {
        const int i0 = idx[k], i1 = idx[k + step], i2 = idx[k + 2 * step], i3 = idx[k + 3 * step];
        T t0 = x[i0], t1 = x[i1], t2 = x[i2], t3 = x[i3];
        if (val) {
            t0 *= (T)val[k]; t1 *= (T)val[k + step]; t2 *= (T)val[k + 2 * step]; t3 *= (T)val[k + 3 * step];
        }
        a0 += t0; a1 += t1; a2 += t2; a3 += t3;
    }
    for (; k < end; k += step) {
        T t = x[idx[k]];
        if (val) t *= (T)val[k];
        a0 += t;
    }
    return (a0 + a1) + (a2 + a3);
}

template <class T, class F>
__device__ T heavy_col_gather(const ColView &cv, int64_t i, const F &w, T *smem) {
    const int beg = cv.ptr[i], end = cv.ptr[i + 1], step = (int)blockDim.x;
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int k = beg + (int)threadIdx.x;
    for (; k + 3 * step < end; k += 4 * step) {
        T t0 = w(cv.idx[k]), t1 = w(cv.idx[k + step]), t2 = w(cv.idx[k + 2 * step]), t3 = w(cv.idx[k + 3 * step]);
        if (cv.val) {
            t0 *= (T)cv.val[k]; t1 *= (T)cv.val[k + step]; t2 *= (T)cv.val[k + 2 * step]; t3 *= (T)cv.val[k + 3 * step];
        }
        a0 += t0; a1 += t1; a2 += t2; a3 += t3;
    }
    for (; k < end; k += step) {
        T t = w(cv.idx[k]);
        if (cv.val) t *= (T)cv.val[k];
        a0 += t;
    }
    return block_sum((a0 + a1) + (a2 + a3), smem);
}

// (A x)_j = coef_j * sum_k val_jk x_k with coef_j = scale / rdiv_j; the scale
// (1/M of the objective row, 1/D of O) lives in device state so that a captured
// iteration stays valid when the probe target changes.
// (scale arrives in T: GB300 runs double-to-float conversions on its FP64
// pipe, so the callers convert once per thread, not once per element)
template <class T> __device__ __forceinline__ T row_coef(const Side<T> &sd, int64_t j, T scale) {
    return sd.rv.rdiv ? scale / (T)sd.rv.rdiv[j] : scale;
}

// T copies of the device-state scalars of the sweep kernels, made once per
// block by one thread: GB300 runs FP64 arithmetic and double/float
// conversions on a narrow pipe, so no thread repeats them.  Every thread of
// the block must call it (it synchronises).
template <class T> struct SweepConsts {
    T eta, s0, s1, fp, fc, kgh, cd, thr, scale0, scale1, alpha_prev, alpha_acc;
    T hi;   // covering rows with z_j >= hi are dropped (+inf: every row is kept)
};
template <class T> __device__ __forceinline__ SweepConsts<T> sweep_consts(const DevState *st) {
    __shared__ SweepConsts<T> c;
    if (threadIdx.x == 0) {
        const double fp = st->scale[0] / st->S[0], fc = st->scale[1] / st->S[1];
        c.eta = (T)st->eta;
        c.s0 = (T)st->s[0];
        c.s1 = (T)st->s[1];
        c.fp = (T)fp;
        c.fc = (T)fc;
        c.kgh = (T)(fp / fc);
        c.cd = (T)st->c_d;
        c.thr = (T)(1.0 - st->grad_tol);   // gradient test threshold on g/h
        c.scale0 = (T)st->scale[0];
        c.scale1 = (T)st->scale[1];
        c.alpha_prev = st->pending ? (T)st->alpha_acc : T(0);
        c.alpha_acc = (T)st->alpha_acc;
        c.hi = (T)st->act_hi;
    }
    __syncthreads();
    return c;
}

// ============================================================ x initialisation
// a0: x_i = eps / (n ||P_{:,i}||_inf) (Alg. 1), and the dense-row dots c^T x.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_x_prep(Problem<T> p, const void *xin, int fp64, int mode) {
    __shared__ double sm_d[32];
    const Side<T> &P = p.side[0];
    const double eps = p.st->eps;
    double dot[2] = {0.0, 0.0};
    // implicit column views without bounds (and a dense row without weights)
    // have every column norm equal to the side's scale: x0 is one value,
    // computed once per thread
    const ColView &cv0 = P.cv;
    const bool uniform = !cv0.rdiv && (cv0.kind == CK_FIXED1 || cv0.kind == CK_FIXED2 || cv0.kind == CK_HALF1 ||
                                       (cv0.kind == CK_DENSE1 && !cv0.cvec));
    const double s0 = p.st->scale[0] > 0.0 ? p.st->scale[0] : 1.0;
    const T x_uniform = (T)(eps / ((double)p.n * s0));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x) {
        T xi;
        if (mode == 0 && uniform) {
            xi = x_uniform;
        } else if (mode == 0) {
            double cm = 0.0;
            const ColView &cv = P.cv;
            switch (cv.kind) {
            case CK_CSR:
                for (int k = cv.ptr[i]; k < cv.ptr[i + 1]; ++k) {
                    double a = (cv.val ? (double)cv.val[k] : 1.0) / (cv.rdiv ? (double)cv.rdiv[cv.idx[k]] : 1.0);
                    cm = fmax(cm, a);
                }
                break;
            case CK_FIXED2: {
                int2 e = reinterpret_cast<const int2 *>(cv.idx)[i];
                double a = cv.rdiv ? 1.0 / (double)cv.rdiv[e.x] : 1.0;
                double b = cv.rdiv ? 1.0 / (double)cv.rdiv[e.y] : 1.0;
                cm = fmax(a, b);
                break;
            }
            case CK_FIXED1: cm = cv.rdiv ? 1.0 / (double)cv.rdiv[cv.idx[i]] : 1.0; break;
            case CK_HALF1: cm = cv.rdiv ? 1.0 / (double)cv.rdiv[i >> 1] : 1.0; break;
            case CK_DENSE1: cm = cv.cvec ? (double)cv.cvec[i] : 1.0; break;
            default: cm = 1.0;
            }
            cm *= p.st->scale[0];
            if (!(cm > 0.0)) cm = 1.0;
            xi = (T)(eps / ((double)p.n * cm));
        } else {
            xi = fp64 ? (T)((const double *)xin)[i] : (T)((const float *)xin)[i];
        }
        p.x[i] = xi;
        for (int s = 0; s < 2; ++s)
            if (p.side[s].cv.kind == CK_DENSE1)
                dot[s] += (double)(p.side[s].cv.cvec ? (T)p.side[s].cv.cvec[i] : T(1)) * (double)xi;
    }
    double t0 = block_sum(dot[0], sm_d);
    double t1 = block_sum(dot[1], sm_d);
    if (threadIdx.x == 0) {
        p.part_var[blockIdx.x * REC + 0] = t0;
        p.part_var[blockIdx.x * REC + 1] = t1;
    }
}

// ============================================================ finalisation helpers
// Merge per-block LSE records of the row kernels plus dense-row values and set
// s, S, ymax, zmin and the stop status (Alg. 2 loop test, see the oracle).
template <class T>
__device__ void finalize_reductions(Problem<T> &p, int gP, int nb_row, int nb_var, bool dense_from_var, double alpha) {
    // LSE block records (float view of part_row): [0] shift s_b, [1] S_b;
    // side 0 in blocks [0, gP), side 1 in [gP, nb_row).  Warp s merges side s
    // on the sign-adjusted shift sg * s_b.
    static_assert(BLOCK == 256, "merge layout assumes 256 threads");
    DevState *st = p.st;
    __shared__ double sh_fin[2][3];
    __shared__ double sh_d[32];
    block_merge_shifted<T, 1, true>(
        2, (T)st->eta,
        [&](int q, int &b0, int &b1) { b0 = q == 0 ? 0 : gP; b1 = q == 0 ? gP : nb_row; },
        [&](int) { return 1u; },
        [&](int q, int b, T &m, T (&r)[1], T &v) {
            const T *o = rec_of<T>(p.part_row, b);
            m = p.side[q].sign > 0 ? o[0] : -o[0];   // sign-adjusted shift: the merge takes the max
            r[0] = o[1];
            v = o[2];
        },
        [&](int q, T M, const double (&tot)[1], T vmin) {
            sh_fin[q][0] = p.side[q].sign > 0 ? (double)M : -(double)M;
            sh_fin[q][1] = tot[0];
            sh_fin[q][2] = (double)vmin;
        });
    double dense[2] = {0.0, 0.0};
    if (dense_from_var) {
        double d0 = 0.0, d1 = 0.0;
        for (int b = threadIdx.x; b < nb_var; b += blockDim.x) {
            d0 += p.part_var[(size_t)b * REC + 0];
            d1 += p.part_var[(size_t)b * REC + 1];
        }
        dense[0] = block_sum(d0, sh_d);
        dense[1] = block_sum(d1, sh_d);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool bad = false;
        const bool drop = isfinite(st->act_hi);
        for (int s = 0; s < 2; ++s) {
            const Side<T> &sd = p.side[s];
            if (sd.rv.kind == RK_DENSE1) {
                if (dense_from_var) st->dense_v[s] = st->scale[s] * dense[s];
                else st->dense_v[s] += alpha * st->dense_dv[s];
                st->s[s] = st->dense_v[s];
                st->S[s] = 1.0;
            } else {
                st->s[s] = sh_fin[s][0];
                st->S[s] = sh_fin[s][1];
                if (s == 1 && drop && !(st->S[1] > 0.0)) {
                    // every covering row dropped (all satisfied): the sums are
                    // empty and the stopping test below ends the probe
                    st->s[1] = sh_fin[1][2];
                    st->S[1] = 1.0;
                }
            }
            if (!isfinite(st->s[s]) || !isfinite(st->S[s]) || !(st->S[s] > 0.0)) bad = true;
            st->lnS[s] = (double)t_log((T)st->S[s]);
            st->invS[s] = 1.0 / st->S[s];
        }
        st->ymax = st->s[0];
        // min z over every row: with dropped rows the shift of the sums is the
        // minimum over the active rows only
        st->zmin = (drop && p.side[1].rv.kind != RK_DENSE1) ? sh_fin[1][2] : st->s[1];
        // compacted rows: the dropped ones (z >= act_hi) are no longer read, so
        // act_hi bounds their minimum; exact while an active row is below it,
        // and the end of the call re-decides a probe that stopped on the bound
        if (p.side[1].orig) st->zmin = fmin(st->zmin, st->act_hi);
        if (bad) {
            st->status = ST_NUMERIC;
            st->numeric_bad = 1;
        } else if (st->status == ST_RUNNING) {
            double eps = st->eps;
            if (st->ratio_stop > 0.0 && st->zmin > 0.0 && st->ymax <= st->ratio_stop * st->zmin) {
                st->status = ST_FEASIBLE;   // x / zmin is a (ratio_stop)-relative solution
                st->reason = RS_RATIO;
            } else if (st->zmin >= 1.0 || st->ymax > 1.0 + eps) {
                if (st->ymax <= (1.0 + eps) * st->zmin) { st->status = ST_FEASIBLE; st->reason = RS_COVERED; }
                else { st->status = ST_INFEASIBLE; st->reason = RS_PACKING; }
            } else if (st->iter >= st->max_iter) {
                st->status = ST_MAX_ITER;
                st->reason = RS_MAXITER;
            }
        }
    }
}

// End of a block's LSE accumulation: warps in T, then an 8-lane tree over the
// warps in T, then one record [shift, S, vmin] per block; vmin is the plain
// minimum over every row the block saw (dropped covering rows included).
template <class T>
__device__ void lse_block_record(const Problem<T> &p, Lse<T> acc, T eta_sgn, int sgn, T vmin) {
    for (int off = 16; off > 0; off >>= 1) {
        T os = shfl_x(acc.s, off), oS = shfl_x(acc.S, off);
        lse_merge<T, T>(acc, os, oS, eta_sgn, sgn);
        vmin = fmin(vmin, shfl_x(vmin, off));
    }
    __shared__ T ws[BLOCK / 32], wS[BLOCK / 32], wm[BLOCK / 32];
    if ((threadIdx.x & 31) == 0) {
        ws[threadIdx.x >> 5] = acc.s;
        wS[threadIdx.x >> 5] = acc.S;
        wm[threadIdx.x >> 5] = vmin;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        Lse<T> q{ws[threadIdx.x & 7], wS[threadIdx.x & 7]};
        T mn = wm[threadIdx.x & 7];
        for (int off = 4; off > 0; off >>= 1) {
            T os = shfl_x(q.s, off), oS = shfl_x(q.S, off);
            lse_merge<T, T>(q, os, oS, eta_sgn, sgn);
            mn = fmin(mn, shfl_x(mn, off));
        }
        if (threadIdx.x == 0) {
            T *rec = rec_of<T>(p.part_row, blockIdx.x);
            rec[0] = q.s;
            rec[1] = q.S;
            rec[2] = mn;
        }
    }
}

// Condition of the step-search loop of a captured iteration: 1 while the
// search of this iteration has passes left.  Each kernel that sets it does so
// from one thread, once per launch.
__device__ __forceinline__ unsigned search_continues(const DevState *st) {
    return (st->status == ST_RUNNING && st->phase != PH_DONE) ? 1u : 0u;
}

// ============================================================ gradient + direction
// End of the direction step (one thread): d = 0 -> INFEASIBLE (Alg. 2), else the
// step-size search starts (Alg. 3: alpha = 1, or the warm start).
__device__ void dir_finish(DevState *st, double np_t, double dd0, double dd1) {
    st->n_pos = (long long)np_t;
    st->dense_dv[0] = st->scale[0] * dd0;
    st->dense_dv[1] = st->scale[1] * dd1;
    if (np_t <= 0.0) {
        st->status = ST_INFEASIBLE;
        st->reason = RS_DZERO;
        st->phase = PH_DONE;
        return;
    }
    st->phase = PH_EXP;
    st->lb = 0.0;
    st->ub = (double)INFINITY;
    st->passes = 0;
    st->early = 0;
    st->alpha_acc = 0.0;
    st->kpass = st->K;
    st->newton_steps = 0;
    st->loop_guard = 0;
    int b0 = 0;
    if (st->warm_start && st->alpha_prev >= 1.0 && st->step_mode != 3) b0 = (int)floor(log2(st->alpha_prev));
    st->b = b0;
    for (int k = 0; k < st->K; ++k) st->alpha[k] = ldexp(1.0, b0 + k);
    if (st->step_mode == 3 && st->alpha_prev >= 1.0) {   // Newton, warm start (Sec. 4.2)
        st->phase = PH_NEWTON;
        st->kpass = 1;
        st->alpha[0] = st->alpha_prev;
    }
    if (st->step_mode == 2) {   // standard step alpha = 1 (Alg. 1)
        st->phase = PH_DONE;
        st->alpha_acc = 1.0;
    }
}


// Heavy columns of a CK_SPLIT2 covering side: one warp per SEG_LEN-entry
// segment of the combined column (first-endpoint rows of z, then the x list of
// the second-endpoint edges), one partial sum each; k_dir adds a heavy
// variable's partials in segment order.  Balances the hub vertices of
// power-law graphs over the whole grid.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_split_seg(Problem<T> p, int potential_mode) {
    DevState *st = p.st;
    if (!potential_mode && st->status != ST_RUNNING) return;
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    const Side<T> &C = p.side[1];
    const ColView &cv = C.cv;
    WeightFn<T> wc{C.v, nullptr, -K0.eta, K0.s1, potential_mode ? t_inf<T>() : K0.hi};
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < cv.n_cseg; q += nw) {
        const int i = cv.cseg_var[q];
        const int c0 = cv.ptr[i], c1 = cv.ptr[i + 1], q0 = cv.ptr2[i], q1 = cv.ptr2[i + 1];
        const int cz = c0 + ((c1 - q1) - (c0 - q0));   // combined index where the x list starts
        const int kb = cv.cseg_beg[q], ke = min(kb + SPLIT_SEG, c1);
        const int zb = (c0 - q0) + (min(max(kb, c0), cz) - c0), ze = (c0 - q0) + (min(ke, cz) - c0);
        const int xb = q0 + (max(kb, cz) - cz), xe = q0 + (max(ke, cz) - cz);
        T sum = split_gather<T>(cv, i, zb, max(zb, ze), xb, max(xb, xe), lane, 32, wc);
        sum = group_sum(sum, 32);
        if (lane == 0) p.cseg_part[q] = sum;
    }
}

// a4, a5 with the deferred x update of the previous iteration fused in.
template <class T>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 4 ? 6 : 4) k_dir(Problem<T> p, int keep_gh, int potential_mode, float *grad_obj) {
    __shared__ T sm[32];
    __shared__ double smd[32];
    DevState *st = p.st;
    if (!potential_mode && st->status != ST_RUNNING && !st->pending) return;
    const bool running = potential_mode || st->status == ST_RUNNING;
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    const T alpha_prev = K0.alpha_prev;
    const Side<T> &P = p.side[0];
    const Side<T> &C = p.side[1];
    WeightFn<T> wp{P.v, P.rv.rdiv, K0.eta, K0.s0, t_inf<T>()};
    // the potential of Sec. 4.1 always takes every row
    WeightFn<T> wc{C.v, C.rv.rdiv, -K0.eta, K0.s1, potential_mode ? t_inf<T>() : K0.hi};
    // h from k_h_scatter's sums (read once and cleared for the next iteration)
    T *const hacc = potential_mode ? nullptr : p.hacc;
    const T fp = K0.fp, fc = K0.fc, cd = K0.cd, thr = K0.thr;
    int npos = 0;   // positives of this thread
    T dense_dot[2] = {T(0), T(0)}, dense_cmp[2] = {T(0), T(0)};   // compensated per thread

    auto finish = [&](int64_t i, T sg, T sh) {
        T xi = p.x[i];
        if (alpha_prev != T(0)) { xi += alpha_prev * p.d[i]; p.x[i] = xi; }
        if (!running) return;
        T g = sg * fp, h = sh * fc;
        if (potential_mode) {
            p.d[i] = g - h;   // d holds the potential gradient in this mode
            if (grad_obj) {
                for (int s = 0; s < 2; ++s)
                    if (p.side[s].cv.kind == CK_DENSE1)
                        grad_obj[i] = (float)((double)p.side[s].sign * st->scale[s] * (double)xi);
            }
            return;
        }
        T di = (g < thr * h) ? cd * (T(1) - g / h) * xi : T(0);
        p.d[i] = di;
        if (keep_gh) { p.g[i] = g; p.h[i] = h; }
        npos += (di > T(0));
        for (int s = 0; s < 2; ++s)
            if (p.side[s].cv.kind == CK_DENSE1)
                kahan_add(dense_dot[s], dense_cmp[s], (p.side[s].cv.cvec ? (T)p.side[s].cv.cvec[i] : T(1)) * di);
    };

    // heavy split columns (P without CSR columns): their segment partials,
    // a warp per variable, added in segment order by the fixed shuffle tree
    const bool split_heavy = C.cv.kind == CK_SPLIT2 && P.cv.kind != CK_CSR && !hacc;
    if (split_heavy) {
        const int wl = threadIdx.x & 31;
        const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t hh = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; hh < p.n_heavy_var; hh += nw) {
            const int64_t i = p.heavy_var[hh];
            T a = T(0);
            for (int q = C.cv.cseg_first[hh] + wl; q < C.cv.cseg_first[hh + 1]; q += 32) a += p.cseg_part[q];
            a = group_sum(a, 32);
            T sg = col_gather<T, true>(P.cv, i, wl, 32, wp, T(1));
            sg = group_sum(sg, 32);
            if (wl == 0) finish(i, sg, a);
        }
    }
    // heavy variables (long CSR columns): whole block
    for (int hh = split_heavy ? p.n_heavy_var : blockIdx.x; hh < p.n_heavy_var; hh += gridDim.x) {
        int64_t i = p.heavy_var[hh];
        T sg, sh;
        if (P.cv.kind == CK_CSR) sg = heavy_col_gather<T>(P.cv, i, wp, sm);
        else { sg = col_gather<T>(P.cv, i, threadIdx.x, 1 << 30, wp, T(1)); sg = block_sum(threadIdx.x == 0 ? sg : T(0), sm); }
        if (hacc) { sh = hacc[i]; }
        else if (C.cv.kind == CK_CSR) sh = heavy_col_gather<T>(C.cv, i, wc, sm);
        else if (C.cv.kind == CK_SPLIT2) {
            // the segments' partial sums (k_split_seg), added in a fixed order
            T a = T(0);
            for (int q = C.cv.cseg_first[hh] + (int)threadIdx.x; q < C.cv.cseg_first[hh + 1]; q += (int)blockDim.x)
                a += p.cseg_part[q];
            sh = block_sum(a, sm);
        }
        else { sh = col_gather<T>(C.cv, i, threadIdx.x, 1 << 30, wc, T(1)); sh = block_sum(threadIdx.x == 0 ? sh : T(0), sm); }
        if (threadIdx.x == 0) {
            if (hacc) hacc[i] = T(0);
            finish(i, sg, sh);
        }
    }
    {   // medium variables: a warp each (warp-uniform loop)
        const int wl = threadIdx.x & 31;
        const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < p.n_med_var; q += nw) {
            const int64_t i = p.med_var[q];
            T sg = col_gather<T, true>(P.cv, i, wl, 32, wp, T(1));
            T sh = hacc ? (wl == 0 ? hacc[i] : T(0)) : col_gather<T, true>(C.cv, i, wl, 32, wc, T(1));
            sg = group_sum(sg, 32);
            sh = group_sum(sh, 32);
            if (wl == 0) {
                if (hacc) hacc[i] = T(0);
                finish(i, sg, sh);
            }
        }
    }
    if (p.n_light_var >= 0) {   // split view: tiny columns one thread each
        const int64_t nt = (int64_t)gridDim.x * blockDim.x;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p.n_tiny_var; q += nt) {
            const int64_t i = p.tiny_var[q];
            const T sg = col_gather<T, true>(P.cv, i, 0, 1, wp, T(1));
            const T sh = col_gather<T, true>(C.cv, i, 0, 1, wc, T(1));
            finish(i, sg, sh);
        }
    }
    int G = p.G_var, lane = threadIdx.x & (G - 1);
    int64_t per_block = blockDim.x / G;
    int64_t stride = (int64_t)gridDim.x * per_block;
    int64_t warp_base = (int64_t)blockIdx.x * per_block + (threadIdx.x & ~31) / G;
    const bool listed = p.n_light_var >= 0;
    const int64_t n_loop = listed ? p.n_light_var : p.n;
    for (int64_t base = warp_base; base < n_loop; base += stride) {
        const int64_t q = base + (threadIdx.x & 31) / G;
        bool live = q < n_loop;
        const int64_t i = (listed && live) ? (int64_t)p.light_var[q] : q;
        T sg = T(0), sh = T(0);
        bool heavy = false;
        if (live) {
            heavy = ((P.cv.kind == CK_CSR || P.cv.kind == CK_SPLIT2) && P.cv.ptr[i + 1] - P.cv.ptr[i] > P.cv.heavy_len) ||
                    ((C.cv.kind == CK_CSR || C.cv.kind == CK_SPLIT2) && C.cv.ptr[i + 1] - C.cv.ptr[i] > C.cv.heavy_len);
            if (!heavy) {
                sg = col_gather<T>(P.cv, i, lane, G, wp, T(1));
                sh = hacc ? (lane == 0 ? hacc[i] : T(0)) : col_gather<T>(C.cv, i, lane, G, wc, T(1));
            }
        }
        sg = group_sum(sg, G);
        sh = group_sum(sh, G);
        if (live && lane == 0 && !heavy) {
            if (hacc) hacc[i] = T(0);
            finish(i, sg, sh);
        }
    }
    if (potential_mode) return;
    // block partials: n_pos, dense dots
    double np = block_sum((double)npos, smd);
    double d0 = block_sum((double)dense_dot[0] - (double)dense_cmp[0], smd);
    double d1 = block_sum((double)dense_dot[1] - (double)dense_cmp[1], smd);
    if (threadIdx.x == 0) {
        double *rec = p.part_var + (size_t)blockIdx.x * REC;
        rec[0] = np; rec[1] = d0; rec[2] = d1;
    }
    if (last_block_done(&st->counter[1])) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
            const double *rec = p.part_var + (size_t)b * REC;
            a0 += rec[0]; a1 += rec[1]; a2 += rec[2];
        }
        double np_t = block_sum(a0, smd);
        double dd[2] = {block_sum(a1, smd), block_sum(a2, smd)};
        if (threadIdx.x == 0) {
            if (st->pending) {   // the deferred update of x is now applied
                st->pending = 0;
            }
            if (running) dir_finish(st, np_t, dd[0], dd[1]);
            st->counter[1] = 0;
            if (p.cond_on) cudaGraphSetConditional(p.cond, search_continues(st));
        }
    }
}

// ------------------------------------------------------------ h by edge scatter
// h for a covering side whose rows are the edges (u, v) of an incidence
// transpose (vertex cover, M^T x >= 1): one stream over the edges, each
// adding its weight w_e = e^{-eta (z_e - s_c)} / rdiv_e to hacc[u] and hacc[v]
// with atomic adds, instead of gathering z over every vertex's incident edges.
// Runs of equal u in a warp (edge lists sorted by u) are summed with shuffles
// first, so they cost one atomic each.  The sums' order depends on scheduling
// (the option trades determinism for speed); k_dir reads and clears them.
// A CSR covering side (explicit C, dominating set) scatters row j's weight
// w_j val_jk into hacc[k] over the row's entries, with the SpMV's length bins
// (a thread per short row, MED_LANES lanes per medium row, a warp per segment
// of a long row).
template <class T>
__device__ void h_scatter_csr(const Problem<T> &p, T eta, T sc, T hi) {
    const Side<T> &C = p.side[1];
    const RowView &rv = C.rv;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
    auto wt = [&](int64_t j) -> T {
        const T z = C.v[j];
        if (!(z < hi)) return T(0);
        T w = t_exp(-eta * (z - sc));
        if (rv.rdiv) w /= (T)rv.rdiv[j];
        return w;
    };
    auto put = [&](int k, T w) { atomicAdd(&p.hacc[rv.idx[k]], rv.val ? w * (T)rv.val[k] : w); };
    {   // segments of long rows: a warp each
        const int lane = threadIdx.x & 31;
        for (int64_t i = tid >> 5; i < rv.n_seg; i += nthr >> 5) {
            const int j = rv.seg_row[i];
            const T w = wt(j);
            if (w == T(0)) continue;
            const int ke = min(rv.seg_beg[i] + SEG_LEN, rv.ptr[j + 1]);
            for (int k = rv.seg_beg[i] + lane; k < ke; k += 32) put(k, w);
        }
    }
    {   // medium rows: MED_LANES lanes each
        const int lane = threadIdx.x & (MED_LANES - 1);
        for (int64_t i = tid / MED_LANES; i < rv.n_med; i += nthr / MED_LANES) {
            const int j = rv.med_rows[i];
            const T w = wt(j);
            if (w == T(0)) continue;
            for (int k = rv.ptr[j] + lane; k < rv.ptr[j + 1]; k += MED_LANES) put(k, w);
        }
    }
    for (int64_t i = tid; i < rv.n_short; i += nthr) {   // short rows: a thread each
        const int j = rv.short_rows[i];
        const T w = wt(j);
        if (w == T(0)) continue;
        for (int k = rv.ptr[j]; k < rv.ptr[j + 1]; ++k) put(k, w);
    }
}

template <class T>
__global__ void __launch_bounds__(BLOCK) k_h_scatter(Problem<T> p) {
    DevState *st = p.st;
    if (st->status != ST_RUNNING) return;
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    const Side<T> &C = p.side[1];
    const T eta = K0.eta, sc = K0.s1, hi = K0.hi;
    if (C.rv.kind == RK_CSR) {
        h_scatter_csr(p, eta, sc, hi);
        return;
    }
    const int2 *ends = reinterpret_cast<const int2 *>(C.rv.idx);
    const int lane = threadIdx.x & 31;
    const int64_t m = C.m, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < m; e0 += stride) {   // warp-uniform
        const int64_t e = e0 + lane;
        const bool live = e < m;
        T w = T(0);
        int2 uv = make_int2(-1, -1);
        if (live) {
            uv = ends[e];
            const T z = C.v[e];
            if (z < hi) {
                w = t_exp(-eta * (z - sc));
                if (C.rv.rdiv) w /= (T)C.rv.rdiv[e];
            }
        }
        // segmented inclusive sum over runs of equal u (lanes in order)
        const int u = uv.x;
        const int u_prev = __shfl_up_sync(0xffffffffu, u, 1);
        const bool head = lane == 0 || u_prev != u;
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        // first lane of this lane's run: the highest head at or below it
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        T run = w;
        for (int off = 1; off < 32; off <<= 1) {
            const T o = __shfl_up_sync(0xffffffffu, run, off);
            if (lane - off >= start) run += o;
        }
        const int u_next = __shfl_down_sync(0xffffffffu, u, 1);
        const bool tail = lane == 31 || u_next != u;
        if (live && tail && run != T(0)) atomicAdd(&p.hacc[u], run);
        if (live && w != T(0)) atomicAdd(&p.hacc[uv.y], w);
    }
}

// ------------------------------------------------------------ k_dir, pair matrices
// The densest-subgraph LP (Sec. 3, Eq. densest_linalg): variable slots 2e, 2e+1
// of edge e sit in packing rows u_e, v_e of O (column view FIXED1 over the edge
// list) and both in covering row e of W (HALF1).  One thread takes both slots:
// one covering weight per edge, two packing weights, 8-byte loads of x, d and
// the endpoints.  Same arithmetic as the generic k_dir per slot.
template <class T>
__global__ void __launch_bounds__(BLOCK, 4) k_dir_pairs(Problem<T> p) {
    __shared__ double smd[32];
    DevState *st = p.st;
    if (st->status != ST_RUNNING && !st->pending) return;
    const bool running = st->status == ST_RUNNING;
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    const T alpha_prev = K0.alpha_prev;
    const Side<T> &P = p.side[0];
    const Side<T> &C = p.side[1];
    const T eta = K0.eta, sp = K0.s0, sc = K0.s1, cd = K0.cd, thr = K0.thr, hi = K0.hi;
    const int64_t E = p.n >> 1;
    const int2 *ends = reinterpret_cast<const int2 *>(P.cv.idx);
    int npos = 0;   // positives of this thread
    // Per slot the test and the step need only r = g/h = (fp/fc) w_p[u] / w_c[e]
    // = (fp/fc) exp(eta (y_u - s_p) + eta (z_e - s_c)) (times rdiv_e / rdiv_u
    // with bounds): one exponential per slot and no division.
    const T kgh = K0.kgh;
    const T scale_c = K0.scale1;
    auto one_edge = [&](int64_t e, const int2 uv, T x0, T x1, T yu, T yv, T ze) {
        const T bz = eta * (ze - sc);
        T r0 = kgh * t_exp(eta * (yu - sp) + bz);
        T r1 = kgh * t_exp(eta * (yv - sp) + bz);
        if (P.rv.rdiv || C.rv.rdiv) {
            const T re = C.rv.rdiv ? (T)C.rv.rdiv[e] : T(1);
            r0 *= re / (P.rv.rdiv ? (T)P.rv.rdiv[uv.x] : T(1));
            r1 *= re / (P.rv.rdiv ? (T)P.rv.rdiv[uv.y] : T(1));
        }
        // a dropped covering row (z_e >= hi) gives h = 0 on both slots: d = 0
        const bool live = ze < hi;
        const T d0 = (live && r0 < thr) ? cd * (T(1) - r0) * x0 : T(0);
        const T d1 = (live && r1 < thr) ? cd * (T(1) - r1) * x1 : T(0);
        if (sizeof(T) == 4) reinterpret_cast<float2 *>(p.d)[e] = make_float2((float)d0, (float)d1);
        else { p.d[2 * e] = d0; p.d[2 * e + 1] = d1; }
        C.dv[e] = (d0 + d1) * row_coef(C, e, scale_c);   // a6 for W: dz_e = d_{2e} + d_{2e+1}
        npos += (d0 > T(0)) + (d1 > T(0));
    };
    auto load_x = [&](int64_t e, T &x0, T &x1) {
        if (sizeof(T) == 4) {
            float2 xx = reinterpret_cast<const float2 *>(p.x)[e];
            x0 = xx.x; x1 = xx.y;
            if (alpha_prev != T(0)) {
                float2 dd = reinterpret_cast<const float2 *>(p.d)[e];
                x0 += alpha_prev * dd.x; x1 += alpha_prev * dd.y;
                reinterpret_cast<float2 *>(p.x)[e] = make_float2((float)x0, (float)x1);
            }
        } else {
            x0 = p.x[2 * e]; x1 = p.x[2 * e + 1];
            if (alpha_prev != T(0)) {
                x0 += alpha_prev * p.d[2 * e]; x1 += alpha_prev * p.d[2 * e + 1];
                p.x[2 * e] = x0; p.x[2 * e + 1] = x1;
            }
        }
    };
    // four edges per lane and iteration: the streamed loads of all four are
    // issued before the dependent gathers of y
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; e + (U - 1) * stride < E; e += U * stride) {
        T x0[U], x1[U], z[U];
        int2 uv[U];
#pragma unroll
        for (int j = 0; j < U; ++j) load_x(e + j * stride, x0[j], x1[j]);
        if (!running) continue;
#pragma unroll
        for (int j = 0; j < U; ++j) { uv[j] = ends[e + j * stride]; z[j] = C.v[e + j * stride]; }
        T yu[U], yv[U];
#pragma unroll
        for (int j = 0; j < U; ++j) { yu[j] = P.v[uv[j].x]; yv[j] = P.v[uv[j].y]; }
#pragma unroll
        for (int j = 0; j < U; ++j) one_edge(e + j * stride, uv[j], x0[j], x1[j], yu[j], yv[j], z[j]);
    }
    for (; e < E; e += stride) {
        T x0, x1;
        load_x(e, x0, x1);
        if (!running) continue;
        const int2 uv = ends[e];
        one_edge(e, uv, x0, x1, P.v[uv.x], P.v[uv.y], C.v[e]);
    }
    const double np = block_sum((double)npos, smd);
    if (threadIdx.x == 0) {
        double *rec = p.part_var + (size_t)blockIdx.x * REC;
        rec[0] = np; rec[1] = 0.0; rec[2] = 0.0;
    }
    if (last_block_done(&st->counter[1])) {
        double a0 = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a0 += p.part_var[(size_t)b * REC];
        const double np_t = block_sum(a0, smd);
        if (threadIdx.x == 0) {
            st->pending = 0;
            if (running) dir_finish(st, np_t, 0.0, 0.0);
            st->counter[1] = 0;
            if (p.cond_on) cudaGraphSetConditional(p.cond, search_continues(st));
        }
    }
}

// ============================================================ step candidates
// Per-thread accumulators of K candidates for one side.
template <class T> struct CandAcc {
    T mx[KMAX], R[KMAX], Tt[KMAX], zm[KMAX];
    T mxmin;   // min_k mx[k] (covering side), maintained on rescale
    T D;       // Newton pass: sum dv e^{x_0 - mx_0}, scaled like R[0]
};

template <class T>
__device__ __forceinline__ void cand_init(CandAcc<T> &c, int sgn) {
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        c.mx[k] = sgn > 0 ? T(0) : -t_inf<T>();
        c.R[k] = T(0); c.Tt[k] = T(0); c.zm[k] = t_inf<T>();
    }
    c.mxmin = sgn > 0 ? T(0) : -t_inf<T>();
    c.D = T(0);
}

// Candidate schedule of one pass (identical for every row).
//   mode 0: alpha_{k+1} = 2 alpha_k          (exponential phase of the search)
//   mode 1: alpha_{k+1} = alpha_k + delta    (refinement on [lb, ub])
//   mode 2: arbitrary alphas                 (mwu_eval_candidates, the backoff)
//   mode 3: one alpha, with the sums of Psi'(alpha), Phi'(alpha) (Newton)
// ca[k] = alpha_k eta, al[k] = alpha_k, cd = delta eta, all in T.
template <class T> struct CandSched {
    int K, mode;
    T ca[KMAX], al[KMAX];
    T cd;
    T hi;   // covering rows with v >= hi are dropped (+inf: all kept)
};

// Largest alpha_k eta of a schedule: the search's schedules ascend, but the
// candidates of an external evaluation come in any order.
template <class T> __device__ __forceinline__ T sched_camax(const T *ca, int K) {
    T m = ca[0];
#pragma unroll
    for (int k = 1; k < KMAX; ++k)
        if (k < K) m = fmax(m, ca[k]);
    return m;
}

__device__ __forceinline__ float fast_exp(float x) { return __expf(x); }
__device__ __forceinline__ double fast_exp(double x) { return exp(x); }

// One row (v, dv) of a side, all K candidates.  With b_k = alpha_k eta dv and
// u_k = 1 - exp(-b_k) (cancellation free):
//   packing (sgn = +1), x_k = eta (y - s_p) + b_k:
//     R_k += exp(x_k - mx_k)            T_k += exp(x_k - mx_k) u_k
//     (T is R - S without cancellation: sum e^{eta(y - s)} expm1(b_k), shifted)
//   covering (sgn = -1), x_k = -eta (z - s_c) - b_k:
//     R_k += exp(x_k - mx_k)            T_k += exp(-eta (z - s_c)) u_k (unshifted, <= S_c)
//     zm_k = min(zm_k, z + alpha_k dz)
// u_k comes from one expm1 per row and an exact recurrence along the schedule:
// doubling b gives u' = u (2 - u); adding delta eta dv gives u' = u + u_d (1 - u).
// mx_k is a running max per thread (rescale on a new max); exp of arguments
// <= 0 uses the __expf intrinsic in FP32 (error 2 + 1.2|x| ulp, and terms with
// large |x| are negligible in the sums).
// Exponent margin below which a term is dropped: exp(-NEGL) ~ 1.8e-35 relative
// to the running shift, beyond FP32 resolution (and FP64 never drops: NEGL_D).
template <class T> __device__ __forceinline__ T negl_margin();
template <> __device__ __forceinline__ float negl_margin<float>() { return 80.0f; }
template <> __device__ __forceinline__ double negl_margin<double>() { return 1.0e300; }

template <class T, int MODE, int SGN, int KC>
__device__ __forceinline__ void cand_push_m(CandAcc<T> &c, const T *ca, const T *al, T cd, int Kr, T v, T dv, T eta,
                                            T s, T hi, T camax) {
    const int K = KC > 0 ? KC : Kr;
    if (SGN < 0 && !(v < hi)) return;   // a dropped covering row
    const T a = (SGN > 0 ? eta : -eta) * (v - s);
    // A row whose exponents lie more than NEGL below every shift adds nothing
    // representable to R_k and T_k.  Packing: x_k = a + b_k <= a + b_{K-1} and
    // mx_k >= 0.  Covering: x_k <= a <= 0 and exp(a) is the T weight (S_c >= 1).
    if (SGN > 0) {
        if (a + camax * dv < -negl_margin<T>()) return;   // camax = max_k alpha_k eta
    } else {
        if (a < -negl_margin<T>() && a < c.mxmin - negl_margin<T>()) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) c.zm[k] = fmin(c.zm[k], v + al[k] * dv);
            return;
        }
    }
    T b = ca[0] * dv;
    T u = one_minus_exp_neg(b);
    T ud = T(0);
    if (MODE == 1) ud = one_minus_exp_neg(cd * dv);
    T A = T(0);
    if (SGN < 0) A = fast_exp(a);
    // rescale only when some lane of the warp meets a new maximum
    const unsigned act = __activemask();
    bool moved = false;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < K) {
            if (k > 0) {
                b = ca[k] * dv;
                if (MODE == 0) u = u * (T(2) - u);
                else if (MODE == 1) u = u + ud * (T(1) - u);
                else u = one_minus_exp_neg(b);
            }
            const T x = SGN > 0 ? a + b : a - b;
            const bool up = x > c.mx[k];
            if (__any_sync(act, up)) {
                if (up) {
                    T f = fast_exp(c.mx[k] - x);
                    c.R[k] *= f;
                    if (SGN > 0) c.Tt[k] *= f;
                    if (MODE == 3 && k == 0) c.D *= f;
                    c.mx[k] = x;
                    moved = true;
                }
            }
            const T t = fast_exp(x - c.mx[k]);
            c.R[k] += t;
            if (MODE == 3 && k == 0) c.D += dv * t;
            if (SGN > 0) c.Tt[k] += t * u;
            else {
                c.Tt[k] += A * u;
                c.zm[k] = fmin(c.zm[k], v + al[k] * dv);
            }
        }
    }
    if (SGN < 0 && moved) {
        T mn = c.mx[0];
#pragma unroll
        for (int k = 1; k < KMAX; ++k)
            if (k < K) mn = fmin(mn, c.mx[k]);
        c.mxmin = mn;
    }
}

// Covering rows of a search pass (FP32, exponential phase MODE 0 or
// refinement MODE 1, K candidates): every exponent x_k = -eta (z + alpha_k dz
// - s_c) is <= 0 (s_c = min z), so R_k needs no running maximum against
// overflow: it is accumulated with the constant shift COV_SHIFT,
//   R_k += e^{a + COV_SHIFT} e^{-b_k},   a = -eta (z - s_c), b_k = alpha_k eta dz,
// with e^{-b_k} from an exact recurrence along the schedule (squaring when
// alpha doubles, a product with e^{-delta eta dz} when it grows by delta), so a
// row costs two exponentials whatever K, and no warp vote or rescale branch.
// Terms below e^{-87} flush to zero; a row with a < -COV_SHIFT - 87 has no
// representable term and updates only the minima.  The finish clamps
// ln R_k (unshifted) at COV_FLOOR: below it the sum is no longer exact and Phi
// takes its lower bound -(COV_FLOOR - ln S_c)/eta, which can only reject a
// candidate (f >= 1 is then decided on a value at most Phi).
constexpr float COV_SHIFT = 60.0f;
constexpr double COV_FLOOR = -110.0;

template <int MODE>
__device__ __forceinline__ void cand_push_cov(CandAcc<float> &c, const float *ca, const float *al, float cd, float v,
                                              float dv, float eta, float s, float hi) {
    if (!(v < hi)) return;   // a dropped covering row
    const float a = -eta * (v - s);
    if (a < -COV_SHIFT - 87.0f) {   // e^{a + COV_SHIFT} flushes to zero: only the minima move
        if (MODE == 0) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k) c.zm[k] = fminf(c.zm[k], fmaf(al[k], dv, v));
        }
        return;
    }
    const float Ash = __expf(a + COV_SHIFT);
    const float A = __expf(a);
    float b = ca[0] * dv;
    float u = one_minus_exp_neg(b);
    float r = __expf(-b);
    float ud = 0.0f, rd = 1.0f;
    if (MODE == 1) {
        const float bd = cd * dv;
        ud = one_minus_exp_neg(bd);
        rd = __expf(-bd);
    }
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k > 0) {
            if (MODE == 0) { u = u * (2.0f - u); r = r * r; }
            else { u = fmaf(ud, 1.0f - u, u); r = r * rd; }
        }
        c.R[k] = fmaf(Ash, r, c.R[k]);
        c.Tt[k] = fmaf(A, u, c.Tt[k]);
        if (MODE == 0) c.zm[k] = fminf(c.zm[k], fmaf(al[k], dv, v));
    }
}

// merge b into a (sgn as above), in precision U with rescale factors in T
template <class T, class U>
__device__ __forceinline__ void cand_merge1(U &mx, U &R, U &Tt, U &zm, U bmx, U bR, U bT, U bzm, int sgn) {
    zm = fmin(zm, bzm);
    if (sgn < 0) {
        Tt += bT;
        if (bR == U(0)) return;
        if (R == U(0)) { mx = bmx; R = bR; return; }
        U m = fmax(mx, bmx);
        R = R * (U)t_exp((T)(mx - m)) + bR * (U)t_exp((T)(bmx - m));
        mx = m;
    } else {
        if (bR == U(0)) return;
        if (R == U(0)) { mx = bmx; R = bR; Tt = bT; return; }
        U m = fmax(mx, bmx);
        U fa = (U)t_exp((T)(mx - m)), fb = (U)t_exp((T)(bmx - m));
        R = R * fa + bR * fb;
        Tt = Tt * fa + bT * fb;
        mx = m;
    }
}

// cand_merge1 for candidate 0, whose Newton sum D scales like R
template <class T, class U>
__device__ __forceinline__ void cand_merge1d(U &mx, U &R, U &Tt, U &zm, U &D, U bmx, U bR, U bT, U bzm, U bD,
                                             int sgn) {
    if (bR == U(0)) { cand_merge1<T, U>(mx, R, Tt, zm, bmx, bR, bT, bzm, sgn); return; }
    if (R == U(0)) { D = bD; cand_merge1<T, U>(mx, R, Tt, zm, bmx, bR, bT, bzm, sgn); return; }
    const U m = fmax(mx, bmx);
    D = D * (U)t_exp((T)(mx - m)) + bD * (U)t_exp((T)(bmx - m));
    cand_merge1<T, U>(mx, R, Tt, zm, bmx, bR, bT, bzm, sgn);
}

// The search step after a pass (runs on one thread).  Mirrors the K-candidate
// search of the oracle: prefix of passing candidates, early exit on
// min(z + alpha dz) >= 1 in the exponential phase, refinement on [lb, ub].
__device__ void search_finish(DevState *st, double acc) {
    st->phase = PH_DONE;
    st->last_passes = st->passes;
    if (acc >= 1.0) st->alpha_acc = acc;
    else {
        st->alpha_acc = 0.0;
        st->status = ST_INFEASIBLE;
        st->reason = RS_ALPHA;
    }
}

// Next backoff value after Newton converged at alpha with f(alpha) < 1: the
// running product alpha (1 - eps)^p, one value per pass (the first one nearly
// always passes, Newton having stopped within tol of the root).  A value below
// 1 ends the search with 0 (alpha < 1 is INFEASIBLE) without evaluating it.
__device__ void backoff_next(DevState *st) {
    st->bo_cur = st->bo_cur * (1.0 - st->eps);
    if (st->bo_cur < 1.0) {
        st->passes += 1;
        st->total_passes += 1;
        search_finish(st, 0.0);
        return;
    }
    st->kpass = 1;
    st->alpha[0] = st->bo_cur;
}

__device__ void newton_start_backoff(DevState *st, double alpha) {
    if (st->passes >= st->max_passes) { search_finish(st, st->lb >= 1.0 ? st->lb : 0.0); return; }
    st->phase = PH_BACKOFF;
    st->bo_cur = alpha;
    backoff_next(st);
}

// After a Newton pass at alpha = alpha[0] (Sec. 4.2): Newton's update of
// g = f - 1 with the bracket safeguard, the convergence test, and the start
// of the (1 - eps)^p backoff when the converged alpha misses Eq. b4b_conv.
// The same steps as the oracle's search_newton.
__device__ void newton_decide(DevState *st, double psi, double phi, double dpsi, double dphi, double zmin) {
    st->passes += 1;
    st->evals += 1;
    st->total_passes += 1;
    st->newton_steps += 1;
    const double a = st->alpha[0];
    const bool ok = phi >= psi;
    // Alg. 3's early exit: a passing step that covers every row completes MWU;
    // one more pass finds the smallest such step (cover_pass)
    if (ok && zmin >= 1.0 && a >= 1.0) {
        st->early = 1;
        st->phase = PH_COVER;
        st->kpass = 1;
        return;
    }
    if (ok) st->lb = fmax(st->lb, a);
    else st->ub = fmin(st->ub, a);
    const double lb = st->lb, ub = st->ub;
    const double den = psi * dphi - phi * dpsi;
    double nxt = (double)NAN;
    if (psi > 0.0 && den < 0.0 && isfinite(den)) nxt = a - (phi - psi) * psi / den;
    // safeguard: the geometric midpoint of the bracket, or a move by the
    // exponential phase's reach per pass (2^8) while one end is unknown
    if (!(isfinite(nxt) && lb < nxt && nxt < ub)) {
        if (lb > 0.0 && isfinite(ub)) nxt = sqrt(lb * ub);
        else if (isfinite(ub)) nxt = ub * (1.0 / 256.0);
        else nxt = a * 256.0;
    }
    if (fabs(nxt - a) <= st->newton_tol * a || st->newton_steps >= st->max_newton || st->passes >= st->max_passes) {
        if (ok) search_finish(st, a);
        else newton_start_backoff(st, a);
        return;
    }
    st->alpha[0] = nxt;
    st->kpass = 1;
}

// After a backoff pass at alpha[0]: accept it when it passes; a spent budget
// returns the largest passing value seen.
__device__ void backoff_decide(DevState *st, int ok) {
    st->passes += 1;
    st->evals += 1;
    st->total_passes += 1;
    if (ok) { search_finish(st, st->alpha[0]); return; }
    if (st->passes >= st->max_passes) { search_finish(st, st->lb >= 1.0 ? st->lb : 0.0); return; }
    backoff_next(st);
}

__device__ void search_decide(DevState *st, const int *ok, const double *zmin_k) {
    int K = st->kpass;
    int p = 0;
    while (p < K && ok[p]) ++p;
    st->passes += 1;
    st->evals += K;
    st->total_passes += 1;
    double *al = st->alpha;
    bool done = false;
    double acc = 0.0;
    if (st->phase == PH_REFINE) {
        if (p > 0) st->lb = al[p - 1];
        if (p < K) st->ub = al[p];
    } else {
        for (int k = 0; k < p; ++k)
            if (zmin_k[k] >= 1.0) { acc = al[k]; done = true; st->early = 1; break; }
        if (!done) {
            if (p > 0) st->lb = fmax(st->lb, al[p - 1]);
            if (p < K) st->ub = fmin(st->ub, al[p]);
            if (st->lb > 0.0 && st->ub < (double)INFINITY) {
                if (st->step_mode == 3) {   // Newton from the bracket's lower end
                    if (st->passes >= st->max_passes) {
                        search_finish(st, st->lb);
                        return;
                    }
                    st->phase = PH_NEWTON;
                    st->kpass = 1;
                    al[0] = st->lb;
                    return;
                }
                st->phase = PH_REFINE;
            } else if (st->lb == 0.0) {
                if (st->b == 0) { acc = 0.0; done = true; }
                else st->b = max(0, st->b - K);
            } else st->b += K;
        }
    }
    if (!done && st->phase == PH_REFINE && (st->ub - st->lb) <= st->eps * st->lb) { acc = st->lb; done = true; }
    if (!done && st->passes >= st->max_passes) { acc = st->lb; done = true; }
    if (done) {
        search_finish(st, acc);
        return;
    }
    // next candidate set
    if (st->phase == PH_REFINE) {
        double lb = st->lb, ub = st->ub;
        for (int j = 1; j <= K; ++j) al[j - 1] = lb + j * (ub - lb) / (K + 1);
    } else {
        for (int k = 0; k < K; ++k) al[k] = ldexp(1.0, st->b + k);
    }
}

// End of one turn of the search loop (k_cand is the last kernel of a turn):
// continue while the search runs.  The decide rules end every search within
// max_passes passes; the guard ends the loop with an error status should that
// ever fail.
__device__ void loop_turn_end(DevState *st, cudaGraphConditionalHandle cond) {
    unsigned v = search_continues(st);
    if (v && ++st->loop_guard > st->guard_limit) {
        st->status = ST_TIMEOUT;   // the decide rules end every search sooner: a bounded give-up
        v = 0u;
    }
    cudaGraphSetConditional(cond, v);
}

// Psi (packing side, sg = +1) or Phi (covering side, sg = -1) at alpha from the
// merged shifted sums R (of e^{x - mx}) and Tt of one candidate.  The
// transcendentals run in T precision (FP32 for the fast form, whose FP64 units
// are scarce), the sums and the final combination in FP64.
template <class T>
__device__ double side_value(const Side<T> &q, int sg, const DevState *st, int ss, double a, double mx, double R,
                             double Tt, bool floor_cov) {
    // ln S, 1/S and 1/eta come precomputed with S and eta: this runs on the
    // critical path of every pass, where FP64 divisions are slow on GB300
    const double inv_eta = st->inv_eta, lS0 = st->lnS[ss];
    if (q.rv.kind == RK_DENSE1) return a * st->dense_dv[ss];   // single row: smax / smin exact
    if (sg > 0) {
        // Psi = (1/eta) ln(R_true / S_p) = (1/eta) ln(1 + T_true / S_p)
        const double lq = mx + (double)t_log((T)Tt) - lS0;
        return (lq < 0.0) ? (double)t_log1p((T)exp_T<T>(lq)) * inv_eta : (mx + (double)t_log((T)R) - lS0) * inv_eta;
    }
    // Phi = -(1/eta) ln(R_true / S_c) = -(1/eta) ln(1 - T_true / S_c)
    const double qv = Tt * st->invS[ss];
    if (qv <= 0.5) return -(double)t_log1p((T)(-qv)) * inv_eta;
    double lr = mx + (double)t_log((T)R);
    if (floor_cov && !(lr > COV_FLOOR)) lr = COV_FLOOR;   // constant-shift sums: Phi's lower bound
    return -(lr - lS0) * inv_eta;
}

// Last block of a candidate pass: merges the (side, k) quantities, k < K,
// over the block records ([4k + 0..3] = mx, R, Tt, zm of candidate k, [32] =
// the Newton sum D of candidate 0; side 0 in blocks [0, gP), side 1 after) and
// writes Psi_k / Phi_k, the derivative of candidate 0 and min(z + alpha_k dz)
// to fin.
template <class T>
__device__ void cand_finish_merge(const Problem<T> &p, int gP, int K, double (*fin)[KMAX][4], bool floor_cov = false) {
    const DevState *st = p.st;
    block_merge_shifted<T, 3, true>(
        2 * K, T(1),
        [&](int q, int &b0, int &b1) { b0 = q < K ? 0 : gP; b1 = q < K ? gP : (int)gridDim.x; },
        [&](int q) { return 1u | (p.side[q < K ? 0 : 1].sign > 0 ? 2u : 0u) | 4u; },   // covering T is unshifted
        [&](int q, int b, T &m, T (&r)[3], T &v) {
            const int k = q % K;
            const T *o = rec_of<T>(p.part_row, b);
            m = o[4 * k + 0];
            r[0] = o[4 * k + 1];
            r[1] = o[4 * k + 2];
            r[2] = k == 0 ? o[32] : T(0);
            v = o[4 * k + 3];
        },
        [&](int q, T M, const double (&tot)[3], T zm) {
            const int ss = q < K ? 0 : 1, k = q % K;
            const Side<T> &sd = p.side[ss];
            const double a = st->alpha[k];
            fin[ss][k][0] = side_value(sd, sd.sign, st, ss, a, (double)M, tot[0], tot[1], floor_cov);
            // Newton: Psi' = D/R (packing side), Phi' = D/R (covering side); both
            // sums carry the same shift, so the ratio needs no rescale
            fin[ss][k][1] = (sd.rv.kind == RK_DENSE1) ? st->dense_dv[ss] : (tot[0] > 0.0 ? tot[2] / tot[0] : 0.0);
            fin[ss][k][3] = (sd.rv.kind == RK_DENSE1) ? st->dense_v[ss] + a * st->dense_dv[ss] : (double)zm;
        });
}

// Later candidate passes: stream the stored (v, dv) of one side.
template <class T, int MODE, int SGN, int KC>
__device__ __forceinline__ void cand_stream(CandAcc<T> &acc, const CandSched<T> &sc, const Side<T> &sd, int64_t m,
                                            int64_t tid, int64_t nthr, T eta, T sh) {
    T ca[KMAX], al[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) { ca[k] = sc.ca[k]; al[k] = sc.al[k]; }
    const T cd = sc.cd, hi = sc.hi;
    const int K = sc.K;
    const T camax = sched_camax(ca, K);
    int64_t start = 4 * tid;
    if constexpr (sizeof(T) == 4 && SGN < 0 && KC == KMAX && (MODE == 0 || MODE == 1)) {
        // covering rows of a search pass: constant shift, recurrences (cand_push_cov)
        CandAcc<float> &c = reinterpret_cast<CandAcc<float> &>(acc);
#pragma unroll
        for (int k = 0; k < KMAX; ++k) c.mx[k] = -COV_SHIFT;
        const float *cap = reinterpret_cast<const float *>(ca), *alp = reinterpret_cast<const float *>(al);
        for (int64_t j0 = start; j0 < m; j0 += 4 * nthr) {
            const int nr = (int)min((int64_t)4, m - j0);
            float vv[4], dd[4];
            if (nr == 4) {
                const float4 a4 = __ldcs(reinterpret_cast<const float4 *>(sd.v + j0));
                const float4 b4 = __ldcs(reinterpret_cast<const float4 *>(sd.dv + j0));
                vv[0] = a4.x; vv[1] = a4.y; vv[2] = a4.z; vv[3] = a4.w;
                dd[0] = b4.x; dd[1] = b4.y; dd[2] = b4.z; dd[3] = b4.w;
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    vv[r] = r < nr ? (float)sd.v[j0 + r] : 0.0f;
                    dd[r] = r < nr ? (float)sd.dv[j0 + r] : 0.0f;
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r < nr) cand_push_cov<MODE>(c, cap, alp, (float)cd, vv[r], dd[r], (float)eta, (float)sh, (float)hi);
        }
        return;
    }
    if (KC == 1 && sizeof(T) == 4) {
        // one candidate per row leaves the pass short of loads in flight: take
        // eight rows per thread and iteration (four float4 loads issued together)
        for (; start + 4 * nthr + 3 < m; start += 8 * nthr) {
            const float4 a0 = *reinterpret_cast<const float4 *>(sd.v + start);
            const float4 b0 = *reinterpret_cast<const float4 *>(sd.dv + start);
            const float4 a1 = *reinterpret_cast<const float4 *>(sd.v + start + 4 * nthr);
            const float4 b1 = *reinterpret_cast<const float4 *>(sd.dv + start + 4 * nthr);
            const T vv[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const T dd[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r) cand_push_m<T, MODE, SGN, KC>(acc, ca, al, cd, K, vv[r], dd[r], eta, sh, hi, camax);
        }
    }
    for (int64_t j0 = start; j0 < m; j0 += 4 * nthr) {
        const int nr = (int)min((int64_t)4, m - j0);
        T vv[4], dd[4];
        if (nr == 4 && sizeof(T) == 4) {
            float4 a4 = *reinterpret_cast<const float4 *>(sd.v + j0);
            float4 b4 = *reinterpret_cast<const float4 *>(sd.dv + j0);
            vv[0] = a4.x; vv[1] = a4.y; vv[2] = a4.z; vv[3] = a4.w;
            dd[0] = b4.x; dd[1] = b4.y; dd[2] = b4.z; dd[3] = b4.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                vv[r] = r < nr ? sd.v[j0 + r] : T(0);
                dd[r] = r < nr ? sd.dv[j0 + r] : T(0);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r < nr) cand_push_m<T, MODE, SGN, KC>(acc, ca, al, cd, K, vv[r], dd[r], eta, sh, hi, camax);
    }
}

template <class T>
__device__ __forceinline__ void spmv_side(const Problem<T> &p, int s, const T *__restrict__ in, int to_v, T scale) {
    const int bid = blockIdx.x, nbs = gridDim.x;
    const Side<T> &sd = p.side[s];
    const RowView &rv = sd.rv;
    if (rv.kind == RK_DENSE1 || rv.kind == RK_NONE) return;
    T *out = to_v ? sd.v : sd.dv;
    const int64_t m = sd.m;
    const int64_t tid = (int64_t)bid * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)nbs * blockDim.x;
    if (rv.kind != RK_CSR) {
        for (int64_t j0 = 4 * tid; j0 < m; j0 += 4 * nthr) {
            const int nr = (int)min((int64_t)4, m - j0);
            T dd[4];
            if (rv.kind == RK_PAIRSUM && nr == 4 && sizeof(T) == 4) {
                const float4 a = reinterpret_cast<const float4 *>(in)[j0 >> 1];
                const float4 b = reinterpret_cast<const float4 *>(in)[(j0 >> 1) + 1];
                dd[0] = a.x + a.y; dd[1] = a.z + a.w; dd[2] = b.x + b.y; dd[3] = b.z + b.w;
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    dd[r] = T(0);
                    if (r < nr) {
                        const int64_t j = j0 + r;
                        dd[r] = (rv.kind == RK_PAIRSUM) ? in[2 * j] + in[2 * j + 1] : row_gather(rv, j, 0, 1, in);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) dd[r] *= row_coef(sd, j0 + r < m ? j0 + r : j0, scale);
            if (nr == 4 && sizeof(T) == 4) {
                *reinterpret_cast<float4 *>(out + j0) = make_float4((float)dd[0], (float)dd[1], (float)dd[2], (float)dd[3]);
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r < nr) out[j0 + r] = dd[r];
            }
        }
        return;
    }
    {   // segments of long rows: one warp each, partial sums to seg_part
        const int lane = threadIdx.x & 31;
        const int64_t w = tid >> 5, nw = nthr >> 5;
        for (int64_t i = w; i < rv.n_seg; i += nw) {
            const int j = rv.seg_row[i];
            const int kb = rv.seg_beg[i];
            const int ke = min(kb + SEG_LEN, rv.ptr[j + 1]);
            T sum = strided_gather(rv.idx, rv.val, in, kb + lane, ke, 32);
            sum = group_sum(sum, 32);
            if (lane == 0) sd.seg_part[i] = sum;
        }
    }
    {   // medium rows: MED_LANES lanes each
        const int lane = threadIdx.x & (MED_LANES - 1);
        const int64_t gid = tid / MED_LANES, ngroups = nthr / MED_LANES;
        const int64_t wbase = gid - (threadIdx.x & 31) / MED_LANES;   // first group of this warp
        for (int64_t b0 = wbase; b0 < rv.n_med; b0 += ngroups) {
            const int64_t i = b0 + (threadIdx.x & 31) / MED_LANES;
            T sum = T(0);
            int64_t j = -1;
            if (i < rv.n_med) {
                j = rv.med_rows[i];
                sum = strided_gather(rv.idx, rv.val, in, rv.ptr[j] + lane, rv.ptr[j + 1], MED_LANES);
            }
            sum = group_sum(sum, MED_LANES);
            if (j >= 0 && lane == 0) out[j] = sum * row_coef(sd, j, scale);
        }
    }
    for (int64_t i = tid; i < rv.n_short; i += nthr) {   // short rows: one thread each
        const int64_t j = rv.short_rows[i];
        out[j] = strided_gather(rv.idx, rv.val, in, rv.ptr[j], rv.ptr[j + 1], 1) * row_coef(sd, j, scale);
    }
}

// Forward SpMV out = A in for both sides: dv = A d each iteration (dy = Pd,
// dz = Cd; Alg. 2) and v = A x at a new x (y = Px, z = Cx).  No candidate work,
// so it runs at high occupancy.  Every block works on both sides in turn (the
// gathers of one side overlap the streaming of the other, and no block runs
// out of work early).  CSR rows are binned by length at setup: rows longer
// than MED_LEN are cut into SEG_LEN-entry segments, one warp per segment, so no
// block holds a long tail; medium rows take MED_LANES lanes, short rows one
// thread.  The pair rows of W and the edge rows of M^T are streamed four per
// thread.  Every gather loop keeps four independent loads in flight.  Segment
// partials are added per row in a fixed order by the last block, so the
// result does not depend on scheduling.
// skip: bit s set -> side s is not computed here (written by the direction
// kernel, or by the staged SpMV).
template <class T>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 4 ? 6 : 5) k_spmv(Problem<T> p, const T *__restrict__ in, int to_v,
                                                                         int skip) {
    DevState *st = p.st;
    if (!to_v && st->status != ST_RUNNING) return;
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    if (!(skip & 1)) spmv_side(p, 0, in, to_v, K0.scale0);
    if (!(skip & 2)) spmv_side(p, 1, in, to_v, K0.scale1);
}

// Long CSR rows after k_spmv: a warp per row adds the row's segment partial
// sums (lanes strided over the segments, then the fixed shuffle tree), so the
// result does not depend on scheduling; the rows' count sets the grid.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_seg_fixup(Problem<T> p, int to_v, int skip) {
    const DevState *st = p.st;
    if (!to_v && st->status != ST_RUNNING) return;
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t base = 0;
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        const Side<T> &sd = p.side[s];
        const RowView &rv = sd.rv;
        if (rv.kind != RK_CSR || ((skip >> s) & 1) || rv.n_long == 0) continue;
        T *out = to_v ? sd.v : sd.dv;
        const T scale = s == 0 ? K0.scale0 : K0.scale1;
        for (int64_t q = w - base; q < rv.n_long; q += nw) {
            if (q < 0) continue;
            const int j = rv.long_rows[q];
            T sum = T(0);
            for (int k = rv.long_seg[q] + lane; k < rv.long_seg[q + 1]; k += 32) sum += sd.seg_part[k];
            sum = group_sum(sum, 32);
            if (lane == 0) out[j] = sum * row_coef(sd, j, scale);
        }
        base += rv.n_long;
    }
}

// Sum over [beg, end) with stride `step` of val[k] * win[idx[k] - lo], the
// input read from a shared-memory window; four independent index loads in
// flight per lane.
template <class T>
__device__ __forceinline__ T strided_window_gather(const int32_t *idx, const float *val, const T *win, int lo, int beg,
                                                   int end, int step) {
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int k = beg;
    for (; k + 3 * step < end; k += 4 * step) {
        const int i0 = idx[k] - lo, i1 = idx[k + step] - lo, i2 = idx[k + 2 * step] - lo, i3 = idx[k + 3 * step] - lo;
        T t0 = win[i0], t1 = win[i1], t2 = win[i2], t3 = win[i3];
        if (val) {
            t0 *= (T)val[k]; t1 *= (T)val[k + step]; t2 *= (T)val[k + 2 * step]; t3 *= (T)val[k + 3 * step];
        }
        a0 += t0; a1 += t1; a2 += t2; a3 += t3;
    }
    for (; k < end; k += step) {
        T t = win[idx[k] - lo];
        if (val) t *= (T)val[k];
        a0 += t;
    }
    return (a0 + a1) + (a2 + a3);
}

// Staged forward SpMV of one CSR side for banded matrices (the CSB-like tiles
// of Sec. 5.1 on one GPU): each block takes tiles of consecutive rows, copies
// the tile's input window [lo, lo + len) into shared memory with coalesced
// loads, and gathers from there; G lanes per row.  A tile whose window does
// not fit gathers from global memory.  Rows are summed whole, so no segment
// pass follows.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_spmv_tiled(Problem<T> p, const T *__restrict__ in, int to_v, int s) {
    DevState *st = p.st;
    if (!to_v && st->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T *win = reinterpret_cast<T *>(sm_raw);
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    const Side<T> &sd = p.side[s];
    const RowView &rv = sd.rv;
    const T scale = s == 0 ? K0.scale0 : K0.scale1;
    T *out = to_v ? sd.v : sd.dv;
    const int G = rv.G;
    const int lane = threadIdx.x & (G - 1);
    const int nslot = BLOCK / G;
    const int wslot = (threadIdx.x & ~31) / G;   // first row slot of this warp
    const int sub = (threadIdx.x & 31) / G;
    for (int t = blockIdx.x; t < rv.n_tiles; t += gridDim.x) {
        const int64_t r0 = (int64_t)t * rv.tile_rows;
        const int64_t r1 = min(sd.m, r0 + rv.tile_rows);
        const int lo = rv.tile_lo[t], len = rv.tile_len[t];
        const bool staged = len <= tile_wmax<T>();
        __syncthreads();   // the previous tile's rows are done with the window
        if (staged)
            for (int k = threadIdx.x; k < len; k += BLOCK) win[k] = in[lo + k];
        __syncthreads();
        for (int64_t jb = r0 + wslot; jb < r1; jb += nslot) {   // warp-uniform trip count
            const int64_t j = jb + sub;
            T sum = T(0);
            if (j < r1) {
                const int kb = rv.ptr[j], ke = rv.ptr[j + 1];
                sum = staged ? strided_window_gather(rv.idx, rv.val, win, lo, kb + lane, ke, G)
                             : strided_gather(rv.idx, rv.val, in, kb + lane, ke, G);
            }
            sum = group_sum(sum, G);
            if (j < r1 && lane == 0) out[j] = sum * row_coef(sd, j, scale);
        }
    }
}

// Log-sum-exp reductions of y and z at a new x (a2, a3): a stream over both
// sides, then the dense rows from k_x_prep's records (dense_keep = 0) or as
// the state holds them (dense_keep = 1: y and z loaded by the stage hook), and
// the stopping test.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_rows_lse(Problem<T> p, int gP, int nb_var, int dense_keep) {
    DevState *st = p.st;
    const int s = (blockIdx.x < gP) ? 0 : 1;
    const int bid = s == 0 ? blockIdx.x : blockIdx.x - gP;
    const int nbs = s == 0 ? gP : gridDim.x - gP;
    const Side<T> &sd = p.side[s];
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    const T eta_sgn = sd.sign > 0 ? K0.eta : -K0.eta;
    Lse<T> acc{T(0), T(0)};
    const T hi = sd.sign > 0 ? t_inf<T>() : K0.hi;   // dropped covering rows leave the sums
    T vmin = t_inf<T>();
    if (sd.rv.kind != RK_DENSE1 && sd.rv.kind != RK_NONE) {
        for (int64_t j = (int64_t)bid * blockDim.x + threadIdx.x; j < sd.m; j += (int64_t)nbs * blockDim.x) {
            const T vj = sd.v[j];
            vmin = fmin(vmin, vj);
            if (vj < hi) lse_push(acc, vj, eta_sgn, sd.sign);
        }
    }
    lse_block_record(p, acc, eta_sgn, sd.sign, vmin);
    if (last_block_done(&st->counter[0])) {
        finalize_reductions(p, gP, gridDim.x, nb_var, !dense_keep, 0.0);
        if (threadIdx.x == 0) st->counter[0] = 0;
    }
}

// a7: K step candidates per constraint row over the stored (v, dv).
// external = 1: evaluate st->alpha[0..K) and store psi/phi/zmin, no decision.
template <class T>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 4 ? 3 : 1) k_cand(Problem<T> p, int gP, int external) {
    __shared__ CandSched<T> s_sc;
    DevState *st = p.st;
    // in a captured iteration the Newton and backoff passes belong to
    // k_cand_newton, the first kernel of each turn of the search loop
    const bool searching = external || (st->phase != PH_DONE && st->phase != PH_COVER &&
                                        !(p.cond_on && (st->phase == PH_NEWTON || st->phase == PH_BACKOFF)));
    if (p.cond_on && blockIdx.x == 0 && threadIdx.x == 0) st->loop_launches += 1;
    if (st->status != ST_RUNNING || !searching) {
        if (p.cond_on && blockIdx.x == 0 && threadIdx.x == 0) loop_turn_end(st, p.cond);
        return;
    }
    const int K = external ? st->K : st->kpass;
    const bool newton = external ? (st->deriv != 0 && K == 1) : st->phase == PH_NEWTON;
    int s = (blockIdx.x < gP) ? 0 : 1;
    int bid = s == 0 ? blockIdx.x : blockIdx.x - gP;
    int nbs = s == 0 ? gP : gridDim.x - gP;
    const Side<T> &sd = p.side[s];
    __shared__ T s_eta, s_sh[2];
    if (threadIdx.x == 0) {
        s_sc.K = K;
        s_sc.mode = newton ? 3 : external ? 2 : (st->phase == PH_EXP ? 0 : st->phase == PH_REFINE ? 1 : 2);
        s_sc.cd = (T)((st->ub - st->lb) / (K + 1) * st->eta);
        s_sc.hi = (T)st->act_hi;
        s_eta = (T)st->eta;
        s_sh[0] = (T)st->s[0];
        s_sh[1] = (T)st->s[1];
    }
    if (threadIdx.x < KMAX) {
        double a = threadIdx.x < K ? st->alpha[threadIdx.x] : 0.0;
        s_sc.ca[threadIdx.x] = (T)(a * st->eta);
        s_sc.al[threadIdx.x] = (T)a;
    }
    __syncthreads();
    const T eta = s_eta;
    const T sh = s_sh[s];
    const CandSched<T> &sc = s_sc;
    CandAcc<T> acc;
    cand_init(acc, sd.sign);
    const int64_t m = sd.m;
    const int64_t tid = (int64_t)bid * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)nbs * blockDim.x;
    if (sd.rv.kind != RK_DENSE1 && sd.rv.kind != RK_NONE) {
        // a pure stream over the stored (v, dv), four rows per thread, with the
        // schedule in registers and the loop specialised per (mode, side)
        const int md = sc.mode;
        if (md == 3) {
            if (sd.sign > 0) cand_stream<T, 3, 1, 1>(acc, sc, sd, m, tid, nthr, eta, sh);
            else cand_stream<T, 3, -1, 1>(acc, sc, sd, m, tid, nthr, eta, sh);
        } else if (sc.K == KMAX) {
            if (sd.sign > 0) {
                if (md == 0) cand_stream<T, 0, 1, KMAX>(acc, sc, sd, m, tid, nthr, eta, sh);
                else if (md == 1) cand_stream<T, 1, 1, KMAX>(acc, sc, sd, m, tid, nthr, eta, sh);
                else cand_stream<T, 2, 1, KMAX>(acc, sc, sd, m, tid, nthr, eta, sh);
            } else {
                if (md == 0) cand_stream<T, 0, -1, KMAX>(acc, sc, sd, m, tid, nthr, eta, sh);
                else if (md == 1) cand_stream<T, 1, -1, KMAX>(acc, sc, sd, m, tid, nthr, eta, sh);
                else cand_stream<T, 2, -1, KMAX>(acc, sc, sd, m, tid, nthr, eta, sh);
            }
        } else {
            if (sd.sign > 0) cand_stream<T, 2, 1, 0>(acc, sc, sd, m, tid, nthr, eta, sh);
            else cand_stream<T, 2, -1, 0>(acc, sc, sd, m, tid, nthr, eta, sh);
        }
    }
    // block merge in T: warp shuffles, then one 8-lane shuffle tree per
    // candidate over the block's 8 warps (only the pass's K candidates); the
    // cross-block levels below run in FP64
    static_assert(BLOCK / 32 == 8 && KMAX == 8, "block merge layout: 8 warps x 8 candidates");
    __shared__ T wm[BLOCK / 32][KMAX][5];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k < K) {
            T mx = acc.mx[k], R = acc.R[k], Tt = acc.Tt[k], zm = acc.zm[k], D = k == 0 ? acc.D : T(0);
            for (int off = 16; off > 0; off >>= 1) {
                T omx = shfl_x(mx, off), oR = shfl_x(R, off), oT = shfl_x(Tt, off), oz = shfl_x(zm, off);
                T oD = shfl_x(D, off);
                cand_merge1d<T, T>(mx, R, Tt, zm, D, omx, oR, oT, oz, oD, sd.sign);
            }
            if ((threadIdx.x & 31) == 0) {
                T *o = wm[threadIdx.x >> 5][k];
                o[0] = mx; o[1] = R; o[2] = Tt; o[3] = zm; o[4] = D;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        const int k = threadIdx.x >> 3, w = threadIdx.x & 7;
        const T *o = wm[w][k < K ? k : 0];
        T mx = o[0], R = o[1], Tt = o[2], zm = o[3], D = o[4];
        for (int off = 4; off > 0; off >>= 1) {
            T omx = shfl_x(mx, off), oR = shfl_x(R, off), oT = shfl_x(Tt, off), oz = shfl_x(zm, off);
            T oD = shfl_x(D, off);
            cand_merge1d<T, T>(mx, R, Tt, zm, D, omx, oR, oT, oz, oD, sd.sign);
        }
        if (w == 0 && k < K) {
            T *rec = rec_of<T>(p.part_row, blockIdx.x);
            rec[4 * k + 0] = mx; rec[4 * k + 1] = R; rec[4 * k + 2] = Tt; rec[4 * k + 3] = zm;
            if (k == 0) rec[32] = D;
        }
    }
    // one completion level: the last block merges all block records
    if (!last_block_done(&st->counter[2])) return;
    {
        __shared__ double fin[2][KMAX][4];
        // covering sums of a search pass with K = KMAX carry the constant shift (cand_push_cov)
        const bool floor_cov = sizeof(T) == 4 && K == KMAX && (s_sc.mode == 0 || s_sc.mode == 1);
        cand_finish_merge(p, gP, K, fin, floor_cov);
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok[KMAX];
            double zmk[KMAX];
            bool bad = false;
            for (int k = 0; k < K; ++k) {
                double val[2] = {fin[0][k][0], fin[1][k][0]};
                if (!isfinite(val[0]) || !isfinite(val[1])) bad = true;
                st->psi[k] = val[0];
                st->phi[k] = val[1];
                zmk[k] = fin[1][k][3];
                st->zmink[k] = zmk[k];
                ok[k] = val[1] >= val[0];
                st->okk[k] = ok[k];
            }
            if (newton) {
                st->dpsi = fin[0][0][1];
                st->dphi = fin[1][0][1];
                if (!isfinite(st->dpsi) || !isfinite(st->dphi)) bad = true;
            }
            if (bad) {
                st->status = ST_NUMERIC;
                st->numeric_bad = 2;
            } else if (!external) {
                if (newton) newton_decide(st, fin[0][0][0], fin[1][0][0], st->dpsi, st->dphi, zmk[0]);
                else if (st->phase == PH_BACKOFF) backoff_decide(st, ok[0]);
                else search_decide(st, ok, zmk);
            }
            if (p.cond_on) loop_turn_end(st, p.cond);
            st->counter[2] = 0;
        }
    }
}

// ============================================================ Newton pass
// One-candidate pass of the Newton step search (Sec. 4.2): Psi, Phi and the
// sums of Psi', Phi' at alpha_0, then newton_decide (or, in the backoff that
// follows a converged Newton step whose value fails, backoff_decide).  Per row
// it is the K-candidate pass in its Newton mode, with one accumulator set and
// small records, so it runs at higher occupancy than k_cand.  In a captured
// iteration it is the first kernel of each turn of the search loop: outside its
// phases it hands the turn to k_cand through the IF node that follows it, and
// after its own pass it skips k_cand and sets the loop condition itself.
template <class T>
__device__ void cover_pass(const Problem<T> &p, int gP);

template <class T>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 4 ? 5 : 2) k_cand_newton(Problem<T> p, int gP) {
    DevState *st = p.st;
    const int phase = st->phase;
    if (p.cond_on && blockIdx.x == 0 && threadIdx.x == 0) st->loop_launches += 1;
    if (st->status == ST_RUNNING && phase == PH_COVER) {
        cover_pass(p, gP);
        return;
    }
    if (st->status != ST_RUNNING || (phase != PH_NEWTON && phase != PH_BACKOFF)) {
        if (p.cond_on && blockIdx.x == 0 && threadIdx.x == 0) {
            const bool kc = st->status == ST_RUNNING && phase != PH_DONE;
            cudaGraphSetConditional(p.cond_kc, kc ? 1u : 0u);
            if (!kc) cudaGraphSetConditional(p.cond, 0u);   // the search has ended: close the loop
        }
        return;
    }
    const int s = (blockIdx.x < gP) ? 0 : 1;
    const int bid = s == 0 ? blockIdx.x : blockIdx.x - gP;
    const int nbs = s == 0 ? gP : gridDim.x - gP;
    const Side<T> &sd = p.side[s];
    __shared__ T s_c[6];
    if (threadIdx.x == 0) {
        s_c[0] = (T)st->eta;
        s_c[1] = (T)st->s[0];
        s_c[2] = (T)st->s[1];
        s_c[3] = (T)(st->alpha[0] * st->eta);
        s_c[4] = (T)st->alpha[0];
        s_c[5] = (T)st->act_hi;
    }
    __syncthreads();
    const T eta = s_c[0];
    const T sh = s_c[1 + s];
    CandSched<T> sc;
    sc.K = 1;
    sc.mode = 3;
    sc.ca[0] = s_c[3];
    sc.al[0] = s_c[4];
    sc.cd = T(0);
    sc.hi = s_c[5];
    CandAcc<T> acc;
    cand_init(acc, sd.sign);
    const int64_t tid = (int64_t)bid * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)nbs * blockDim.x;
    if (sd.rv.kind != RK_DENSE1 && sd.rv.kind != RK_NONE) {
        if (sd.sign > 0) cand_stream<T, 3, 1, 1>(acc, sc, sd, sd.m, tid, nthr, eta, sh);
        else cand_stream<T, 3, -1, 1>(acc, sc, sd, sd.m, tid, nthr, eta, sh);
    }
    // block merge in T, float record in the k_cand layout (candidate 0)
    T mx = acc.mx[0], R = acc.R[0], Tt = acc.Tt[0], zm = acc.zm[0], D = acc.D;
    for (int off = 16; off > 0; off >>= 1) {
        T omx = shfl_x(mx, off), oR = shfl_x(R, off), oT = shfl_x(Tt, off), oz = shfl_x(zm, off), oD = shfl_x(D, off);
        cand_merge1d<T, T>(mx, R, Tt, zm, D, omx, oR, oT, oz, oD, sd.sign);
    }
    __shared__ T wm[BLOCK / 32][5];
    if ((threadIdx.x & 31) == 0) {
        T *o = wm[threadIdx.x >> 5];
        o[0] = mx; o[1] = R; o[2] = Tt; o[3] = zm; o[4] = D;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const T *o = wm[threadIdx.x & 7];
        mx = o[0]; R = o[1]; Tt = o[2]; zm = o[3]; D = o[4];
        for (int off = 4; off > 0; off >>= 1) {
            T omx = shfl_x(mx, off), oR = shfl_x(R, off), oT = shfl_x(Tt, off), oz = shfl_x(zm, off), oD = shfl_x(D, off);
            cand_merge1d<T, T>(mx, R, Tt, zm, D, omx, oR, oT, oz, oD, sd.sign);
        }
        if (threadIdx.x == 0) {
            T *rec = rec_of<T>(p.part_row, blockIdx.x);
            rec[0] = mx; rec[1] = R; rec[2] = Tt; rec[3] = zm; rec[32] = D;
        }
    }
    if (!last_block_done(&st->counter[2])) return;
    __shared__ double fin[2][KMAX][4];
    cand_finish_merge(p, gP, 1, fin);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double psi = fin[0][0][0], phi = fin[1][0][0];
        st->psi[0] = psi;
        st->phi[0] = phi;
        st->zmink[0] = fin[1][0][3];
        st->okk[0] = phi >= psi;
        st->dpsi = fin[0][0][1];
        st->dphi = fin[1][0][1];
        if (!isfinite(psi) || !isfinite(phi) || !isfinite(st->dpsi) || !isfinite(st->dphi)) {
            st->status = ST_NUMERIC;
            st->numeric_bad = 2;
        } else if (phase == PH_NEWTON) {
            newton_decide(st, psi, phi, st->dpsi, st->dphi, st->zmink[0]);
        } else {
            backoff_decide(st, phi >= psi);
        }
        if (p.cond_on) {
            cudaGraphSetConditional(p.cond_kc, 0u);
            loop_turn_end(st, p.cond);
        }
        st->counter[2] = 0;
    }
}

// The pass after a Newton value alpha that passed and covered every row:
// alpha_c = max over the open covering rows (z_j < 1) of (1 - z_j)/dz_j, the
// smallest step that covers them all (+inf if an open row has dz_j <= 0), and
// the search ends with max(1, min(alpha, alpha_c)): by Prop. 4.2 it passes,
// as alpha_c <= alpha and 1 <= alpha do.
template <class T>
__device__ void cover_pass(const Problem<T> &p, int gP) {
    DevState *st = p.st;
    const Side<T> &C = p.side[1];
    T mr = T(0);
    if (blockIdx.x >= gP && C.rv.kind != RK_DENSE1 && C.rv.kind != RK_NONE) {
        const int64_t nthr = (int64_t)(gridDim.x - gP) * blockDim.x;
        for (int64_t j = (int64_t)(blockIdx.x - gP) * blockDim.x + threadIdx.x; j < C.m; j += nthr) {
            const T v = C.v[j];
            if (v < T(1)) {
                const T dv = C.dv[j];
                mr = fmax(mr, dv > T(0) ? (T(1) - v) / dv : t_inf<T>());
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) mr = fmax(mr, shfl_x(mr, off));
    __shared__ T wmax[BLOCK / 32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mr;
    __syncthreads();
    if (threadIdx.x == 0) {
        T b = wmax[0];
        for (int w = 1; w < BLOCK / 32; ++w) b = fmax(b, wmax[w]);
        rec_of<T>(p.part_row, blockIdx.x)[0] = b;
    }
    if (!last_block_done(&st->counter[2])) return;
    T gm = T(0);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) gm = fmax(gm, rec_of<T>(p.part_row, b)[0]);
    for (int off = 16; off > 0; off >>= 1) gm = fmax(gm, shfl_x(gm, off));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ac = (double)wmax[0];
        for (int w = 1; w < BLOCK / 32; ++w) ac = fmax(ac, (double)wmax[w]);
        if (C.rv.kind == RK_DENSE1) {   // the single objective row: its own covering step
            const double v = st->dense_v[1], dv = st->dense_dv[1];
            ac = v >= 1.0 ? 0.0 : (dv > 0.0 ? (1.0 - v) / dv : (double)INFINITY);
        }
        st->passes += 1;
        st->total_passes += 1;
        search_finish(st, fmax(1.0, fmin(st->alpha[0], ac)));
        if (p.cond_on) {
            cudaGraphSetConditional(p.cond_kc, 0u);
            loop_turn_end(st, p.cond);
        }
        st->counter[2] = 0;
    }
}

// ============================================================ update
// a8: v += alpha dv with the LSE reductions of the new v; x is updated lazily
// by the next k_dir (or k_flush).
template <class T>
__global__ void __launch_bounds__(BLOCK) k_update(Problem<T> p, int gP) {
    DevState *st = p.st;
    if (st->status != ST_RUNNING || st->phase != PH_DONE || !(st->alpha_acc >= 1.0)) return;
    const double alpha = st->alpha_acc;
    int s = (blockIdx.x < gP) ? 0 : 1;
    int bid = s == 0 ? blockIdx.x : blockIdx.x - gP;
    int nbs = s == 0 ? gP : gridDim.x - gP;
    const Side<T> &sd = p.side[s];
    const SweepConsts<T> K0 = sweep_consts<T>(st);
    const T eta_sgn = sd.sign > 0 ? K0.eta : -K0.eta;
    const T a = K0.alpha_acc;
    const T hi = sd.sign > 0 ? t_inf<T>() : K0.hi;   // dropped covering rows leave the sums
    T vmin = t_inf<T>();
    Lse<T> acc{T(0), T(0)};
    if (sd.cv.kind == CK_SPLIT2) {
        // edge rows kept exact: z_e = x_u + x_v from the x that k_xstep has just
        // updated (the same sum the direction kernel forms for the second endpoint)
        const int64_t tid = (int64_t)bid * blockDim.x + threadIdx.x, nthr = (int64_t)nbs * blockDim.x;
        const int2 *ed = reinterpret_cast<const int2 *>(sd.rv.idx);
        const T scale = s == 0 ? K0.scale0 : K0.scale1;
        for (int64_t j0 = 4 * tid; j0 < sd.m; j0 += 4 * nthr) {
            const int nr = (int)min((int64_t)4, sd.m - j0);
            T vv[4];
            if (nr == 4) {
                const int4 e01 = __ldcs(reinterpret_cast<const int4 *>(ed + j0));
                const int4 e23 = __ldcs(reinterpret_cast<const int4 *>(ed + j0 + 2));
                vv[0] = (p.x[e01.x] + p.x[e01.y]) * scale;
                vv[1] = (p.x[e01.z] + p.x[e01.w]) * scale;
                vv[2] = (p.x[e23.x] + p.x[e23.y]) * scale;
                vv[3] = (p.x[e23.z] + p.x[e23.w]) * scale;
                if (sizeof(T) == 4) {
                    __stcs(reinterpret_cast<float4 *>(sd.v + j0),
                           make_float4((float)vv[0], (float)vv[1], (float)vv[2], (float)vv[3]));
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) sd.v[j0 + r] = vv[r];
                }
                if (sd.orig) {   // compacted rows: the full z the direction reads
                    const int4 o = *reinterpret_cast<const int4 *>(sd.orig + j0);
                    sd.vfull[o.x] = vv[0]; sd.vfull[o.y] = vv[1]; sd.vfull[o.z] = vv[2]; sd.vfull[o.w] = vv[3];
                }
            } else {
                for (int r = 0; r < nr; ++r) {
                    const int2 e = ed[j0 + r];
                    vv[r] = (p.x[e.x] + p.x[e.y]) * scale;
                    sd.v[j0 + r] = vv[r];
                    if (sd.orig) sd.vfull[sd.orig[j0 + r]] = vv[r];
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r >= nr) break;
                vmin = fmin(vmin, vv[r]);
                if (vv[r] < hi) lse_push(acc, vv[r], eta_sgn, sd.sign);
            }
        }
    } else if (sd.rv.kind != RK_DENSE1 && sd.rv.kind != RK_NONE) {
        const int64_t tid = (int64_t)bid * blockDim.x + threadIdx.x, nthr = (int64_t)nbs * blockDim.x;
        for (int64_t j0 = 4 * tid; j0 < sd.m; j0 += 4 * nthr) {
            const int nr = (int)min((int64_t)4, sd.m - j0);
            if (nr == 4 && sizeof(T) == 4) {
                float4 v4 = *reinterpret_cast<const float4 *>(sd.v + j0);
                float4 d4 = *reinterpret_cast<const float4 *>(sd.dv + j0);
                v4.x += (float)a * d4.x; v4.y += (float)a * d4.y; v4.z += (float)a * d4.z; v4.w += (float)a * d4.w;
                *reinterpret_cast<float4 *>(sd.v + j0) = v4;
                const T vv[4] = {(T)v4.x, (T)v4.y, (T)v4.z, (T)v4.w};
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    vmin = fmin(vmin, vv[r]);
                    if (vv[r] < hi) lse_push(acc, vv[r], eta_sgn, sd.sign);
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (r >= nr) break;
                    T vj = sd.v[j0 + r] + a * sd.dv[j0 + r];
                    sd.v[j0 + r] = vj;
                    vmin = fmin(vmin, vj);
                    if (vj < hi) lse_push(acc, vj, eta_sgn, sd.sign);
                }
            }
        }
    }
    // block record in T, then one completion level: the last block merges the
    // records of both sides (warp per side) and runs the stopping test
    lse_block_record(p, acc, eta_sgn, sd.sign, vmin);
    if (last_block_done(&st->counter[3])) {
        if (threadIdx.x == 0) {
            st->iter += 1;
            st->pending = p.x_eager ? 0 : 1;   // k_xstep has already applied x += alpha d
            st->alpha_prev = alpha;
        }
        __syncthreads();
        finalize_reductions(p, gP, gridDim.x, 0, false, alpha);
        if (threadIdx.x == 0) st->counter[3] = 0;
    }
}

// apply a pending x += alpha d
template <class T>
__global__ void __launch_bounds__(BLOCK) k_flush(Problem<T> p) {
    DevState *st = p.st;
    if (!st->pending) return;
    const T a = (T)st->alpha_acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x)
        p.x[i] += a * p.d[i];
    if (last_block_done(&st->counter[4])) {
        if (threadIdx.x == 0) { st->pending = 0; st->counter[4] = 0; }
    }
}

// x += alpha d before the update of a problem whose update rebuilds edge rows
// from x (p.x_eager); runs exactly when k_update does.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_xstep(Problem<T> p) {
    const DevState *st = p.st;
    if (st->status != ST_RUNNING || st->phase != PH_DONE || !(st->alpha_acc >= 1.0)) return;
    const T a = (T)st->alpha_acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x)
        p.x[i] += a * p.d[i];
}

// d pot / d val for the explicit CSR values of one side: sign * coef_j * w_j * x_i
template <class T>
__global__ void __launch_bounds__(BLOCK) k_grad_vals(Problem<T> p, int s, float *gv) {
    DevState *st = p.st;
    const Side<T> &sd = p.side[s];
    const RowView &rv = sd.rv;
    const double eta_sgn = st->eta * sd.sign;
    const double s0 = st->s[s], S0 = st->S[s];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < sd.m; j += (int64_t)gridDim.x * blockDim.x) {
        double w = exp(eta_sgn * ((double)sd.v[j] - s0)) / S0;
        double coef = st->scale[s] / (rv.rdiv ? (double)rv.rdiv[j] : 1.0);
        for (int k = rv.ptr[j]; k < rv.ptr[j + 1]; ++k)
            gv[k] = (float)((double)sd.sign * coef * w * (double)p.x[rv.idx[k]]);
    }
}

template <class T, class U>
__global__ void k_convert(const T *src, U *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (U)src[i];
}

// Single objective row of a side applied to a loaded direction (the stage
// hook mwu_set_direction): dense_dv[s] = scale_s c^T d, the value the direction
// kernel otherwise accumulates with d.  Per-block FP64 sums, the last block
// adds them in block order.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_dense_dot(Problem<T> p, const T *vec) {
    __shared__ double sm_d[32];
    DevState *st = p.st;
    double dot[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x)
        for (int s = 0; s < 2; ++s)
            if (p.side[s].cv.kind == CK_DENSE1)
                dot[s] += (p.side[s].cv.cvec ? (double)p.side[s].cv.cvec[i] : 1.0) * (double)vec[i];
    const double t0 = block_sum(dot[0], sm_d);
    const double t1 = block_sum(dot[1], sm_d);
    if (threadIdx.x == 0) {
        p.part_var[(size_t)blockIdx.x * REC + 0] = t0;
        p.part_var[(size_t)blockIdx.x * REC + 1] = t1;
    }
    if (last_block_done(&st->counter[6])) {
        double a0 = 0.0, a1 = 0.0;
        if (threadIdx.x == 0) {
            for (int b = 0; b < (int)gridDim.x; ++b) {
                a0 += p.part_var[(size_t)b * REC + 0];
                a1 += p.part_var[(size_t)b * REC + 1];
            }
            if (p.side[0].rv.kind == RK_DENSE1) st->dense_dv[0] = st->scale[0] * a0;
            if (p.side[1].rv.kind == RK_DENSE1) st->dense_dv[1] = st->scale[1] * a1;
            st->counter[6] = 0;
        }
    }
}

// ============================================================ launchers
static int grid_for(int64_t n, int cap) {
    int64_t g = (n + BLOCK - 1) / BLOCK;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// Blocks of a candidate pass are split between the two sides in proportion to
// their work: the candidate arithmetic (K exp terms per row, weighed as 4
// gathers each) plus, on the first pass, one unit per gathered entry of A d.
template <class T> static void split_rows(const Problem<T> &p, int *gP, int *gC, bool first = true, int total = 0) {
    if (total <= 0) total = p.grid_row;
    auto work = [&](const Side<T> &s) -> double {
        if (s.rv.kind == RK_DENSE1 || s.rv.kind == RK_NONE) return 0.0;
        double w = 4.0 * KMAX * (double)s.m;
        if (first) w += (double)s.rv.nnz;
        return w;
    };
    double wP = work(p.side[0]), wC = work(p.side[1]);
    auto need = [&](const Side<T> &s) -> int {
        if (s.rv.kind == RK_DENSE1 || s.rv.kind == RK_NONE) return 0;
        int64_t groups_per_block = BLOCK / s.rv.G;
        int64_t g = (s.m + groups_per_block - 1) / groups_per_block;
        return (int)std::max<int64_t>(1, g);
    };
    int nP = need(p.side[0]), nC = need(p.side[1]);
    if (wP + wC <= 0.0) { *gP = 1; *gC = 0; return; }
    int aP = (int)((double)total * wP / (wP + wC) + 0.5);
    if (wP > 0 && aP < 1) aP = 1;
    if (wC > 0 && total - aP < 1) aP = total - 1;
    int aC = total - aP;
    if (wP <= 0) aP = 0;
    if (wC <= 0) aC = 0;
    *gP = std::min(aP, nP);
    *gC = std::min(aC, nC);
    if (*gP + *gC == 0) *gP = 1;
}

// grid of the forward SpMV: every block covers both sides; no more blocks than
// the larger side has work items (a warp per segment, four rows per thread)
template <class T> static int spmv_grid(const Problem<T> &p, int skip) {
    // threads the side can use: one per short row, MED_LANES per medium row and
    // a warp per long-row segment (CSR); one per four rows otherwise
    auto need = [&](const Side<T> &sd) -> int64_t {
        if (sd.rv.kind == RK_DENSE1 || sd.rv.kind == RK_NONE) return 0;
        const int64_t items = sd.rv.kind == RK_CSR ? (int64_t)sd.rv.n_short + (int64_t)MED_LANES * sd.rv.n_med +
                                                         32 * (int64_t)sd.rv.n_seg
                                                   : (sd.m + 3) / 4;
        return (items + BLOCK - 1) / BLOCK;
    };
    const int64_t n = std::max((skip & 1) ? 0 : need(p.side[0]), (skip & 2) ? 0 : need(p.side[1]));
    return (int)std::max<int64_t>(0, std::min<int64_t>(n, p.grid_spmv));
}

// out = A in on both sides (to_v: v = A x, else dv = A d): the staged kernel
// for tiled CSR sides, the binned kernel for the rest; skip bit s leaves side s.
template <class T> static cudaError_t spmv_sides(const Problem<T> &p, const T *in, int to_v, int skip, cudaStream_t s) {
    for (int q = 0; q < 2; ++q) {
        const RowView &rv = p.side[q].rv;
        if (((skip >> q) & 1) || rv.kind != RK_CSR || rv.n_tiles <= 0) continue;
        const int g = std::max(1, std::min(rv.n_tiles, p.grid_tiled));
        k_spmv_tiled<T><<<g, BLOCK, TILE_SMEM, s>>>(p, in, to_v, q);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        skip |= 1 << q;
    }
    if (skip == 3) return cudaSuccess;
    const int gs = spmv_grid(p, skip);
    if (gs == 0) return cudaSuccess;
    k_spmv<T><<<gs, BLOCK, 0, s>>>(p, in, to_v, skip);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nl = ((skip & 1) ? 0 : (int64_t)p.side[0].rv.n_long) + ((skip & 2) ? 0 : (int64_t)p.side[1].rv.n_long);
    if (nl > 0) {
        k_seg_fixup<T><<<grid_for(32 * nl, p.grid_spmv), BLOCK, 0, s>>>(p, to_v, skip);
        e = cudaGetLastError();
    }
    return e;
}

template <class T> static cudaError_t rows_at_x(const Problem<T> &p, int nb_var, cudaStream_t s) {
    cudaError_t e = spmv_sides(p, p.x, 1, 0, s);
    if (e != cudaSuccess) return e;
    int gP, gC;
    split_rows(p, &gP, &gC, false);
    k_rows_lse<T><<<gP + gC, BLOCK, 0, s>>>(p, gP, nb_var, 0);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_rows_reduce(const Problem<T> &p, cudaStream_t s) {
    int gP, gC;
    split_rows(p, &gP, &gC, false);
    k_rows_lse<T><<<gP + gC, BLOCK, 0, s>>>(p, gP, 0, 1);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_dense_dir(const Problem<T> &p, cudaStream_t s) {
    if (p.side[0].rv.kind != RK_DENSE1 && p.side[1].rv.kind != RK_DENSE1) return cudaSuccess;
    k_dense_dot<T><<<grid_for(p.n, p.grid_var), BLOCK, 0, s>>>(p, p.d);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_x_init(const Problem<T> &p, cudaStream_t s) {
    int g = grid_for(p.n, p.grid_var);
    k_x_prep<T><<<g, BLOCK, 0, s>>>(p, nullptr, 0, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return rows_at_x(p, g, s);
}

template <class T> cudaError_t launch_x_set(const Problem<T> &p, const void *x, int fp64, cudaStream_t s) {
    int g = grid_for(p.n, p.grid_var);
    k_x_prep<T><<<g, BLOCK, 0, s>>>(p, x, fp64, 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return rows_at_x(p, g, s);
}

template <class T> cudaError_t launch_rows_eval(const Problem<T> &p, cudaStream_t s) {
    return launch_x_set(p, p.x, sizeof(T) == 8 ? 1 : 0, s);
}

template <class T> cudaError_t launch_dir(const Problem<T> &p, int keep_gh, cudaStream_t s) {
    if (dir_fuses_dz(p, keep_gh)) {
        int g = (int)std::max<int64_t>(1, std::min<int64_t>((p.n / 2 + BLOCK - 1) / BLOCK, p.grid_var));
        k_dir_pairs<T><<<g, BLOCK, 0, s>>>(p);
        return cudaGetLastError();
    }
    if (p.hacc) {   // h of the covering side by scatter, read by k_dir
        const RowView &rv = p.side[1].rv;
        const int64_t items = rv.kind == RK_CSR ? (int64_t)rv.n_short + (int64_t)MED_LANES * rv.n_med + 32 * (int64_t)rv.n_seg
                                                : p.side[1].m;
        const int gs = (int)std::max<int64_t>(1, std::min<int64_t>((items + BLOCK - 1) / BLOCK, p.grid_upd));
        k_h_scatter<T><<<gs, BLOCK, 0, s>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (p.side[1].cv.kind == CK_SPLIT2 && p.side[1].cv.n_cseg > 0) {
        const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)p.side[1].cv.n_cseg * 32 + BLOCK - 1) / BLOCK,
                                                                    p.grid_spmv));
        k_split_seg<T><<<gs, BLOCK, 0, s>>>(p, 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int64_t per_block = BLOCK / p.G_var;
    int64_t need = std::max<int64_t>((p.n + per_block - 1) / per_block, p.n_heavy_var);
    int g = (int)std::max<int64_t>(1, std::min<int64_t>(need, p.grid_var));
    k_dir<T><<<g, BLOCK, 0, s>>>(p, keep_gh, 0, nullptr);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_spmv(const Problem<T> &p, cudaStream_t s, int skip_c) {
    return spmv_sides(p, p.d, 0, skip_c ? 2 : 0, s);
}

template <class T> cudaError_t launch_cand(const Problem<T> &p, int external, cudaStream_t s) {
    int gP, gC;
    split_rows(p, &gP, &gC, false);
    k_cand<T><<<gP + gC, BLOCK, 0, s>>>(p, gP, external);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_cand_newton(const Problem<T> &p, cudaStream_t s) {
    int gP, gC;
    split_rows(p, &gP, &gC, false, p.grid_newton);
    k_cand_newton<T><<<gP + gC, BLOCK, 0, s>>>(p, gP);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_update(const Problem<T> &p, cudaStream_t s) {
    // the update is a plain stream over the rows (four per thread): split the
    // update grid by rows
    auto rows = [&](const Side<T> &sd) -> int64_t {
        return (sd.rv.kind == RK_DENSE1 || sd.rv.kind == RK_NONE) ? 0 : sd.m;
    };
    const int64_t mP = rows(p.side[0]), mC = rows(p.side[1]);
    auto need = [&](int64_t m) -> int { return m > 0 ? grid_for((m + 3) / 4, p.grid_upd) : 0; };
    int gP = 0, gC = 0;
    if (mP + mC > 0) {
        int total = p.grid_upd;
        gP = mP > 0 ? std::max(1, (int)((double)total * (double)mP / (double)(mP + mC))) : 0;
        gC = mC > 0 ? std::max(1, total - gP) : 0;
        gP = std::min(gP, need(mP));
        gC = std::min(gC, need(mC));
    }
    if (gP + gC == 0) gP = 1;
    if (p.x_eager) {
        k_xstep<T><<<grid_for(p.n, p.grid_var), BLOCK, 0, s>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_update<T><<<gP + gC, BLOCK, 0, s>>>(p, gP);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_flush(const Problem<T> &p, cudaStream_t s) {
    k_flush<T><<<grid_for(p.n, p.grid_var), BLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_search_begin(const Problem<T> &, cudaStream_t) { return cudaSuccess; }

template <class T> cudaError_t launch_potential_grads(const Problem<T> &p, const float *x, float *gx, float *gobj,
                                                      float *gvals_p, float *gvals_c, cudaStream_t s) {
    (void)x;
    if (p.side[1].cv.kind == CK_SPLIT2 && p.side[1].cv.n_cseg > 0) {
        const int gs = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)p.side[1].cv.n_cseg * 32 + BLOCK - 1) / BLOCK,
                                                                    p.grid_spmv));
        k_split_seg<T><<<gs, BLOCK, 0, s>>>(p, 1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int64_t per_block = BLOCK / p.G_var;
    int64_t need = std::max<int64_t>((p.n + per_block - 1) / per_block, p.n_heavy_var);
    int g = (int)std::max<int64_t>(1, std::min<int64_t>(need, p.grid_var));
    k_dir<T><<<g, BLOCK, 0, s>>>(p, 0, 1, gobj);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (gx) {
        k_convert<T, float><<<grid_for(p.n, p.grid_var), BLOCK, 0, s>>>(p.d, gx, p.n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (gvals_p && p.side[0].rv.kind == RK_CSR) {
        k_grad_vals<T><<<grid_for(p.side[0].m, p.grid_row), BLOCK, 0, s>>>(p, 0, gvals_p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (gvals_c && p.side[1].rv.kind == RK_CSR) {
        k_grad_vals<T><<<grid_for(p.side[1].m, p.grid_row), BLOCK, 0, s>>>(p, 1, gvals_c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class T> cudaError_t launch_copy_vec(const T *src, void *dst, int64_t n, int fp64, cudaStream_t s) {
    int g = grid_for(n, 4096);
    if (fp64) k_convert<T, double><<<g, BLOCK, 0, s>>>(src, (double *)dst, n);
    else k_convert<T, float><<<g, BLOCK, 0, s>>>(src, (float *)dst, n);
    return cudaGetLastError();
}

template <class T>
__global__ void k_nonneg_finite(const T *v, int64_t n, int *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T a = v[i];
        if (!(a >= T(0)) || !isfinite(a)) atomicOr(bad, 1);
    }
}

template <class T> cudaError_t launch_check_nonneg(const T *v, int64_t n, int *bad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_nonneg_finite<T><<<grid_for(n, 4096), BLOCK, 0, s>>>(v, n, bad);
    return cudaGetLastError();
}
template cudaError_t launch_check_nonneg<float>(const float *, int64_t, int *, cudaStream_t);
template cudaError_t launch_check_nonneg<double>(const double *, int64_t, int *, cudaStream_t);

__global__ void k_same_f32(const float *a, const float *b, int64_t n, int *differ) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float va = a ? a[i] : 1.0f;
        if (__float_as_uint(va) != __float_as_uint(b[i])) atomicOr(differ, 1);
    }
}

cudaError_t launch_same_f32(const float *a, const float *b, int64_t n, int *differ, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_same_f32<<<grid_for(n, 4096), BLOCK, 0, s>>>(a, b, n, differ);
    return cudaGetLastError();
}

template <class T, class U> cudaError_t launch_convert_in(const U *src, T *dst, int64_t n, cudaStream_t s) {
    k_convert<U, T><<<grid_for(n, 4096), BLOCK, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}
template cudaError_t launch_convert_in<float, float>(const float *, float *, int64_t, cudaStream_t);
template cudaError_t launch_convert_in<float, double>(const double *, float *, int64_t, cudaStream_t);
template cudaError_t launch_convert_in<double, float>(const float *, double *, int64_t, cudaStream_t);
template cudaError_t launch_convert_in<double, double>(const double *, double *, int64_t, cudaStream_t);

template <class T> int sweep_blocks_per_sm(int *var_bps, int *row_bps, int *upd_bps) {
    int a = 0, b = 0, c = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_dir<T>, BLOCK, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cand<T>, BLOCK, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_update<T>, BLOCK, 0);
    *var_bps = a > 0 ? a : 1;
    *row_bps = b > 0 ? b : 1;
    *upd_bps = c > 0 ? c : 1;
    return 0;
}

template <class T> int newton_blocks_per_sm() {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cand_newton<T>, BLOCK, 0);
    return a > 0 ? a : 1;
}

template <class T> int spmv_blocks_per_sm() {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_spmv<T>, BLOCK, 0);
    return a > 0 ? a : 1;
}

// Also raises the kernel's dynamic shared memory limit to the window size (its
// static shared memory plus TILE_SMEM exceed the 48 KB default); it runs
// before the first launch of a context.
template <class T> int tiled_blocks_per_sm() {
    cudaFuncSetAttribute(k_spmv_tiled<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_SMEM);
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_spmv_tiled<T>, BLOCK, TILE_SMEM);
    return a > 0 ? a : 1;
}

// ============================================================ batched b-matching
// One persistent launch solves a batch of independent b-matching LPs
// (Appendix A.1 with lb = 0: max 1^T x, diag(1/b) M x <= 1, a pure packing LP
// whose covering side is the objective row (1/M) 1^T x >= 1, Sec. 2.2).  A
// crew -- one block, or a thread-block cluster of C blocks -- takes the next
// instance from a device work queue (instances ordered by decreasing size) and
// runs its whole solve: the bracket and the geometric bisection on M, and per
// probe Alg. 2's iterations with the K-candidate or Newton search (the
// library's own decision rules, dir_finish / search_decide / newton_decide, on
// a DevState that every block of the crew keeps and updates identically).
//
// Cluster launches (C > 1) first drain a queue of the large instances (at
// least batch_cluster_edges(NT, C) edges), each solved by the whole cluster:
// every loop is strided over the C * NT threads, and every sum is reduced in
// the block, published in a shared-memory slot, and combined by each block
// from the C slots in rank order through distributed shared memory after one
// cluster barrier (release / acquire), so that all blocks hold bit-identical
// totals and take identical decisions.  The barriers also order the global
// writes of one block before another block's gathers (of y in the direction,
// of d and x in P v); those gathers bypass L1 (ld.global.cg).  Then every block
// takes the remaining small instances alone from a second queue.  An
// instance's result depends only on the block size and on whether a cluster
// (and of which size) solved it, never on the batch or the schedule.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// A double in block `rank`'s shared memory at the address of p in this block's.
__device__ __forceinline__ double ld_peer(const double *p, unsigned rank) {
    uint32_t a = (uint32_t)__cvta_generic_to_shared(p), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(r));
    return v;
}

constexpr int XS = 5 * KMAX;   // doubles per exchange slot (K candidate records)

template <int NT, int C> struct Crew {
    static constexpr int S = NT * C;   // loop stride over an instance's edges and vertices
    unsigned rank;                     // block rank in the cluster (0 when C == 1)
    int par;                           // exchange-slot parity (alternates per exchange)
    double *slot;                      // this block's exchange slots, [2][XS] in shared memory
    __device__ int64_t tid() const { return (int64_t)rank * NT + threadIdx.x; }
    // the slot of the next exchange; the alternation makes one barrier per
    // exchange enough (a slot is rewritten only after the next exchange's
    // barrier, which every block reaches after its reads of this one)
    __device__ double *next() {
        double *p = slot + par * XS;
        par ^= 1;
        return p;
    }
};

// Gathered load of data that another block of the crew wrote
template <int C> __device__ __forceinline__ float gload(const float *p) {
    if constexpr (C == 1) return *p;
    else return __ldcg(p);
}

// ---- crew reductions.  GB300 runs FP64 at a small fraction of its FP32 rate,
// so the per-thread and per-warp work is FP32 and FP64 is kept to short trees
// over the warps' and blocks' totals.  Every result is valid at thread 0 of
// each block of the crew (identical in all blocks: the same values combined by
// the same tree); the callers broadcast what the other threads need.

// Sums over the crew of per-thread partials P (FP32, or FP64 where a solve's
// certificate depends on them): P within each warp, FP64 over the warps (a
// tree in warp 0) and over the cluster's blocks (a tree over lanes 0 .. C-1
// after one exchange).
template <int NT, int C, int NV, class P>
__device__ void crew_sums(Crew<NT, C> &cw, P (&v)[NV], double (&out)[NV], double *sm) {
    constexpr int W = NT / 32;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        for (int off = 16; off > 0; off >>= 1) v[i] += shfl_x(v[i], off);
        if (l == 0) sm[i * W + w] = (double)v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = 0.0;
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double t = l < W ? sm[i * W + l] : 0.0;
            for (int off = W / 2; off > 0; off >>= 1) t += shfl_x(t, off);
            out[i] = t;
        }
    }
    if constexpr (C > 1) {
        double *sl = cw.next();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i) sl[i] = out[i];
        }
        cluster_barrier();
        if (w == 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                double t = l < C ? ld_peer(sl + i, l) : 0.0;
                for (int off = C / 2; off > 0; off >>= 1) t += shfl_x(t, off);
                out[i] = t;
            }
        }
    }
    __syncthreads();
}

// Maximum over the crew of per-thread values (all >= 0), FP32.
template <int NT, int C> __device__ float crew_max(Crew<NT, C> &cw, float v, float *smf) {
    constexpr int W = NT / 32;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, shfl_x(v, off));
    if (l == 0) smf[w] = v;
    __syncthreads();
    float t = 0.0f;
    if (w == 0) {
        t = l < W ? smf[l] : 0.0f;
        for (int off = W / 2; off > 0; off >>= 1) t = fmaxf(t, shfl_x(t, off));
    }
    if constexpr (C > 1) {
        double *sl = cw.next();
        if (threadIdx.x == 0) sl[0] = (double)t;
        cluster_barrier();
        if (w == 0) {
            t = l < C ? (float)ld_peer(sl, l) : 0.0f;
            for (int off = C / 2; off > 0; off >>= 1) t = fmaxf(t, shfl_x(t, off));
        }
    }
    __syncthreads();
    return t;
}

// Log-sum-exp of y (packing rows, sign +1): s = max y, S = sum e^{eta (y - s)},
// FP32 throughout (per thread, a tree over the lanes, the warps and the
// cluster's blocks); valid at thread 0.
template <int NT, int C>
__device__ void bt_lse(Crew<NT, C> &cw, const float *y, int64_t n, float eta, float *smf, float &s_out,
                       float &S_out) {
    constexpr int W = NT / 32;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    Lse<float> acc{0.0f, 0.0f};
    for (int64_t j = cw.tid(); j < n; j += Crew<NT, C>::S) lse_push(acc, y[j], eta, 1);
    for (int off = 16; off > 0; off >>= 1) {
        const float os = shfl_x(acc.s, off), oS = shfl_x(acc.S, off);
        lse_merge<float, float>(acc, os, oS, eta, 1);
    }
    if (l == 0) { smf[w] = acc.s; smf[W + w] = acc.S; }
    __syncthreads();
    Lse<float> t{0.0f, 0.0f};
    if (w == 0) {
        if (l < W) t = Lse<float>{smf[l], smf[W + l]};
        for (int off = W / 2; off > 0; off >>= 1) {
            const float os = shfl_x(t.s, off), oS = shfl_x(t.S, off);
            lse_merge<float, float>(t, os, oS, eta, 1);
        }
    }
    if constexpr (C > 1) {
        double *sl = cw.next();
        if (threadIdx.x == 0) { sl[0] = (double)t.s; sl[1] = (double)t.S; }
        cluster_barrier();
        if (w == 0) {
            t = Lse<float>{0.0f, 0.0f};
            if (l < C) t = Lse<float>{(float)ld_peer(sl, l), (float)ld_peer(sl + 1, l)};
            for (int off = C / 2; off > 0; off >>= 1) {
                const float os = shfl_x(t.s, off), oS = shfl_x(t.S, off);
                lse_merge<float, float>(t, os, oS, eta, 1);
            }
        }
    }
    __syncthreads();
    s_out = t.s;
    S_out = t.S;
}

// y_w = (1/b_w) sum_{e at w} v_e over the vertex -> incident-edge lists: four
// vertices per thread and round, their list bounds loaded together, then four
// edge ids of each and their four gathers in flight at a time.  Vertex w is
// handled by the thread that owns index w in every other strided loop.
template <int NT, int C>
__device__ void bt_rows(const Crew<NT, C> &cw, const int32_t *vp, const int32_t *ei, const float *bnd, const float *v,
                        float *out, int64_t n) {
    constexpr int S = Crew<NT, C>::S;
    for (int64_t w0 = cw.tid(); w0 < n; w0 += 4 * S) {
        int kb[4], ke[4];
        float acc[4];
        int len = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t w = w0 + r * S;
            kb[r] = w < n ? vp[w] : 0;
            ke[r] = w < n ? vp[w + 1] : 0;
            acc[r] = 0.0f;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) len = max(len, ke[r] - kb[r]);
        for (int t = 0; t < len; t += 4) {
            int id[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = kb[r] + t + q;
                    id[r][q] = k < ke[r] ? ei[k] : -1;
                }
            float g[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) g[r][q] = id[r][q] >= 0 ? gload<C>(v + id[r][q]) : 0.0f;
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r] += (g[r][0] + g[r][1]) + (g[r][2] + g[r][3]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t w = w0 + r * S;
            if (w < n) out[w] = bnd ? acc[r] / bnd[w] : acc[r];
        }
    }
}

// Candidate records of one pass: the warps' records (wrec, wD) merged by warp
// 0, four lanes per candidate (each merges every fourth warp, then two
// butterfly steps), then the cluster's blocks likewise after one exchange.
// Candidate k's record lands in lane 4k of warp 0.
template <int NT, int C>
__device__ void bt_cand_reduce(Crew<NT, C> &cw, const float (*wrec)[KMAX][4], const float *wD, int K, float &mx,
                               float &R, float &Tt, float &zm, float &D) {
    constexpr int W = NT / 32;
    const int l = threadIdx.x & 31, k = l >> 2, j = l & 3;
    mx = 0.0f; R = 0.0f; Tt = 0.0f; zm = t_inf<float>(); D = 0.0f;
    const bool wz = (threadIdx.x >> 5) == 0;
    if (wz) {
        if (k < K)
            for (int q = j; q < W; q += 4)
                cand_merge1d<float, float>(mx, R, Tt, zm, D, wrec[q][k][0], wrec[q][k][1], wrec[q][k][2], wrec[q][k][3],
                                           k == 0 ? wD[q] : 0.0f, 1);
        for (int off = 1; off < 4; off <<= 1) {
            const float omx = shfl_x(mx, off), oR = shfl_x(R, off), oT = shfl_x(Tt, off), oz = shfl_x(zm, off),
                        oD = shfl_x(D, off);
            cand_merge1d<float, float>(mx, R, Tt, zm, D, omx, oR, oT, oz, oD, 1);
        }
    }
    if constexpr (C > 1) {
        double *sl = cw.next();
        if (wz && j == 0 && k < K) {
            double *o = sl + 5 * k;
            o[0] = mx; o[1] = R; o[2] = Tt; o[3] = zm; o[4] = D;
        }
        cluster_barrier();
        if (wz) {
            mx = 0.0f; R = 0.0f; Tt = 0.0f; zm = t_inf<float>(); D = 0.0f;
            if (k < K) {
                const double *o = sl + 5 * k;
                for (int q = j; q < C; q += 4)
                    cand_merge1d<float, float>(mx, R, Tt, zm, D, (float)ld_peer(o, q), (float)ld_peer(o + 1, q),
                                               (float)ld_peer(o + 2, q), (float)ld_peer(o + 3, q),
                                               (float)ld_peer(o + 4, q), 1);
            }
            for (int off = 1; off < 4; off <<= 1) {
                const float omx = shfl_x(mx, off), oR = shfl_x(R, off), oT = shfl_x(Tt, off), oz = shfl_x(zm, off),
                            oD = shfl_x(D, off);
                cand_merge1d<float, float>(mx, R, Tt, zm, D, omx, oR, oT, oz, oD, 1);
            }
        }
    }
}

// Scalars of one solve, owned by thread 0 (the doubles) and broadcast to the
// block through shared memory (the floats and the flag).
// Each broadcast field is written by thread 0 before a barrier and read by the
// others after it, and thread 0 rewrites it only after a later barrier (go is
// shared by decisions that have at least one barrier between them; phase and
// kpass copy the search state for the pass loop; acc / af end a step search).
struct BtCtl {
    double eta, hi, lo, best, M, rho, z, dz, lnS;
    long long iters, evals, passes;
    int probes, it, status, go, acc, phase, kpass;
    float eta_f, thr, x0, cdf, invM, fp, sf, af;
};

// Thread 0, at the end of a step search: accept alpha (>= 1) or end the probe.
__device__ __forceinline__ void bt_step_end(BtCtl &cs, DevState *st) {
    const double alpha = st->alpha_acc;
    cs.acc = st->status == ST_RUNNING && alpha >= 1.0;
    if (cs.acc) {
        cs.af = (float)alpha;
        cs.z += alpha * cs.dz;
        cs.it += 1;
        st->alpha_prev = alpha;
        st->iter = cs.it;
    }
}

template <int NT, int C>
__device__ void bt_solve(const BatchDesc &B, int inst, DevState *st, Crew<NT, C> &cw) {
    constexpr int S = Crew<NT, C>::S, W = NT / 32;
    __shared__ double sm[2 * W];
    __shared__ float smf[2 * W];
    __shared__ float s_al[KMAX], s_ca[KMAX];
    __shared__ float wrec[W][KMAX][4];
    __shared__ float wD[W];
    __shared__ double s_psi[KMAX], s_dpsi;
    __shared__ BtCtl cs;
    const int64_t tid = cw.tid();
    const int64_t e0 = B.eoff[inst], E = B.eoff[inst + 1] - e0;
    const int64_t v0 = B.voff[inst], n = B.voff[inst + 1] - v0;
    const int2 *ed = reinterpret_cast<const int2 *>(B.edges) + e0;
    const float *bnd = B.bound ? B.bound + v0 : nullptr;
    const int32_t *vp = B.vptr + v0 + inst;
    const int32_t *ei = B.eids + 2 * e0;
    float *x = B.x + e0, *d = B.d + e0, *y = B.y + v0, *dy = B.dy + v0;
    const double eps = B.eps;
    if (cw.rank == 0 && threadIdx.x == 0) B.t_beg[inst] = (int64_t)globaltimer_ns();
    // bracket (packing, c = 1, a_we = 1/b_w): hi = sum_e max(b_u, b_v), lo = sum_e min(b_u, b_v) / E
    {
        float v[2] = {0.0f, 0.0f};
        for (int64_t e = tid; e < E; e += S) {
            const int2 uv = ed[e];
            const float bu = bnd ? bnd[uv.x] : 1.0f, bv = bnd ? bnd[uv.y] : 1.0f;
            v[0] += fmaxf(bu, bv);
            v[1] += fminf(bu, bv);
        }
        double o[2];
        crew_sums(cw, v, o, sm);
        if (threadIdx.x == 0) {
            const double eta = B.eta_factor * log((double)(n + 1)) / eps;
            cs.eta = eta; cs.eta_f = (float)eta; cs.cdf = (float)(1.0 / eta);
            cs.thr = (float)(1.0 - B.grad_tol);
            cs.x0 = (float)(eps / (double)E);
            cs.hi = o[0]; cs.lo = o[1] / (double)E; cs.best = cs.lo;
            cs.probes = 0; cs.iters = 0; cs.evals = 0; cs.passes = 0;
        }
        __syncthreads();
    }
    const double eta = cs.eta;
    const float eta_f = cs.eta_f, thr = cs.thr, cd_f = cs.cdf, x0 = cs.x0;
    for (;;) {
        if (threadIdx.x == 0) {
            cs.go = cs.hi > (1.0 + B.outer_tol) * cs.lo && cs.probes < B.max_probes;
            if (cs.go) {
                cs.M = sqrt(cs.lo * cs.hi);
                cs.rho = (1.0 + B.outer_tol) * cs.M / cs.hi;   // the certificate closes the bracket (R12)
                cs.invM = (float)(1.0 / cs.M);
            }
        }
        __syncthreads();
        if (!cs.go) break;
        const float invM = cs.invM;
        // a0: x_e = eps / (E max(1/b_u, 1/b_v)) = (eps / E) min(b_u, b_v), y = Px, z = 1^T x / M
        {
            double v[1] = {0.0};   // FP32 over runs of 8 edges, folded into FP64
            float run = 0.0f;
            int cnt = 0;
            for (int64_t e = tid; e < E; e += S) {
                const int2 uv = ed[e];
                const float xe = x0 * (bnd ? fminf(bnd[uv.x], bnd[uv.y]) : 1.0f);
                x[e] = xe;
                run += xe;
                if (++cnt == 8) { v[0] += (double)run; run = 0.0f; cnt = 0; }
            }
            v[0] += (double)run;
            double o[1];
            crew_sums(cw, v, o, sm);   // (the exchange orders the x writes before the gathers)
            if (threadIdx.x == 0) cs.z = o[0] / cs.M;
        }
        bt_rows(cw, vp, ei, bnd, x, y, n);
        // the probe's search state starts from zero in every block of the crew
        for (int i = threadIdx.x; i < (int)(sizeof(DevState) / 8); i += NT) reinterpret_cast<long long *>(st)[i] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            st->eta = eta; st->eps = eps; st->c_d = 1.0 / eta; st->K = B.K; st->max_passes = B.max_passes;
            st->warm_start = B.warm_start; st->step_mode = B.step_mode; st->max_newton = B.max_newton;
            st->newton_tol = B.newton_tol; st->alpha_prev = 0.0; st->scale[0] = 1.0;
            st->scale[1] = 1.0 / cs.M; st->status = ST_RUNNING; st->reason = RS_NONE; st->iter = 0;
            cs.it = 0;
            cs.status = ST_RUNNING;
        }
        __syncthreads();
        for (;;) {
            float sp, Sp;
            bt_lse(cw, y, n, eta_f, smf, sp, Sp);   // (its exchange orders the y writes before the gathers)
            // stopping tests before each iteration (Alg. 2, R8, R12), zmin = z (one exact row)
            if (threadIdx.x == 0) {
                const double ymax = sp, z = cs.z;
                int stt = ST_RUNNING;
                if (cs.rho > 0.0 && z > 0.0 && ymax <= cs.rho * z) stt = ST_FEASIBLE;
                else if (z >= 1.0 || ymax > 1.0 + eps) stt = ymax <= (1.0 + eps) * z ? ST_FEASIBLE : ST_INFEASIBLE;
                else if (cs.it >= B.max_iter) stt = ST_MAX_ITER;
                cs.status = stt;
                cs.go = stt == ST_RUNNING;
                cs.fp = (float)(1.0 / (double)Sp);
                cs.sf = sp;
                cs.lnS = (double)logf(Sp);
            }
            __syncthreads();
            if (!cs.go) break;
            // a4, a5: g_e = (w_u / b_u + w_v / b_v) / S_p, h_e = 1/M; d_e = c_d max(0, 1 - g/h) x_e
            const float fp = cs.fp, s_f = cs.sf;
            {
                float v[2] = {0.0f, 0.0f};   // count of d_e > 0, sum of d_e
                // four edges per thread and round: their endpoint and x loads, then
                // the gathers of y and b, then the arithmetic
                for (int64_t ea = tid; ea < E; ea += 4 * S) {
                    int2 uv[4];
                    float xe[4], yu[4], yv[4], bu[4], bv[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int64_t e = ea + r * S;
                        uv[r] = e < E ? ed[e] : make_int2(0, 0);
                        xe[r] = e < E ? x[e] : 0.0f;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        yu[r] = gload<C>(y + uv[r].x);
                        yv[r] = gload<C>(y + uv[r].y);
                        bu[r] = bnd ? bnd[uv[r].x] : 1.0f;
                        bv[r] = bnd ? bnd[uv[r].y] : 1.0f;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int64_t e = ea + r * S;
                        if (e < E) {
                            float wu = t_exp(eta_f * (yu[r] - s_f)), wv = t_exp(eta_f * (yv[r] - s_f));
                            if (bnd) { wu /= bu[r]; wv /= bv[r]; }
                            const float g = (wu + wv) * fp, h = invM;
                            const float de = (g < thr * h) ? cd_f * (1.0f - g / h) * xe[r] : 0.0f;
                            d[e] = de;
                            v[0] += de > 0.0f ? 1.0f : 0.0f;
                            v[1] += de;
                        }
                    }
                }
                double o[2];
                crew_sums(cw, v, o, sm);   // (orders the d writes before the gathers of P d)
                bt_rows(cw, vp, ei, bnd, d, dy, n);   // a6: dy = P d
                if (threadIdx.x == 0) {
                    st->phase = PH_DONE;
                    dir_finish(st, o[0], 0.0, o[1]);   // d = 0 -> INFEASIBLE, else the search starts
                    st->dense_v[1] = cs.z;
                    cs.dz = st->dense_dv[1];
                    cs.go = st->status == ST_RUNNING;
                    cs.status = ST_INFEASIBLE;   // unless a step is accepted (the next stop test rewrites it)
                    cs.acc = 0;
                    cs.phase = st->phase;
                    cs.kpass = st->kpass;
                }
                __syncthreads();
                if (!cs.go) break;
            }
            // a7: the step search over the packing rows (Phi_k = alpha_k dz, Phi' = dz
            // exactly): K-candidate passes (exponential phase, refinement), Newton
            // and backoff passes (one candidate with Psi'), the covering step
            for (int guard = 0; guard < 128; ++guard) {
                const int phase = cs.phase;
                if (phase == PH_COVER) {   // the smallest step that covers the objective row
                    if (threadIdx.x == 0) {
                        const double z = cs.z, dz = cs.dz;
                        const double ac = z >= 1.0 ? 0.0 : (dz > 0.0 ? (1.0 - z) / dz : (double)INFINITY);
                        st->passes += 1;
                        st->total_passes += 1;
                        search_finish(st, fmax(1.0, fmin(st->alpha[0], ac)));
                        bt_step_end(cs, st);
                    }
                    __syncthreads();
                    break;
                }
                const bool nwt = phase == PH_NEWTON || phase == PH_BACKOFF;
                const int K = nwt ? 1 : cs.kpass;
                if (threadIdx.x < KMAX) {
                    const double a = threadIdx.x < K ? st->alpha[threadIdx.x] : 0.0;
                    s_al[threadIdx.x] = (float)a;
                    s_ca[threadIdx.x] = (float)(a * eta);
                }
                __syncthreads();
                float ca[KMAX], al[KMAX];
#pragma unroll
                for (int k = 0; k < KMAX; ++k) { ca[k] = s_ca[k]; al[k] = s_al[k]; }
                const float camax = sched_camax(ca, K);
                CandAcc<float> acc;
                cand_init(acc, 1);
                if (nwt) {
                    for (int64_t j = tid; j < n; j += S)
                        cand_push_m<float, 3, 1, 1>(acc, ca, al, 0.0f, 1, y[j], dy[j], eta_f, s_f, t_inf<float>(), camax);
                } else {
                    for (int64_t j = tid; j < n; j += S)
                        cand_push_m<float, 2, 1, 0>(acc, ca, al, 0.0f, K, y[j], dy[j], eta_f, s_f, t_inf<float>(), camax);
                }
#pragma unroll
                for (int k = 0; k < KMAX; ++k) {
                    if (k < K) {
                        float mx = acc.mx[k], R = acc.R[k], Tt = acc.Tt[k], zm = acc.zm[k], D = k == 0 ? acc.D : 0.0f;
                        for (int off = 16; off > 0; off >>= 1) {
                            const float omx = shfl_x(mx, off), oR = shfl_x(R, off), oT = shfl_x(Tt, off),
                                        oz = shfl_x(zm, off), oD = shfl_x(D, off);
                            cand_merge1d<float, float>(mx, R, Tt, zm, D, omx, oR, oT, oz, oD, 1);
                        }
                        if ((threadIdx.x & 31) == 0) {
                            float *o = wrec[threadIdx.x >> 5][k];
                            o[0] = mx; o[1] = R; o[2] = Tt; o[3] = zm;
                            if (k == 0) wD[threadIdx.x >> 5] = D;
                        }
                    }
                }
                __syncthreads();
                {
                    float mx, R, Tt, zm, D;
                    bt_cand_reduce(cw, wrec, wD, K, mx, R, Tt, zm, D);
                    const int l = threadIdx.x & 31, k = l >> 2;
                    if (threadIdx.x < 32 && (l & 3) == 0 && k < K) {
                        // Psi = (1/eta) ln(R_true / S_p) = (1/eta) ln(1 + T_true / S_p) (Sec. 4.1);
                        // the transcendentals in FP32, the combination in FP64
                        const double lS = cs.lnS;
                        const double lq = (double)mx + (double)logf(Tt) - lS;
                        s_psi[k] = (lq < 0.0) ? (double)log1pf(expf((float)lq)) / eta
                                              : ((double)mx + (double)logf(R) - lS) / eta;
                        if (k == 0) s_dpsi = R > 0.0f ? (double)D / (double)R : 0.0;   // Psi' (Sec. 4.2)
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    const double z = cs.z, dz = cs.dz;
                    int ok[KMAX];
                    double zmk[KMAX];
                    for (int k = 0; k < K; ++k) {
                        const double phi = st->alpha[k] * dz;
                        st->psi[k] = s_psi[k];
                        st->phi[k] = phi;
                        ok[k] = phi >= s_psi[k];
                        zmk[k] = z + st->alpha[k] * dz;
                    }
                    if (phase == PH_NEWTON) {
                        st->dpsi = s_dpsi;
                        st->dphi = dz;
                        newton_decide(st, s_psi[0], st->phi[0], s_dpsi, dz, zmk[0]);
                    } else if (phase == PH_BACKOFF) {
                        backoff_decide(st, ok[0]);
                    } else {
                        search_decide(st, ok, zmk);
                    }
                    cs.go = (st->status == ST_RUNNING && st->phase != PH_DONE) ? 1 : 0;
                    cs.phase = st->phase;
                    cs.kpass = st->kpass;
                    if (!cs.go) bt_step_end(cs, st);
                }
                __syncthreads();
                if (!cs.go) break;
            }
            // a8: x += alpha d, y += alpha dy (z += alpha dz in bt_step_end); a search
            // that accepted no step >= 1 (or ran out of passes) ends the probe infeasible
            if (!cs.acc) break;
            const float af = cs.af;
            for (int64_t e = tid; e < E; e += S) x[e] = fmaf(af, d[e], x[e]);
            for (int64_t w = tid; w < n; w += S) y[w] = fmaf(af, dy[w], y[w]);
        }
        // certificate of the probe's x: 1^T x / max(Px), with y recomputed from x
        double v[1] = {0.0};   // FP32 over runs of 8 edges, folded into FP64
        {
            float run = 0.0f;
            int cnt = 0;
            for (int64_t e = tid; e < E; e += S) {
                run += x[e];
                if (++cnt == 8) { v[0] += (double)run; run = 0.0f; cnt = 0; }
            }
            v[0] += (double)run;
        }
        double o[1];
        crew_sums(cw, v, o, sm);   // (orders the last x writes before the gathers)
        bt_rows(cw, vp, ei, bnd, x, y, n);
        __syncthreads();
        float ym = 0.0f;
        for (int64_t w = tid; w < n; w += S) ym = fmaxf(ym, y[w]);
        ym = crew_max(cw, ym, smf);
        if (threadIdx.x == 0) {
            cs.evals += st->evals;
            cs.passes += st->total_passes;
            cs.iters += cs.it;
            cs.probes += 1;
            const double cert = ym > 0.0f ? o[0] / (double)ym : 0.0;
            cs.best = fmax(cs.best, cert);
            cs.lo = fmax(cs.lo, cert);
            if (cs.status == ST_FEASIBLE) cs.lo = fmax(cs.lo, cs.M);
            else cs.hi = fmin(cs.hi, cs.M);
        }
        __syncthreads();
    }
    if (cw.rank == 0 && threadIdx.x == 0) {
        B.obj[inst] = cs.best;
        B.iters[inst] = cs.iters;
        B.probes[inst] = cs.probes;
        B.evals[inst] = cs.evals;
        B.passes[inst] = cs.passes;
        B.t_end[inst] = (int64_t)globaltimer_ns();
    }
}

// Block-alone solves of the instances order[n_cluster ..] from queue[1]
template <int NT> __device__ void bt_alone(const BatchDesc &B, DevState *st, double *slot) {
    __shared__ int s_q;
    Crew<NT, 1> cw{0u, 0, slot};
    for (;;) {
        if (threadIdx.x == 0) s_q = (int)atomicAdd(B.queue + 1, 1u);
        __syncthreads();
        const int q = B.n_cluster + s_q;
        __syncthreads();
        if (q >= B.count) return;
        bt_solve<NT, 1>(B, B.order[q], st, cw);
        __syncthreads();
    }
}

template <int NT, int C>
__global__ void __launch_bounds__(NT) k_batch_solve(BatchDesc B) {
    __shared__ double slot[2 * XS];
    // the search state lives in shared memory: thread 0's decision rules touch
    // it dozens of times per pass, each a dependent access
    __shared__ DevState st_sh;
    DevState *st = &st_sh;
    if constexpr (C > 1) {
        // the cluster's instances: rank 0 takes the next from queue[0] and
        // publishes it; all C blocks solve it together
        __shared__ int s_q;
        Crew<NT, C> cw{cluster_rank(), 0, slot};
        for (;;) {
            double *sl = cw.next();
            if (cw.rank == 0 && threadIdx.x == 0) sl[0] = (double)atomicAdd(B.queue, 1u);
            cluster_barrier();
            if (threadIdx.x == 0) s_q = (int)ld_peer(sl, 0);
            __syncthreads();
            const int q = s_q;
            __syncthreads();
            if (q >= B.n_cluster) break;
            bt_solve<NT, C>(B, B.order[q], st, cw);
        }
        cluster_barrier();   // no block reads a peer's shared memory past this point
    }
    bt_alone<NT>(B, st, slot);
}

template <int NT, int C> static cudaError_t batch_launch_cfg(const BatchDesc &B, int blocks, cudaStream_t s) {
    if constexpr (C == 1) {
        k_batch_solve<NT, 1><<<blocks, NT, 0, s>>>(B);
        return cudaGetLastError();
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)blocks);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_batch_solve<NT, C>, B);
    }
}

template <int NT, int C> static int batch_blocks_cfg(int n_sms) {
    if constexpr (C == 1) {
        int a = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_solve<NT, 1>, NT, 0);
        return n_sms * std::min(8, a > 0 ? a : 1);
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(C * n_sms));
        cfg.blockDim = dim3(NT);
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (C > 8 && cudaFuncSetAttribute(k_batch_solve<NT, C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                         cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, k_batch_solve<NT, C>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return std::min(ncl * C, (n_sms * 8 / C) * C);
    }
}

#define MWU_BATCH_CFGS(X) \
    X(256, 1) X(512, 1) X(1024, 1) X(256, 4) X(512, 4) X(256, 8) X(512, 8) X(256, 16) X(512, 16)

cudaError_t launch_batch_solve(const BatchDesc &Bin, int nt, int cl, int n_cluster, int blocks, cudaStream_t s) {
    BatchDesc B = Bin;
    B.n_cluster = cl > 1 ? n_cluster : 0;
    cudaError_t e = cudaMemsetAsync(B.queue, 0, 2 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
#define MWU_BATCH_LAUNCH(a, b) \
    if (nt == a && cl == b) return batch_launch_cfg<a, b>(B, blocks, s);
    MWU_BATCH_CFGS(MWU_BATCH_LAUNCH)
#undef MWU_BATCH_LAUNCH
    return cudaErrorInvalidValue;
}

int batch_blocks(int nt, int cl, int n_sms) {
#define MWU_BATCH_BLOCKS(a, b) \
    if (nt == a && cl == b) return batch_blocks_cfg<a, b>(n_sms);
    MWU_BATCH_CFGS(MWU_BATCH_BLOCKS)
#undef MWU_BATCH_BLOCKS
    return 0;
}

// ============================================================ active-row compaction
// (drop_covered on the vertex-cover split view) a stable stream compaction of
// the covering rows with v < hi: per tile of CMP_TILE rows (eight consecutive
// rows per thread) a count, one exclusive scan over the tiles, then a scatter
// at each tile's offset plus the in-tile prefix.  Fixed order, no atomics.
__device__ __forceinline__ int block_excl_scan_int(int v, int *sm_w, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = v;
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += o;
    }
    if (lane == 31) sm_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < BLOCK / 32 ? sm_w[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += o;
        }
        if (lane < BLOCK / 32) sm_w[lane] = t;   // inclusive over the warps
    }
    __syncthreads();
    total = sm_w[BLOCK / 32 - 1];
    const int before = w > 0 ? sm_w[w - 1] : 0;
    __syncthreads();
    return before + inc - v;
}

template <class T>
__global__ void __launch_bounds__(BLOCK) k_cmp_count(const T *v, int64_t m, T hi, int32_t *tile_cnt) {
    __shared__ int sm_w[32];
    const int64_t tiles = cmp_tiles(m);
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t base = t * CMP_TILE + (int64_t)threadIdx.x * 8;
        int c = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) c += (base + r < m && v[base + r] < hi) ? 1 : 0;
        int tot;
        block_excl_scan_int(c, sm_w, tot);
        if (threadIdx.x == 0) tile_cnt[t] = tot;
    }
}

// exclusive scan of the tile counts in place (one block), the total to *total
__global__ void __launch_bounds__(BLOCK) k_cmp_scan(int32_t *tile_cnt, int64_t tiles, int64_t *total) {
    __shared__ long long sm_l[32];
    const int64_t chunk = (tiles + BLOCK - 1) / BLOCK;
    const int64_t b = (int64_t)threadIdx.x * chunk, e = min(tiles, b + chunk);
    long long sum = 0;
    for (int64_t i = b; i < e; ++i) sum += tile_cnt[i];
    // exclusive scan of the thread sums (64-bit)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = sum;
    for (int off = 1; off < 32; off <<= 1) {
        const long long o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += o;
    }
    if (lane == 31) sm_l[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long t = lane < BLOCK / 32 ? sm_l[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const long long o = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += o;
        }
        if (lane < BLOCK / 32) sm_l[lane] = t;
    }
    __syncthreads();
    long long off = (w > 0 ? sm_l[w - 1] : 0) + inc - sum;
    for (int64_t i = b; i < e; ++i) {
        const int32_t c = tile_cnt[i];
        tile_cnt[i] = (int32_t)off;
        off += c;
    }
    if (threadIdx.x == 0) *total = sm_l[BLOCK / 32 - 1];
}

template <class T>
__global__ void __launch_bounds__(BLOCK) k_cmp_scatter(const int2 *pairs, const T *v, const int32_t *orig, int64_t m,
                                                       T hi, const int32_t *tile_off, int2 *pairs_o, T *v_o,
                                                       int32_t *orig_o) {
    __shared__ int sm_w[32];
    const int64_t tiles = cmp_tiles(m);
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t base = t * CMP_TILE + (int64_t)threadIdx.x * 8;
        T vv[8];
        int c = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            vv[r] = base + r < m ? v[base + r] : hi;
            c += vv[r] < hi ? 1 : 0;
        }
        int tot;
        int64_t pos = (int64_t)tile_off[t] + block_excl_scan_int(c, sm_w, tot);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            if (vv[r] < hi) {
                const int64_t j = base + r;
                pairs_o[pos] = pairs[j];
                v_o[pos] = vv[r];
                orig_o[pos] = orig ? orig[j] : (int32_t)j;
                ++pos;
            }
        }
    }
}

template <class T>
__global__ void __launch_bounds__(BLOCK) k_cmp_refresh(Problem<T> p) {
    const Side<T> &sd = p.side[1];
    const int2 *ed = reinterpret_cast<const int2 *>(sd.rv.idx);
    const T scale = (T)p.st->scale[1];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < sd.m; j += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = ed[j];
        sd.v[j] = (p.x[e.x] + p.x[e.y]) * scale;
    }
}

static int cmp_grid(int64_t tiles) { return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 152 * 16)); }

template <class T>
cudaError_t launch_cmp_count(const T *v, int64_t m, double hi, int32_t *tile_off, int64_t *total, cudaStream_t s) {
    const int64_t tiles = cmp_tiles(m);
    if (tiles == 0) return cudaMemsetAsync(total, 0, sizeof(int64_t), s);
    k_cmp_count<T><<<cmp_grid(tiles), BLOCK, 0, s>>>(v, m, (T)hi, tile_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cmp_scan<<<1, BLOCK, 0, s>>>(tile_off, tiles, total);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_cmp_scatter(const int32_t *pairs, const T *v, const int32_t *orig, int64_t m, double hi,
                               const int32_t *tile_off, int32_t *pairs_o, T *v_o, int32_t *orig_o, cudaStream_t s) {
    const int64_t tiles = cmp_tiles(m);
    if (tiles == 0) return cudaSuccess;
    k_cmp_scatter<T><<<cmp_grid(tiles), BLOCK, 0, s>>>(reinterpret_cast<const int2 *>(pairs), v, orig, m, (T)hi,
                                                       tile_off, reinterpret_cast<int2 *>(pairs_o), v_o, orig_o);
    return cudaGetLastError();
}

template <class T> cudaError_t launch_cmp_refresh(const Problem<T> &p, cudaStream_t s) {
    k_cmp_refresh<T><<<grid_for(p.side[1].m, p.grid_upd), BLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

#define MWU_INSTANTIATE(T)                                                                                     \
    template cudaError_t launch_x_init<T>(const Problem<T> &, cudaStream_t);                                   \
    template cudaError_t launch_x_set<T>(const Problem<T> &, const void *, int, cudaStream_t);                 \
    template cudaError_t launch_rows_eval<T>(const Problem<T> &, cudaStream_t);                                \
    template cudaError_t launch_rows_reduce<T>(const Problem<T> &, cudaStream_t);                              \
    template cudaError_t launch_dense_dir<T>(const Problem<T> &, cudaStream_t);                                \
    template cudaError_t launch_dir<T>(const Problem<T> &, int, cudaStream_t);                                 \
    template cudaError_t launch_spmv<T>(const Problem<T> &, cudaStream_t, int);                                \
    template cudaError_t launch_cand<T>(const Problem<T> &, int, cudaStream_t);                                \
    template cudaError_t launch_cand_newton<T>(const Problem<T> &, cudaStream_t);                              \
    template int newton_blocks_per_sm<T>();                                                                     \
    template cudaError_t launch_update<T>(const Problem<T> &, cudaStream_t);                                   \
    template cudaError_t launch_flush<T>(const Problem<T> &, cudaStream_t);                                    \
    template cudaError_t launch_search_begin<T>(const Problem<T> &, cudaStream_t);                             \
    template cudaError_t launch_potential_grads<T>(const Problem<T> &, const float *, float *, float *,        \
                                                   float *, float *, cudaStream_t);                            \
    template cudaError_t launch_copy_vec<T>(const T *, void *, int64_t, int, cudaStream_t);                    \
    template int sweep_blocks_per_sm<T>(int *, int *, int *);                                                  \
    template int spmv_blocks_per_sm<T>();                                                                      \
    template int tiled_blocks_per_sm<T>();                                                                     \
    template cudaError_t launch_cmp_count<T>(const T *, int64_t, double, int32_t *, int64_t *, cudaStream_t);     \
    template cudaError_t launch_cmp_scatter<T>(const int32_t *, const T *, const int32_t *, int64_t, double,       \
                                               const int32_t *, int32_t *, T *, int32_t *, cudaStream_t);          \
    template cudaError_t launch_cmp_refresh<T>(const Problem<T> &, cudaStream_t);

MWU_INSTANTIATE(float)
MWU_INSTANTIATE(double)

}  // namespace mwu

// ============================================================ allocation-free candidates
// mwu_candidates_static (mwu.h): the candidate evaluation of one side with its
// scratch in a static device array instead of context buffers.
#include <mutex>

namespace mwu {
namespace stat {

constexpr int MAXB = MWU_STATIC_MAX_BLOCKS;
constexpr int RPB = MWU_STATIC_ROWS_PER_BLOCK;

struct Scratch {
    double rec[MAXB][KMAX][4];   // per-block (mx, R, T, min) of every candidate
    double out[KMAX][2];         // value and min(v + alpha dv) per candidate
    unsigned int ticket;         // completion count; the last block resets it to 0
};

__global__ void __launch_bounds__(BLOCK) k_cand_static(Scratch *scr, const float *v, const float *dv, int64_t m,
                                                       int sign, double eta, double shift, double S,
                                                       CandSched<float> sc) {
    CandAcc<float> acc;
    cand_init(acc, sign);
    const float eta_f = (float)eta, sh = (float)shift;
    const int64_t r0 = (int64_t)blockIdx.x * RPB, r1 = min(m, r0 + RPB);
    const float camax = sched_camax(sc.ca, sc.K);
    for (int64_t j = r0 + threadIdx.x; j < r1; j += blockDim.x) {
        if (sign > 0)
            cand_push_m<float, 2, 1, 0>(acc, sc.ca, sc.al, sc.cd, sc.K, v[j], dv[j], eta_f, sh, sc.hi, camax);
        else
            cand_push_m<float, 2, -1, 0>(acc, sc.ca, sc.al, sc.cd, sc.K, v[j], dv[j], eta_f, sh, sc.hi, camax);
    }
    // block merge (as in k_cand), record to the static array
    __shared__ double wm[BLOCK / 32][KMAX][4];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        float mx = acc.mx[k], R = acc.R[k], Tt = acc.Tt[k], zm = acc.zm[k];
        for (int off = 16; off > 0; off >>= 1) {
            float omx = shfl_x(mx, off), oR = shfl_x(R, off), oT = shfl_x(Tt, off), oz = shfl_x(zm, off);
            cand_merge1<float, float>(mx, R, Tt, zm, omx, oR, oT, oz, sign);
        }
        if ((threadIdx.x & 31) == 0) {
            wm[threadIdx.x >> 5][k][0] = mx; wm[threadIdx.x >> 5][k][1] = R;
            wm[threadIdx.x >> 5][k][2] = Tt; wm[threadIdx.x >> 5][k][3] = zm;
        }
    }
    __syncthreads();
    if (threadIdx.x < KMAX) {
        const int k = threadIdx.x;
        double mx = sign > 0 ? 0.0 : -(double)INFINITY, R = 0.0, Tt = 0.0, zm = (double)INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            cand_merge1<float, double>(mx, R, Tt, zm, wm[w][k][0], wm[w][k][1], wm[w][k][2], wm[w][k][3], sign);
        scr->rec[blockIdx.x][k][0] = mx; scr->rec[blockIdx.x][k][1] = R;
        scr->rec[blockIdx.x][k][2] = Tt; scr->rec[blockIdx.x][k][3] = zm;
    }
    if (!last_block_done(&scr->ticket)) return;
    if (threadIdx.x < KMAX) {
        const int k = threadIdx.x;
        double mx = sign > 0 ? 0.0 : -(double)INFINITY, R = 0.0, Tt = 0.0, zm = (double)INFINITY;
        for (int b = 0; b < (int)gridDim.x; ++b)
            cand_merge1<float, double>(mx, R, Tt, zm, scr->rec[b][k][0], scr->rec[b][k][1], scr->rec[b][k][2],
                                       scr->rec[b][k][3], sign);
        // the final combination (one thread per candidate) runs in FP64
        const double lS0 = log(S);
        double val;
        if (sign > 0) {
            double lq = mx + log(Tt) - lS0;
            val = (lq < 0.0) ? log1p(exp(lq)) / eta : (mx + log(R) - lS0) / eta;
        } else {
            double qv = Tt / S;
            val = (qv <= 0.5) ? -log1p(-qv) / eta : -(mx + log(R) - lS0) / eta;
        }
        scr->out[k][0] = val;
        scr->out[k][1] = zm;
    }
    if (threadIdx.x == 0) scr->ticket = 0;
}

// The scratch of every call: one copy per device that loads the library.
static __device__ __align__(256) Scratch g_static_scratch;

constexpr int MAXDEV = 64;
static std::mutex g_mu;
static Scratch *g_ptr[MAXDEV] = {nullptr};

// Once per device, with that device current: the device address of the array
// (its host-side name is only a stand-in) and a cleared completion ticket.
static int device_scratch(Scratch **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) {
        cudaGetLastError();
        set_global_error("mwu_candidates_static: no usable CUDA device");
        return MWU_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_global_error((std::string("mwu_candidates_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
            return MWU_ERR_CUDA;
        }
        Scratch *sp = static_cast<Scratch *>(p);
        e = cudaMemset(&sp->ticket, 0, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            set_global_error((std::string("mwu_candidates_static: clearing the ticket: ") + cudaGetErrorString(e)).c_str());
            return MWU_ERR_CUDA;
        }
        g_ptr[dev] = sp;
    }
    *out = g_ptr[dev];
    return MWU_OK;
}

}  // namespace stat
}  // namespace mwu

extern "C" int mwu_candidates_static(const float *v, const float *dv, int64_t m, int32_t sign, double eta,
                                     double shift, double S, const double *alphas, int32_t K, double *val,
                                     double *vmin, void *stream) {
    using namespace mwu;
    if (!v || !dv || !alphas || !val || m <= 0 || (sign != 1 && sign != -1) || K < 1 || K > KMAX ||
        !(eta > 0.0) || !(S > 0.0) || !std::isfinite(shift)) {
        set_global_error("mwu_candidates_static: bad argument (null pointer, m <= 0, sign not +-1, K not in 1..8, "
                         "eta <= 0 or S <= 0)");
        return MWU_ERR_INVALID;
    }
    if (m > MWU_STATIC_MAX_ROWS) {
        set_global_error("mwu_candidates_static: m exceeds MWU_STATIC_MAX_ROWS (the static scratch holds "
                         "MWU_STATIC_MAX_BLOCKS block records of MWU_STATIC_ROWS_PER_BLOCK rows)");
        return MWU_ERR_INVALID;
    }
    stat::Scratch *scr = nullptr;
    int rc = stat::device_scratch(&scr);
    if (rc != MWU_OK) return rc;
    CandSched<float> sc{};
    sc.K = K;
    sc.mode = 2;
    sc.cd = 0.0f;
    sc.hi = INFINITY;   // every row of the given side counts
    for (int k = 0; k < KMAX; ++k) {
        double a = k < K ? alphas[k] : 0.0;
        sc.ca[k] = (float)(a * eta);
        sc.al[k] = (float)a;
    }
    const int grid = (int)((m + stat::RPB - 1) / stat::RPB);
    cudaStream_t s = (cudaStream_t)stream;
    stat::k_cand_static<<<grid, BLOCK, 0, s>>>(scr, v, dv, m, sign, eta, shift, S, sc);
    cudaError_t e = cudaGetLastError();
    double out[KMAX][2];
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, scr->out, sizeof(out), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_global_error((std::string("mwu_candidates_static: ") + cudaGetErrorString(e)).c_str());
        return MWU_ERR_CUDA;
    }
    for (int k = 0; k < K; ++k) {
        val[k] = out[k][0];
        if (vmin) vmin[k] = out[k][1];
    }
    return MWU_OK;
}

// ---------------------------------------------------------------- diagnostics
namespace mwu {
__global__ void k_diag_ome(const float *b, float *u, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = one_minus_exp_neg(b[i]);
}
}   // namespace mwu

extern "C" int mwu_diag_one_minus_exp_neg(const float *b, float *u, int64_t n, void *stream) {
    if (!b || !u || n < 0) return MWU_ERR_INVALID;
    if (n == 0) return MWU_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    mwu::k_diag_ome<<<grid, 256, 0, (cudaStream_t)stream>>>(b, u, n);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    return e == cudaSuccess ? MWU_OK : MWU_ERR_CUDA;
}
