// Forward product dv = A d of a CSR constraint side by scatter over the
// columns of the variables that move (option dv_scatter; a6 of the iteration,
// Alg. 2's dz = C d).
//
// The direction test leaves d_i = 0 for every variable with g_i >= h_i, and
// late in a probe most variables are such.  The row-wise gather of the SpMV
// reads every entry of A whatever d holds; this form reads only the columns
// of the variables with d_i > 0 (the column view that the direction kernel
// uses for h) and adds d_i A_ji into dv[j] with atomic adds, then scales the
// rows by their coefficient.  The order of the adds depends on scheduling,
// so the last bits of dv vary from run to run (the option is off by default).
#include "mwu_internal.cuh"

#include <algorithm>

namespace mwu {

namespace {

// sum of v over the G lanes of each group (G a power of two <= 32)
template <class T> __device__ __forceinline__ T group_total(T v, int G) {
    for (int off = G >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <class T>
__device__ __forceinline__ void scatter_column(const ColView &cv, T *dv, int64_t i, T di, int first, int step) {
    for (int k = cv.ptr[i] + first; k < cv.ptr[i + 1]; k += step)
        atomicAdd(&dv[cv.idx[k]], cv.val ? di * (T)cv.val[k] : di);
}

// One pass over the variables in the direction kernel's length classes:
// heavy columns a block each, medium a warp each, light ones G lanes each.
template <class T>
__global__ void __launch_bounds__(BLOCK) k_dv_scatter(Problem<T> p, int s) {
    const DevState *st = p.st;
    if (st->status != ST_RUNNING) return;
    const Side<T> &sd = p.side[s];
    const ColView &cv = sd.cv;
    T *dv = sd.dv;
    for (int hh = blockIdx.x; hh < p.n_heavy_var; hh += gridDim.x) {
        const int64_t i = p.heavy_var[hh];
        const T di = p.d[i];
        if (di > T(0)) scatter_column(cv, dv, i, di, (int)threadIdx.x, (int)blockDim.x);
    }
    {
        const int wl = threadIdx.x & 31;
        const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < p.n_med_var; q += nw) {
            const int64_t i = p.med_var[q];
            const T di = p.d[i];
            if (di > T(0)) scatter_column(cv, dv, i, di, wl, 32);
        }
    }
    const int G = p.G_var, lane = threadIdx.x & (G - 1);
    const int64_t per_block = blockDim.x / G;
    const int64_t stride = (int64_t)gridDim.x * per_block;
    for (int64_t i = (int64_t)blockIdx.x * per_block + threadIdx.x / G; i < p.n; i += stride) {
        const T di = p.d[i];
        if (!(di > T(0))) continue;
        const ColView &P = p.side[0].cv, &C = p.side[1].cv;
        const bool light = (P.kind != CK_CSR || P.ptr[i + 1] - P.ptr[i] <= P.heavy_len) &&
                           (C.kind != CK_CSR || C.ptr[i + 1] - C.ptr[i] <= C.heavy_len);
        if (light) scatter_column(cv, dv, i, di, lane, G);
    }
}

// dv_j *= coef_j = scale_s / rdiv_j (the sums above are of A_jk d_k)
template <class T>
__global__ void __launch_bounds__(BLOCK) k_dv_rowcoef(Problem<T> p, int s) {
    const DevState *st = p.st;
    if (st->status != ST_RUNNING) return;
    const Side<T> &sd = p.side[s];
    const T scale = (T)st->scale[s];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < sd.m; j += (int64_t)gridDim.x * blockDim.x)
        sd.dv[j] *= sd.rv.rdiv ? scale / (T)sd.rv.rdiv[j] : scale;
}

}  // namespace

template <class T> cudaError_t launch_spmv_scatter(const Problem<T> &p, int s, cudaStream_t stream) {
    const Side<T> &sd = p.side[s];
    cudaError_t e = cudaMemsetAsync(sd.dv, 0, sizeof(T) * (size_t)sd.m, stream);
    if (e != cudaSuccess) return e;
    const int64_t per_block = BLOCK / p.G_var;
    const int64_t need = std::max<int64_t>((p.n + per_block - 1) / per_block, p.n_heavy_var);
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(need, p.grid_var));
    k_dv_scatter<T><<<g, BLOCK, 0, stream>>>(p, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int gr = (int)std::max<int64_t>(1, std::min<int64_t>((sd.m + BLOCK - 1) / BLOCK, p.grid_upd));
    k_dv_rowcoef<T><<<gr, BLOCK, 0, stream>>>(p, s);
    return cudaGetLastError();
}

template cudaError_t launch_spmv_scatter<float>(const Problem<float> &, int, cudaStream_t);
template cudaError_t launch_spmv_scatter<double>(const Problem<double> &, int, cudaStream_t);

}  // namespace mwu
