// Setup-time construction of the row and column views of the paper's graph
// matrices (Sec. 3) and of explicit CSR matrices, plus input validation.
// Runs once per context in mwu_create, never inside an MWU iteration.
//
//   vertex -> slot lists : for an edge list (u_e, v_e), slot 2e+b holds
//                          endpoint b of e; a stable radix sort of the slots by
//                          vertex gives, per vertex, its incident slots in
//                          increasing order.  Incidence M (Eq. incidence) uses
//                          slot >> 1 (the edge), the pair matrix O (Eq.
//                          oddshifted_incidence) uses the slot itself.
//   CSR transpose        : stable sort of the nonzeros by column.
//   heavy lists          : rows longer than a threshold, in increasing order.
// Sorting and scans use CUB (setup only; the sweep kernels are hand-written).
#include "mwu_setup.cuh"

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

#include <cmath>

namespace mwu {

// ------------------------------------------------------------ validation
__global__ void k_check_csr(const int32_t *ptr, const int32_t *idx, const float *val, int64_t rows, int64_t cols,
                            int64_t nnz, int require_nonempty, int *err) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.x * blockDim.x) {
        int a = ptr[j], b = ptr[j + 1];
        if (a < 0 || b < a || b > nnz) { atomicMax(err, 1); continue; }
        if (require_nonempty && b == a) atomicMax(err, 4);
    }
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        int c = idx[k];
        if (c < 0 || c >= cols) atomicMax(err, 2);
        if (val) {
            float v = val[k];
            if (!(v >= 0.0f) || !isfinite(v)) atomicMax(err, 3);
        }
    }
}

__global__ void k_check_edges(const int32_t *e, int64_t m, int32_t nv, int *err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        int a = e[2 * k], b = e[2 * k + 1];
        if (a < 0 || a >= nv || b < 0 || b >= nv) atomicMax(err, 5);
        else if (a == b) atomicMax(err, 6);
    }
}

__global__ void k_check_pos(const float *v, int64_t n, int *err, int code) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        float a = v[k];
        if (!(a > 0.0f) || !isfinite(a)) atomicMax(err, code);
    }
}

__global__ void k_check_nonneg(const float *v, int64_t n, int *err, int code) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        float a = v[k];
        if (!(a >= 0.0f) || !isfinite(a)) atomicMax(err, code);
    }
}

static int g1d(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g < 1) g = 1;
    if (g > 8192) g = 8192;
    return (int)g;
}

const char *validation_message(int code) {
    switch (code) {
    case 1: return "CSR row pointer not monotone or out of range";
    case 2: return "CSR column index out of range";
    case 3: return "CSR value negative, NaN or infinite";
    case 4: return "empty covering row (the covering LP is infeasible)";
    case 5: return "edge endpoint out of range";
    case 6: return "self loop in the edge list";
    case 7: return "row bound not positive and finite";
    case 8: return "objective coefficient negative, NaN or infinite";
    case 9: return "vertex without incident edge in a covering incidence row";
    default: return "invalid input";
    }
}

cudaError_t validate_csr(const int32_t *ptr, const int32_t *idx, const float *val, int64_t rows, int64_t cols,
                         int64_t nnz, int require_nonempty, int *d_err, cudaStream_t s) {
    k_check_csr<<<g1d(rows > nnz ? rows : nnz), 256, 0, s>>>(ptr, idx, val, rows, cols, nnz, require_nonempty, d_err);
    return cudaGetLastError();
}
cudaError_t validate_edges(const int32_t *e, int64_t m, int32_t nv, int *d_err, cudaStream_t s) {
    k_check_edges<<<g1d(m), 256, 0, s>>>(e, m, nv, d_err);
    return cudaGetLastError();
}
cudaError_t validate_positive(const float *v, int64_t n, int code, int *d_err, cudaStream_t s) {
    k_check_pos<<<g1d(n), 256, 0, s>>>(v, n, d_err, code);
    return cudaGetLastError();
}
cudaError_t validate_nonneg(const float *v, int64_t n, int code, int *d_err, cudaStream_t s) {
    k_check_nonneg<<<g1d(n), 256, 0, s>>>(v, n, d_err, code);
    return cudaGetLastError();
}

// ------------------------------------------------------------ building blocks
__global__ void k_iota(int32_t *a, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        a[k] = (int32_t)k;
}
__global__ void k_count(const int32_t *keys, int64_t n, int32_t *cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[keys[k]], 1);
}
__global__ void k_rows_of_nnz(const int32_t *ptr, int64_t rows, int32_t *row_of) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.x * blockDim.x)
        for (int k = ptr[j]; k < ptr[j + 1]; ++k) row_of[k] = (int32_t)j;
}
__global__ void k_gather_i(const int32_t *src, const int32_t *perm, int32_t *dst, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[perm[k]];
}
__global__ void k_gather_f(const float *src, const int32_t *perm, float *dst, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[perm[k]];
}
__global__ void k_shift_right1(const int32_t *src, int32_t *dst, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[k] >> 1;
}
__global__ void k_heavy_flags(const int32_t *ptr, int64_t rows, int thr, char *flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.x * blockDim.x)
        flag[j] = (ptr[j + 1] - ptr[j]) > thr;
}
__global__ void k_heavy_flags2(const int32_t *p1, int thr1, const int32_t *p2, int thr2, int64_t rows, char *flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.x * blockDim.x) {
        bool h = false;
        if (p1) h |= (p1[j + 1] - p1[j]) > thr1;
        if (p2) h |= (p2[j + 1] - p2[j]) > thr2;
        flag[j] = h;
    }
}

// rows whose longer column over the two views has a length in (lo, hi]
__global__ void k_range_flags2(const int32_t *p1, const int32_t *p2, int64_t rows, int lo, int hi, char *flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.x * blockDim.x) {
        int len = 0;
        if (p1) len = max(len, p1[j + 1] - p1[j]);
        if (p2) len = max(len, p2[j + 1] - p2[j]);
        flag[j] = len > lo && len <= hi;
    }
}

// Histogram of the longer column length per row in power-of-two buckets:
// bucket 0 holds lengths 0 and 1, bucket b > 0 lengths in (2^(b-1), 2^b].
__global__ void k_len_hist(const int32_t *p1, const int32_t *p2, int64_t rows, unsigned long long *hist) {
    __shared__ unsigned int h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.x * blockDim.x) {
        int len = 0;
        if (p1) len = max(len, p1[j + 1] - p1[j]);
        if (p2) len = max(len, p2[j + 1] - p2[j]);
        const int b = len <= 1 ? 0 : 32 - __clz(len - 1);
        atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

// Exclusive scan of counts[0..n) into ptr[0..n] (ptr[n] = total), int32.
static cudaError_t scan_counts(Arena &ar, const int32_t *cnt, int32_t *ptr, int64_t n, cudaStream_t s) {
    size_t tmp = 0;
    cudaError_t e = cub::DeviceScan::InclusiveSum(nullptr, tmp, cnt, ptr + 1, (int)n, s);
    if (e != cudaSuccess) return e;
    void *t = ar.scratch(tmp);
    if (!t) return cudaErrorMemoryAllocation;
    if ((e = cudaMemsetAsync(ptr, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    return cub::DeviceScan::InclusiveSum(t, tmp, cnt, ptr + 1, (int)n, s);
}

// Stable sort of (key, value) int32 pairs by key (bits: key range).
static cudaError_t sort_pairs(Arena &ar, const int32_t *kin, int32_t *kout, const int32_t *vin, int32_t *vout,
                              int64_t n, int key_bits, cudaStream_t s) {
    size_t tmp = 0;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, tmp, kin, kout, vin, vout, (int)n, 0, key_bits, s);
    if (e != cudaSuccess) return e;
    void *t = ar.scratch(tmp);
    if (!t) return cudaErrorMemoryAllocation;
    return cub::DeviceRadixSort::SortPairs(t, tmp, kin, kout, vin, vout, (int)n, 0, key_bits, s);
}

static int bits_for(int64_t range) {
    int b = 1;
    while ((int64_t(1) << b) < range) ++b;
    return b;
}

cudaError_t build_vertex_slots(Arena &ar, const int32_t *edges, int64_t m, int32_t nv, int32_t **ptr_out,
                               int32_t **slots_out, cudaStream_t s) {
    int64_t ns = 2 * m;
    int32_t *ptr = ar.alloc<int32_t>(nv + 1);
    int32_t *slots = ar.alloc<int32_t>(ns);
    int32_t *cnt = (int32_t *)ar.scratch_keep(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    int32_t *iota = ar.alloc_tmp<int32_t>(ns);
    int32_t *kout = ar.alloc_tmp<int32_t>(ns);
    if (!ptr || !slots || !cnt || !iota || !kout) return cudaErrorMemoryAllocation;
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)nv, s)) != cudaSuccess) return e;
    k_count<<<g1d(ns), 256, 0, s>>>(edges, ns, cnt);
    if ((e = scan_counts(ar, cnt, ptr, nv, s)) != cudaSuccess) return e;
    k_iota<<<g1d(ns), 256, 0, s>>>(iota, ns);
    if ((e = sort_pairs(ar, edges, kout, iota, slots, ns, bits_for(nv), s)) != cudaSuccess) return e;
    ar.release_tmp();
    *ptr_out = ptr;
    *slots_out = slots;
    return cudaGetLastError();
}

cudaError_t slots_to_edges(Arena &ar, const int32_t *slots, int64_t ns, int32_t **out, cudaStream_t s) {
    int32_t *e = ar.alloc<int32_t>(ns);
    if (!e) return cudaErrorMemoryAllocation;
    k_shift_right1<<<g1d(ns), 256, 0, s>>>(slots, e, ns);
    *out = e;
    return cudaGetLastError();
}

// flag[0] = 1 when the edge list's first endpoints decrease anywhere
__global__ void k_first_sorted(const int32_t *edges, int64_t m, int *flag) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e + 1 < m; e += (int64_t)gridDim.x * blockDim.x)
        if (edges[2 * (e + 1)] < edges[2 * e]) atomicMax(flag, 1);
}
__global__ void k_count_endpoint(const int32_t *edges, int64_t m, int b, int32_t *cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[edges[2 * e + b]], 1);
}
__global__ void k_endpoint(const int32_t *edges, int64_t m, int b, int32_t *out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = edges[2 * e + b];
}
__global__ void k_first_of(const int32_t *edges, const int32_t *perm, int64_t m, int32_t *out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = edges[2 * (int64_t)perm[k]];
}
__global__ void k_add_ptr(const int32_t *a, const int32_t *b, int64_t n, int32_t *out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = a[k] + b[k];
}

cudaError_t build_split_view(Arena &ar, const int32_t *edges, int64_t m, int32_t nv, int32_t **cptr_out,
                             int32_t **vptr_out, int32_t **u2_out, int *sorted, cudaStream_t s) {
    *sorted = 0;
    int *flag = (int *)ar.scratch_keep(sizeof(int));
    if (!flag) return cudaErrorMemoryAllocation;
    cudaError_t e;
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), s)) != cudaSuccess) return e;
    k_first_sorted<<<g1d(m), 256, 0, s>>>(edges, m, flag);
    int h = 0;
    if ((e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (h != 0) return cudaSuccess;   // not sorted by first endpoint: the caller keeps the gather view
    int32_t *cptr = ar.alloc<int32_t>(nv + 1);
    int32_t *vptr = ar.alloc<int32_t>(nv + 1);
    int32_t *u2 = ar.alloc<int32_t>(m);
    int32_t *uptr = ar.alloc_tmp<int32_t>(nv + 1);
    int32_t *cnt = ar.alloc_tmp<int32_t>(nv);
    int32_t *keys = ar.alloc_tmp<int32_t>(m);
    int32_t *kout = ar.alloc_tmp<int32_t>(m);
    int32_t *iota = ar.alloc_tmp<int32_t>(m);
    int32_t *perm = ar.alloc_tmp<int32_t>(m);
    if (!cptr || !vptr || !u2 || !uptr || !cnt || !keys || !kout || !iota || !perm) return cudaErrorMemoryAllocation;
    for (int b = 0; b < 2; ++b) {
        if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)nv, s)) != cudaSuccess) return e;
        k_count_endpoint<<<g1d(m), 256, 0, s>>>(edges, m, b, cnt);
        if ((e = scan_counts(ar, cnt, b == 0 ? uptr : vptr, nv, s)) != cudaSuccess) return e;
    }
    k_add_ptr<<<g1d(nv + 1), 256, 0, s>>>(uptr, vptr, nv + 1, cptr);
    k_endpoint<<<g1d(m), 256, 0, s>>>(edges, m, 1, keys);
    k_iota<<<g1d(m), 256, 0, s>>>(iota, m);
    if ((e = sort_pairs(ar, keys, kout, iota, perm, m, bits_for(nv), s)) != cudaSuccess) return e;
    k_first_of<<<g1d(m), 256, 0, s>>>(edges, perm, m, u2);
    ar.release_tmp();
    *cptr_out = cptr;
    *vptr_out = vptr;
    *u2_out = u2;
    *sorted = 1;
    return cudaGetLastError();
}

cudaError_t csr_transpose(Arena &ar, const int32_t *ptr, const int32_t *idx, const float *val, int64_t rows,
                          int64_t cols, int64_t nnz, int32_t **tptr, int32_t **tidx, float **tval, cudaStream_t s) {
    int32_t *P = ar.alloc<int32_t>(cols + 1);
    int32_t *I = ar.alloc<int32_t>(nnz > 0 ? nnz : 1);
    float *V = val ? ar.alloc<float>(nnz > 0 ? nnz : 1) : nullptr;
    int32_t *cnt = (int32_t *)ar.scratch_keep(sizeof(int32_t) * (size_t)(cols > 0 ? cols : 1));
    int32_t *row_of = ar.alloc_tmp<int32_t>(nnz > 0 ? nnz : 1);
    int32_t *iota = ar.alloc_tmp<int32_t>(nnz > 0 ? nnz : 1);
    int32_t *perm = ar.alloc_tmp<int32_t>(nnz > 0 ? nnz : 1);
    int32_t *kout = ar.alloc_tmp<int32_t>(nnz > 0 ? nnz : 1);
    if (!P || !I || (val && !V) || !cnt || !row_of || !iota || !perm || !kout) return cudaErrorMemoryAllocation;
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)cols, s)) != cudaSuccess) return e;
    k_count<<<g1d(nnz), 256, 0, s>>>(idx, nnz, cnt);
    if ((e = scan_counts(ar, cnt, P, cols, s)) != cudaSuccess) return e;
    k_rows_of_nnz<<<g1d(rows), 256, 0, s>>>(ptr, rows, row_of);
    k_iota<<<g1d(nnz), 256, 0, s>>>(iota, nnz);
    if ((e = sort_pairs(ar, idx, kout, iota, perm, nnz, bits_for(cols), s)) != cudaSuccess) return e;
    k_gather_i<<<g1d(nnz), 256, 0, s>>>(row_of, perm, I, nnz);
    if (val) k_gather_f<<<g1d(nnz), 256, 0, s>>>(val, perm, V, nnz);
    ar.release_tmp();
    *tptr = P;
    *tidx = I;
    *tval = V;
    return cudaGetLastError();
}

static cudaError_t select_flagged(Arena &ar, const char *flag, int64_t rows, int32_t **list, int32_t *count,
                                  cudaStream_t s) {
    int32_t *iota = ar.alloc_tmp<int32_t>(rows > 0 ? rows : 1);
    int32_t *out = ar.alloc_tmp<int32_t>(rows > 0 ? rows : 1);
    int32_t *nsel = (int32_t *)ar.scratch_keep(sizeof(int32_t));
    if (!iota || !out || !nsel) return cudaErrorMemoryAllocation;
    k_iota<<<g1d(rows), 256, 0, s>>>(iota, rows);
    size_t tmp = 0;
    cudaError_t e = cub::DeviceSelect::Flagged(nullptr, tmp, iota, flag, out, nsel, (int)rows, s);
    if (e != cudaSuccess) return e;
    void *t = ar.scratch(tmp);
    if (!t) return cudaErrorMemoryAllocation;
    if ((e = cub::DeviceSelect::Flagged(t, tmp, iota, flag, out, nsel, (int)rows, s)) != cudaSuccess) return e;
    int32_t h = 0;
    if ((e = cudaMemcpyAsync(&h, nsel, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *count = h;
    if (h > 0) {
        int32_t *L = ar.alloc<int32_t>(h);
        if (!L) return cudaErrorMemoryAllocation;
        if ((e = cudaMemcpyAsync(L, out, sizeof(int32_t) * (size_t)h, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            return e;
        *list = L;
    } else {
        *list = nullptr;
    }
    ar.release_tmp();
    return cudaSuccess;
}

cudaError_t heavy_list(Arena &ar, const int32_t *ptr, int64_t rows, int thr, int32_t **list, int32_t *count,
                       cudaStream_t s) {
    char *flag = ar.alloc_tmp<char>(rows > 0 ? rows : 1);
    if (!flag) return cudaErrorMemoryAllocation;
    k_heavy_flags<<<g1d(rows), 256, 0, s>>>(ptr, rows, thr, flag);
    cudaError_t e = select_flagged(ar, flag, rows, list, count, s);
    return e;
}

__global__ void k_bin_flags(const int32_t *ptr, int64_t rows, int lo, int hi, char *flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.x * blockDim.x) {
        int len = ptr[j + 1] - ptr[j];
        flag[j] = len > lo && len <= hi;
    }
}

cudaError_t bin_list(Arena &ar, const int32_t *ptr, int64_t rows, int lo, int hi, int32_t **list, int32_t *count,
                     cudaStream_t s) {
    char *flag = ar.alloc_tmp<char>(rows > 0 ? rows : 1);
    if (!flag) return cudaErrorMemoryAllocation;
    k_bin_flags<<<g1d(rows), 256, 0, s>>>(ptr, rows, lo, hi, flag);
    return select_flagged(ar, flag, rows, list, count, s);
}

// one block per tile: min and max column over the tile's entries; fit[0]
// counts the tiles whose window fits, fit[1] the entries those tiles hold
__global__ void k_tile_windows(const int32_t *ptr, const int32_t *idx, int64_t rows, int tile_rows, int wmax,
                               int32_t *lo, int32_t *len, unsigned long long *fit) {
    __shared__ int s_lo[8], s_hi[8];
    const int64_t t = blockIdx.x;
    const int64_t r0 = t * tile_rows, r1 = r0 + tile_rows < rows ? r0 + tile_rows : rows;
    int mn = INT32_MAX, mx = -1;
    for (int64_t k = ptr[r0] + threadIdx.x; k < ptr[r1]; k += blockDim.x) {
        const int c = idx[k];
        mn = min(mn, c);
        mx = max(mx, c);
    }
    for (int off = 16; off > 0; off >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    if ((threadIdx.x & 31) == 0) { s_lo[threadIdx.x >> 5] = mn; s_hi[threadIdx.x >> 5] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { mn = min(mn, s_lo[w]); mx = max(mx, s_hi[w]); }
        mn = min(mn, s_lo[0]);
        mx = max(mx, s_hi[0]);
        const int span = mx >= mn ? mx - mn + 1 : 0;
        lo[t] = span > 0 ? mn : 0;
        len[t] = span;
        if (span <= wmax) {
            atomicAdd(fit, 1ull);
            atomicAdd(fit + 1, (unsigned long long)(ptr[r1] - ptr[r0]));
        }
    }
}

cudaError_t build_tiles(Arena &ar, const int32_t *ptr, const int32_t *idx, int64_t rows, int tile_rows, int wmax,
                        int32_t **lo, int32_t **len, int32_t *n_tiles, int32_t *fit, int64_t *fit_nnz, cudaStream_t s) {
    const int64_t nt = (rows + tile_rows - 1) / tile_rows;
    *n_tiles = (int32_t)nt;
    *fit = 0;
    *fit_nnz = 0;
    if (nt <= 0) return cudaSuccess;
    *lo = ar.alloc<int32_t>(nt);
    *len = ar.alloc<int32_t>(nt);
    unsigned long long *d_fit = ar.alloc_tmp<unsigned long long>(2);
    if (!*lo || !*len || !d_fit) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(d_fit, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_tile_windows<<<(unsigned)nt, 256, 0, s>>>(ptr, idx, rows, tile_rows, wmax, *lo, *len, d_fit);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned long long h[2] = {0, 0};
    if ((e = cudaMemcpyAsync(h, d_fit, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *fit = (int32_t)h[0];
    *fit_nnz = (int64_t)h[1];
    return cudaSuccess;
}

cudaError_t range_list2(Arena &ar, const int32_t *p1, const int32_t *p2, int64_t rows, int lo, int hi,
                        int32_t **list, int32_t *count, cudaStream_t s) {
    char *flag = ar.alloc_tmp<char>(rows > 0 ? rows : 1);
    if (!flag) return cudaErrorMemoryAllocation;
    k_range_flags2<<<g1d(rows), 256, 0, s>>>(p1, p2, rows, lo, hi, flag);
    return select_flagged(ar, flag, rows, list, count, s);
}

cudaError_t length_quantile2(Arena &ar, const int32_t *p1, const int32_t *p2, int64_t rows, double q, int *len_q,
                             cudaStream_t s) {
    unsigned long long *d_h = ar.alloc_tmp<unsigned long long>(33);
    if (!d_h) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(d_h, 0, 33 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_len_hist<<<g1d(rows), 256, 0, s>>>(p1, p2, rows, d_h);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned long long h[33];
    if ((e = cudaMemcpyAsync(h, d_h, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    const double want = q * (double)rows;
    double acc = 0.0;
    *len_q = 1;
    for (int b = 0; b < 33; ++b) {
        acc += (double)h[b];
        if (acc >= want) { *len_q = b == 0 ? 1 : (b >= 31 ? INT32_MAX : (1 << b)); break; }
    }
    return cudaSuccess;
}

cudaError_t heavy_list2(Arena &ar, const int32_t *p1, int thr1, const int32_t *p2, int thr2, int64_t rows,
                        int32_t **list, int32_t *count, cudaStream_t s) {
    char *flag = ar.alloc_tmp<char>(rows > 0 ? rows : 1);
    if (!flag) return cudaErrorMemoryAllocation;
    k_heavy_flags2<<<g1d(rows), 256, 0, s>>>(p1, thr1, p2, thr2, rows, flag);
    return select_flagged(ar, flag, rows, list, count, s);
}

// ------------------------------------------------------------ search brackets
// Per-variable column statistics of one side's matrix: min and max of A_ji
// over its nonzeros (A_ji = val / rdiv_j).
__global__ void k_colstats(ColView cv, int64_t n, const float *c, double *part) {
    __shared__ double sh[3][256];
    double s_min = 0.0, s_max = 0.0, deg_max = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double mn = INFINITY, mx = 0.0;
        auto put = [&](double a) { mn = fmin(mn, a); mx = fmax(mx, a); };
        switch (cv.kind) {
        case CK_CSR:
            if (!cv.val && !cv.rdiv) {   // unit entries: one value, no division per entry
                if (cv.ptr[i + 1] > cv.ptr[i]) put(1.0);
                break;
            }
            for (int k = cv.ptr[i]; k < cv.ptr[i + 1]; ++k)
                put((cv.val ? (double)cv.val[k] : 1.0) / (cv.rdiv ? (double)cv.rdiv[cv.idx[k]] : 1.0));
            break;
        case CK_FIXED2: {
            int2 e = reinterpret_cast<const int2 *>(cv.idx)[i];
            put(cv.rdiv ? 1.0 / (double)cv.rdiv[e.x] : 1.0);
            put(cv.rdiv ? 1.0 / (double)cv.rdiv[e.y] : 1.0);
            break;
        }
        case CK_FIXED1: put(cv.rdiv ? 1.0 / (double)cv.rdiv[cv.idx[i]] : 1.0); break;
        case CK_HALF1: put(cv.rdiv ? 1.0 / (double)cv.rdiv[i >> 1] : 1.0); break;
        case CK_SPLIT2:   // entries all 1 (no row bounds); empty for an isolated vertex
            if (cv.ptr[i + 1] > cv.ptr[i]) put(1.0);
            break;
        default: put(1.0);
        }
        double ci = c ? (double)c[i] : 1.0;
        if (mx > 0.0) {
            s_min += ci / mn;   // sum_i c_i max_j 1/a_ji
            s_max += ci / mx;   // sum_i c_i / max_j a_ji
        }
        if (cv.kind == CK_CSR || cv.kind == CK_SPLIT2) deg_max = fmax(deg_max, (double)(cv.ptr[i + 1] - cv.ptr[i]));
    }
    sh[0][threadIdx.x] = s_min;
    sh[1][threadIdx.x] = s_max;
    sh[2][threadIdx.x] = deg_max;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, d = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) { a += sh[0][t]; b += sh[1][t]; d = fmax(d, sh[2][t]); }
        part[blockIdx.x * 3 + 0] = a;
        part[blockIdx.x * 3 + 1] = b;
        part[blockIdx.x * 3 + 2] = d;
    }
}

// Per covering row j: min over its nonzeros of c_i / a_ji; reduce the max over rows.
__global__ void k_rowratio(RowView rv, int64_t rows, const float *c, double *part) {
    __shared__ double sh[256];
    double best = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows; j += (int64_t)gridDim.x * blockDim.x) {
        double coef = rv.rdiv ? 1.0 / (double)rv.rdiv[j] : 1.0;
        double mn = INFINITY;
        switch (rv.kind) {
        case RK_CSR:
            if (!rv.val) {
                // every entry of the row is coef: a correctly rounded division by a
                // positive constant is monotone, so min_k (c_k / coef) is
                // (min_k c_k) / coef exactly, with one FP64 division per row
                // (the minimum itself in FP32: float -> double is exact and monotone)
                if (coef > 0.0 && rv.ptr[j + 1] > rv.ptr[j]) {
                    float cm = INFINITY;
                    if (c) {
                        for (int k = rv.ptr[j]; k < rv.ptr[j + 1]; ++k) cm = fminf(cm, c[rv.idx[k]]);
                    } else {
                        cm = 1.0f;
                    }
                    mn = (double)cm / coef;
                }
                break;
            }
            for (int k = rv.ptr[j]; k < rv.ptr[j + 1]; ++k) {
                double a = (rv.val ? (double)rv.val[k] : 1.0) * coef;
                if (a > 0.0) mn = fmin(mn, (c ? (double)c[rv.idx[k]] : 1.0) / a);
            }
            break;
        case RK_FIXED2: {
            int2 e = reinterpret_cast<const int2 *>(rv.idx)[j];
            mn = fmin((c ? (double)c[e.x] : 1.0), (c ? (double)c[e.y] : 1.0)) / coef;
            break;
        }
        case RK_PAIRSUM:
            mn = fmin((c ? (double)c[2 * j] : 1.0), (c ? (double)c[2 * j + 1] : 1.0)) / coef;
            break;
        default: break;
        }
        if (mn < INFINITY) best = fmax(best, mn);
    }
    sh[threadIdx.x] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) a = fmax(a, sh[t]);
        part[blockIdx.x] = a;
    }
}

cudaError_t bracket_stats(Arena &ar, const ColView &cv, int64_t n, const float *c, double *sum_inv_min,
                          double *sum_inv_max, double *deg_max, cudaStream_t s) {
    int g = 512;
    double *part = (double *)ar.scratch_keep(sizeof(double) * 3 * g);
    if (!part) return cudaErrorMemoryAllocation;
    k_colstats<<<g, 256, 0, s>>>(cv, n, c, part);
    std::vector<double> h(3 * g);
    cudaError_t e = cudaMemcpyAsync(h.data(), part, sizeof(double) * 3 * g, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double a = 0, b = 0, d = 0;
    for (int i = 0; i < g; ++i) { a += h[3 * i]; b += h[3 * i + 1]; d = fmax(d, h[3 * i + 2]); }
    *sum_inv_min = a;
    *sum_inv_max = b;
    *deg_max = d;
    return cudaSuccess;
}

cudaError_t bracket_rowratio(Arena &ar, const RowView &rv, int64_t rows, const float *c, double *out,
                             cudaStream_t s) {
    int g = 512;
    double *part = (double *)ar.scratch_keep(sizeof(double) * g);
    if (!part) return cudaErrorMemoryAllocation;
    k_rowratio<<<g, 256, 0, s>>>(rv, rows, c, part);
    std::vector<double> h(g);
    cudaError_t e = cudaMemcpyAsync(h.data(), part, sizeof(double) * g, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    double a = 0;
    for (int i = 0; i < g; ++i) a = fmax(a, h[i]);
    *out = a;
    return cudaSuccess;
}

}  // namespace mwu
