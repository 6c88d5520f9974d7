// Setup helpers: a device-allocation arena owned by a context, input
// validation and construction of the row/column views (see mwu_setup.cu).
#pragma once

#include "mwu_internal.cuh"

#include <cstdlib>
#include <vector>

namespace mwu {

// Owns the device buffers of one context.  alloc() buffers live until the
// context is destroyed; alloc_tmp()/scratch() buffers until release_tmp().
class Arena {
public:
    // MWU_FAULT_ALLOC_AT=k in the environment makes the k-th allocation of each
    // arena fail (a host-side fault injection for the out-of-memory paths)
    explicit Arena(cudaStream_t s = nullptr) : stream_(s) {
        if (const char *f = std::getenv("MWU_FAULT_ALLOC_AT")) fail_at_ = std::atol(f);
    }
    ~Arena() { free_all(); }
    Arena(const Arena &) = delete;
    Arena &operator=(const Arena &) = delete;

    void set_stream(cudaStream_t s) { stream_ = s; }
    size_t bytes() const { return bytes_; }
    bool failed() const { return failed_; }

    void *raw(size_t nbytes) {
        void *p = nullptr;
        if (nbytes == 0) nbytes = 16;
        if (injected_failure() || cudaMalloc(&p, nbytes) != cudaSuccess) { failed_ = true; cudaGetLastError(); return nullptr; }
        keep_.push_back(p);
        bytes_ += nbytes;
        return p;
    }
    template <class T> T *alloc(int64_t n) { return (T *)raw(sizeof(T) * (size_t)(n > 0 ? n : 1)); }

    void *raw_tmp(size_t nbytes) {
        void *p = nullptr;
        if (nbytes == 0) nbytes = 16;
        if (injected_failure() || cudaMalloc(&p, nbytes) != cudaSuccess) { failed_ = true; cudaGetLastError(); return nullptr; }
        tmp_.push_back(p);
        return p;
    }
    template <class T> T *alloc_tmp(int64_t n) { return (T *)raw_tmp(sizeof(T) * (size_t)(n > 0 ? n : 1)); }
    void *scratch(size_t nbytes) { return raw_tmp(nbytes); }
    void *scratch_keep(size_t nbytes) { return raw_tmp(nbytes); }

    void release_tmp() {
        if (tmp_.empty()) return;
        cudaStreamSynchronize(stream_);
        for (void *p : tmp_) cudaFree(p);
        tmp_.clear();
    }
    void free_all() {
        release_tmp();
        for (void *p : keep_) cudaFree(p);
        keep_.clear();
        bytes_ = 0;
    }

private:
    bool injected_failure() { return fail_at_ > 0 && ++count_ == fail_at_; }
    long fail_at_ = 0, count_ = 0;
    cudaStream_t stream_;
    std::vector<void *> keep_, tmp_;
    size_t bytes_ = 0;
    bool failed_ = false;
};

const char *validation_message(int code);
cudaError_t validate_csr(const int32_t *ptr, const int32_t *idx, const float *val, int64_t rows, int64_t cols,
                         int64_t nnz, int require_nonempty, int *d_err, cudaStream_t s);
cudaError_t validate_edges(const int32_t *e, int64_t m, int32_t nv, int *d_err, cudaStream_t s);
cudaError_t validate_positive(const float *v, int64_t n, int code, int *d_err, cudaStream_t s);
cudaError_t validate_nonneg(const float *v, int64_t n, int code, int *d_err, cudaStream_t s);

cudaError_t build_vertex_slots(Arena &ar, const int32_t *edges, int64_t m, int32_t nv, int32_t **ptr_out,
                               int32_t **slots_out, cudaStream_t s);
// Split column view of an incidence transpose M^T (rows = edges (u_e, v_e),
// sorted by first endpoint u_e): per vertex i, the edges whose first endpoint
// is i form the contiguous range [cptr[i] - vptr[i], cptr[i+1] - vptr[i+1]),
// and the edges whose second endpoint is i are listed, by increasing edge id,
// through their first endpoints u2[vptr[i] .. vptr[i+1]).  cptr = uptr + vptr
// (the combined column lengths).  *sorted = 0 (nothing built) when the edge
// list is not sorted by first endpoint.
cudaError_t build_split_view(Arena &ar, const int32_t *edges, int64_t m, int32_t nv, int32_t **cptr,
                             int32_t **vptr, int32_t **u2, int *sorted, cudaStream_t s);
cudaError_t slots_to_edges(Arena &ar, const int32_t *slots, int64_t ns, int32_t **out, cudaStream_t s);
cudaError_t csr_transpose(Arena &ar, const int32_t *ptr, const int32_t *idx, const float *val, int64_t rows,
                          int64_t cols, int64_t nnz, int32_t **tptr, int32_t **tidx, float **tval, cudaStream_t s);
cudaError_t heavy_list(Arena &ar, const int32_t *ptr, int64_t rows, int thr, int32_t **list, int32_t *count,
                       cudaStream_t s);
// rows j with lo < len(j) <= hi, in increasing order
cudaError_t bin_list(Arena &ar, const int32_t *ptr, int64_t rows, int lo, int hi, int32_t **list, int32_t *count,
                     cudaStream_t s);
cudaError_t heavy_list2(Arena &ar, const int32_t *p1, int thr1, const int32_t *p2, int thr2, int64_t rows,
                        int32_t **list, int32_t *count, cudaStream_t s);
// rows whose longer column (of the views p1, p2; either may be NULL) has a
// length in (lo, hi], in increasing order
cudaError_t range_list2(Arena &ar, const int32_t *p1, const int32_t *p2, int64_t rows, int lo, int hi,
                        int32_t **list, int32_t *count, cudaStream_t s);
// *len_q = the power-of-two upper end of the bucket holding quantile q of the
// longer column lengths
cudaError_t length_quantile2(Arena &ar, const int32_t *p1, const int32_t *p2, int64_t rows, double q, int *len_q,
                             cudaStream_t s);
// Tile plan of a CSR row view for the staged SpMV: tiles of tile_rows
// consecutive rows; per tile the first column and the column span of its
// entries (0 for an empty tile).  *fit = tiles whose span is at most wmax,
// *fit_nnz = the entries of those tiles.
cudaError_t build_tiles(Arena &ar, const int32_t *ptr, const int32_t *idx, int64_t rows, int tile_rows, int wmax,
                        int32_t **lo, int32_t **len, int32_t *n_tiles, int32_t *fit, int64_t *fit_nnz,
                        cudaStream_t s);
cudaError_t bracket_stats(Arena &ar, const ColView &cv, int64_t n, const float *c, double *sum_inv_min,
                          double *sum_inv_max, double *deg_max, cudaStream_t s);
cudaError_t bracket_rowratio(Arena &ar, const RowView &rv, int64_t rows, const float *c, double *out,
                             cudaStream_t s);

}  // namespace mwu
