// sgtv_util.cu -- set-up kernels (value conversion, input validation) and the
// fixed-order finaliser of the FP64 reductions.
#include <cuda_bf16.h>
#include <math.h>

#include "sgtv_internal.h"

namespace sgtv {

namespace {

constexpr int kT = 256;

int blocks_for(int64_t n, int cap = 8192)
{
    int64_t b = (n + kT - 1) / kT;
    if (b < 1) b = 1;
    return int(b < cap ? b : cap);
}

__global__ void k_to_bf16(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst, int64_t n)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        dst[k] = __float2bfloat16_rn(src[k]);
}

__global__ void k_to_f64(const float *__restrict__ src, double *__restrict__ dst, int64_t n)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        dst[k] = double(src[k]);
}

__global__ void k_check_idx(const int32_t *__restrict__ idx, int64_t n, int64_t bound, int *flag)
{
    bool bad = false;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int32_t v = idx[k];
        bad |= (v < 0) || (int64_t(v) >= bound);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void k_check_vals(const float *__restrict__ val, int64_t n, int *flag)
{
    bool bad = false;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float v = val[k];
        bad |= !(v >= 0.0f) || !isfinite(v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 2);
}

// Strictly ascending indices inside every segment [ptr[s], ptr[s+1]).
__global__ void k_check_sorted(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                               int64_t nseg, int *flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    bool bad = false;
    for (int64_t s = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < nseg; s += nwarps) {
        const int64_t a = ptr[s], b = ptr[s + 1];
        for (int64_t p = a + lane; p + 1 < b; p += 32) bad |= !(idx[p] < idx[p + 1]);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 8);
}

// Every CSR nonzero (i, j, v) must be found in CSC column j with row i and
// value v (binary search; CSC rows are strictly ascending after k_check_sorted).
// With equal nnz and no duplicates on either side this makes the copies equal.
__global__ void k_check_match(int64_t I, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const float *__restrict__ rval, const int64_t *__restrict__ colptr,
                              const int32_t *__restrict__ row, const float *__restrict__ cval, int *flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    bool bad = false;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < I; i += nwarps) {
        for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
            const int32_t j = col[p];
            int64_t lo = colptr[j], hi = colptr[j + 1];
            while (lo < hi) {
                const int64_t mid = lo + ((hi - lo) >> 1);
                if (row[mid] < i) lo = mid + 1; else hi = mid;
            }
            bad |= !(lo < colptr[j + 1] && row[lo] == i && cval[lo] == rval[p]);
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 4);
}

template <typename I>
__global__ void k_add_offset(I *__restrict__ a, int64_t n, I off)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        a[k] += off;
}

__device__ __forceinline__ double red_warp(double v, bool mx)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, v, o);
        v = mx ? fmax(v, t) : v + t;
    }
    return v;
}

// One block; thread t folds partials t, t+256, ... in order, then a fixed tree.
__global__ void k_finalize(const double *__restrict__ part, int nblocks, int nfields, unsigned max_mask,
                           double *__restrict__ out)
{
    __shared__ double sh[32];
    for (int fld = 0; fld < nfields; fld++) {
        const bool mx = (max_mask >> fld) & 1u;
        double v = mx ? -INFINITY : 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double t = part[size_t(fld) * nblocks + b];
            v = mx ? fmax(v, t) : v + t;
        }
        v = red_warp(v, mx);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) sh[w] = v;
        __syncthreads();
        if (w == 0) {
            v = (lane < int(blockDim.x >> 5)) ? sh[lane] : (mx ? -INFINITY : 0.0);
            v = red_warp(v, mx);
            if (lane == 0) out[fld] = v;
        }
    }
}

}  // namespace

void convert_values_bf16(const float *src, void *dst, int64_t n, cudaStream_t st)
{
    k_to_bf16<<<blocks_for(n), kT, 0, st>>>(src, static_cast<__nv_bfloat16 *>(dst), n);
}

void convert_values_f64(const float *src, void *dst, int64_t n, cudaStream_t st)
{
    k_to_f64<<<blocks_for(n), kT, 0, st>>>(src, static_cast<double *>(dst), n);
}

void convert_vec_f64(const float *src, void *dst, int64_t n, cudaStream_t st)
{
    k_to_f64<<<blocks_for(n), kT, 0, st>>>(src, static_cast<double *>(dst), n);
}

void validate_indices(const int32_t *idx, int64_t n, int64_t bound, int *flag, cudaStream_t st)
{
    if (n > 0) k_check_idx<<<blocks_for(n), kT, 0, st>>>(idx, n, bound, flag);
}

void validate_values(const float *val, int64_t n, int *flag, cudaStream_t st)
{
    if (n > 0) k_check_vals<<<blocks_for(n), kT, 0, st>>>(val, n, flag);
}

void validate_sorted(const int64_t *ptr, const int32_t *idx, int64_t nseg, int *flag, int sm_count,
                     cudaStream_t st)
{
    if (nseg > 0) k_check_sorted<<<blocks_for(nseg * 32, sm_count * 8), kT, 0, st>>>(ptr, idx, nseg, flag);
}

void validate_match(int64_t I, const int64_t *rowptr, const int32_t *col, const float *rval,
                    const int64_t *colptr, const int32_t *row, const float *cval, int *flag,
                    int sm_count, cudaStream_t st)
{
    if (I > 0)
        k_check_match<<<blocks_for(I * 32, sm_count * 8), kT, 0, st>>>(I, rowptr, col, rval, colptr, row,
                                                                       cval, flag);
}

void add_offset_i32(int32_t *a, int64_t n, int32_t off, cudaStream_t st)
{
    if (n > 0) k_add_offset<int32_t><<<blocks_for(n), kT, 0, st>>>(a, n, off);
}

void add_offset_i64(int64_t *a, int64_t n, int64_t off, cudaStream_t st)
{
    if (n > 0) k_add_offset<int64_t><<<blocks_for(n), kT, 0, st>>>(a, n, off);
}

void finalize(const double *part, int nblocks, int nfields, unsigned max_mask, double *out, cudaStream_t st)
{
    k_finalize<<<1, kT, 0, st>>>(part, nblocks, nfields, max_mask, out);
}

}  // namespace sgtv
