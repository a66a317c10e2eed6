// sgtv_internal.h -- types shared by the host code and the kernel translation
// units of libsgtv.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sgtv {

// Image geometry and the neighbour stencil of the group-TV operator (Eq. 2):
// direction p moves (dx[p], dz[p]) in (x, z); w[p] is its weight.
struct Geom {
    int32_t Nx, Nz, Nq, n_dirs;
    int64_t J;
    int32_t dx[4], dz[4];
    double w[4];
};

// Device pointers of one problem; vector element type depends on the precision
// (float, or double in the FP64 mode), A's value type on the precision too.
struct Dev {
    int64_t I, J, nnz;
    const int64_t *rowptr, *colptr;
    const int32_t *col, *row;
    const void *rval, *cval;  // CSR / CSC values
    const void *y, *r;
    int r_scalar;
    void *s;                  // A^T 1
    void *f, *f_next;         // image, double-buffered
    void *ratio;              // y / (A f + r)
    void *e;                  // A^T ratio (KKT only)
    void *d, *c;              // split and dual variables, [n_dirs][J]
    double *part;             // reduction partials, >= 4 * red_blocks doubles
    double *red;              // reduced results (device), >= 8 doubles
    int *flag;                // non-finite flag
    int sm_count;
    int red_blocks;           // grid of the reduction kernels
};

typedef void (*ForwardFn)(const Dev &, const void *f, void *ratio, cudaStream_t);
typedef void (*BackUpdateFn)(const Dev &, const Geom &, const void *f, void *f_new, double rho,
                             cudaStream_t);
constexpr int kMaxVariants = 8;

// One precision's launchers (T = vector type, V = value type of A). The two
// sparse products come in several tilings (segments per warp, prefetch depth,
// pipelining, register cap); every variant gives bit-identical results, the
// autotuner only picks the fastest for the problem at hand.
struct KernelSet {
    int n_fwd;
    ForwardFn fwd[kMaxVariants];
    const char *fwd_name[kMaxVariants];
    int n_back;
    BackUpdateFn back[kMaxVariants];
    const char *back_name[kMaxVariants];
    void (*shrink)(const Dev &, const Geom &, const void *f, double tau, cudaStream_t);
    void (*backproject)(const Dev &, const void *v, void *out, cudaStream_t);
    void (*colsum)(const Dev &, cudaStream_t);
    void (*wgrad)(const Dev &, const Geom &, const void *f, void *out, cudaStream_t);
    void (*fill)(int64_t n, void *a, double val, cudaStream_t);
    // FP64 reductions: results land in d.red[...] (device)
    void (*sum)(const Dev &, int64_t n, const void *a, int slot, cudaStream_t);
    void (*deviance)(const Dev &, const void *f, int slot, cudaStream_t);
    void (*tv)(const Dev &, const Geom &, const void *f, const void *dsplit, int slot, cudaStream_t);
    void (*kkt)(const Dev &, const Geom &, const void *f, double rho, int slot, cudaStream_t);
    int elem_size;   // bytes of T
    int val_size;    // bytes of V
};

extern const KernelSet kset_f32;
extern const KernelSet kset_bf16;
extern const KernelSet kset_f64;

// Values converted on the device after upload (float -> V).
void convert_values_bf16(const float *src, void *dst, int64_t n, cudaStream_t st);
void convert_values_f64(const float *src, void *dst, int64_t n, cudaStream_t st);
void convert_vec_f64(const float *src, void *dst, int64_t n, cudaStream_t st);

// Validation of uploaded CSR/CSC data; sets bits in *flag (device):
//   1 = index out of range, 2 = negative or non-finite value,
//   8 = indices not strictly ascending inside a row or column,
//   4 = a CSR nonzero is missing from the CSC copy (or has another value).
void validate_indices(const int32_t *idx, int64_t n, int64_t bound, int *flag, cudaStream_t st);
void validate_values(const float *val, int64_t n, int *flag, cudaStream_t st);
void validate_sorted(const int64_t *ptr, const int32_t *idx, int64_t nseg, int *flag, int sm_count,
                     cudaStream_t st);
void validate_match(int64_t I, const int64_t *rowptr, const int32_t *col, const float *rval,
                    const int64_t *colptr, const int32_t *row, const float *cval, int *flag,
                    int sm_count, cudaStream_t st);

// Reduce the field-major partials of `nfields` fields (nblocks each) in a fixed
// order; field k is a max if bit k of max_mask is set, else a sum.
void finalize(const double *part, int nblocks, int nfields, unsigned max_mask, double *out,
              cudaStream_t st);

}  // namespace sgtv
