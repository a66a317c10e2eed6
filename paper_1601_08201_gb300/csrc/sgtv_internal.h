// sgtv_internal.h -- types shared by the host code and the kernel translation
// units of libsgtv.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sgtv {

// One scan of a batch. A handle holds one or more independent scans stored
// back to back: their hyper-voxels, spatial sites and measurements are
// concatenated in scan order (a block-diagonal system matrix).
struct Scan {
    int64_t vox0, site0;        // first hyper-voxel and first spatial site
    int32_t Nx, Nz, Nq, pad_;
    double rho, tau, beta;      // ADMM penalty, shrink threshold beta / rho, regularisation weight
    float rhof, tauf;           // rho and tau rounded to FP32 once (the FP32 kernels' operands)
};

// The group-TV stencil (Eq. 2): direction p moves (dx[p], dz[p]) in (x, z)
// with weight w[p]; plus the per-scan geometry (device tables).
struct Geom {
    int32_t n_dirs, nscans;
    int64_t J, S;               // totals over the scans
    int32_t dx[4], dz[4];
    double w[4];
    float wf[4];                // w rounded to FP32 once (the FP32 kernels' operands)
    const Scan *scans;          // [nscans]
    const int64_t *vox_off;     // [nscans + 1] first hyper-voxel of each scan, then J
    const int64_t *site_off;    // [nscans + 1] first site of each scan, then S
    int32_t max_nq;             // largest Nq of the scans
    int32_t per_bin;            // 0: group TV (one group per site, Eq. 2); 1: standard
                                // isotropic TV (one group per site and q-bin)
};

// Tiled local-index form of one compressed matrix (see sgtv_tli.cu):
// tiles of kTliTile consecutive segments, 16-bit local indices into a staging
// buffer that is, per tile, either its aligned index window (wlen[t] > 0) or
// its unique index list (wlen[t] == 0). fmt: 0 = not built (plain kernels
// only), 1 = built, every tile a list; 2 = built, every tile a window;
// 3 = built, mixed.
constexpr int kTliTile = 64;
struct TliMat {
    int fmt;
    int max_stage;        // elements of the largest staging buffer
    int64_t ntiles;
    uint16_t *lidx;       // [nnz]
    int64_t *uoff;        // [ntiles + 1]; window tiles hold no list entries
    int32_t *uidx;        // [uoff[ntiles]]
    int32_t *wbase;       // [ntiles]
    int32_t *wlen;        // [ntiles]; 0 = list tile
    // one stage of the TMA-streamed pipeline (byte offsets, 128-aligned);
    // tma_stage_bytes = 0 when the form is not built
    int tma_stage_bytes, tma_off_lidx, tma_off_val, tma_off_uidx, tma_off_xs;
    int smem_optin;       // the device's opt-in shared memory per block (bytes)
};

// Single-pass row stream (built for SGTV_FLAG_SINGLE_PASS only; see
// sgtv_sp.cu): the tiled CSR form's local indices and A's values again, each
// row padded to a multiple of 4 elements and its elements dealt out to the
// warp's access instructions by shared-memory bank.
struct SpStream {
    int64_t *rp;          // [I + 1] row starts, multiples of 4 (host copy in the handle)
    uint16_t *lidx;       // [rp[I]] local indices; padding slots hold the tile's staging size
    void *val;            // [rp[I]] values of type V; padding slots hold 0
    int built;
};

// Device pointers of one problem; vector element type depends on the precision
// (float, or double in the FP64 mode), A's value type on the precision too.
struct Dev {
    int64_t I, J, nnz;
    const int64_t *rowptr, *colptr;  // padded to ntiles * kTliTile + 2 entries (tail = nnz)
    const int32_t *col, *row;
    const void *rval, *cval;  // CSR / CSC values
    const void *y, *r;
    int r_scalar;
    void *s;                  // A^T 1
    void *f, *f_next;         // image, double-buffered
    void *ratio;              // y / (A f + r)
    void *e;                  // A^T ratio (KKT only)
    void *d, *c;              // split and dual variables, [n_dirs][J]
    void *d_prev;             // d before the last shrink, [n_dirs][J]; the next shrink
                              // writes there and the two buffers swap
    void *u;                  // u = d - c, [n_dirs][J], kept by the shrink for the
                              // single-pass f-update (NULL in the other forms)
    double *part;             // reduction partials, >= 4 * red_blocks doubles
    double *red;              // reduced results (device), >= 8 doubles
    int *flag;                // bit 0: non-finite iterate, bit 1: a bounded wait gave up
    TliMat tr, tc;            // tiled local-index forms of the CSR and CSC copies
    SpStream sp;              // single-pass row stream (sp.built = 0 unless requested)
    int sm_count;
    int smem_optin;           // opt-in shared memory per block (bytes)
    int red_blocks;           // grid of the reduction kernels
};

typedef void (*ForwardFn)(const Dev &, const void *f, void *ratio, cudaStream_t);
// State of the persistent kernel's grid-wide barrier (count and gen zeroed
// at set-up) and how long a block waits in it before it gives up.
struct GridBar {
    unsigned int count, gen;
    unsigned long long limit_ns;
};
// One cooperative launch of a whole iteration; returns the launch status.
typedef cudaError_t (*PersistentFn)(const Dev &, const Geom &, const void *f, void *f_new, int do_shrink,
                                    GridBar *bar, cudaStream_t);
typedef void (*BackUpdateFn)(const Dev &, const Geom &, const void *f, void *f_new, cudaStream_t);
constexpr int kMaxVariants = 32;

// One precision's launchers (T = vector type, V = value type of A). The two
// sparse products come in several tilings (segments per warp, prefetch depth,
// pipelining, register cap, 4-wide loads); variants of one element order give
// bit-identical results (the 4-wide forms round differently, equally
// deterministic), the autotuner only picks the fastest for the problem at hand.
struct KernelSet {
    int n_fwd;
    ForwardFn fwd[kMaxVariants];
    const char *fwd_name[kMaxVariants];
    int fwd_need[kMaxVariants];     // 0 plain; 1 tiled (Dev::tr); NS >= 3: TMA pipeline of NS stages
    int n_back;
    BackUpdateFn back[kMaxVariants];
    const char *back_name[kMaxVariants];
    int back_need[kMaxVariants];    // same, for Dev::tc
    // v = w.G f + c, d_out = group shrink of v (Eq. 6), c = v - d_out (Eq. 7),
    // and, when Dev::u is not NULL, u = d_out - c (the f-update's operand)
    void (*shrink)(const Dev &, const Geom &, const void *f, void *d_out, cudaStream_t);
    void (*sub)(int64_t n, const void *a, const void *b, void *out, cudaStream_t);  // out = a - b
    // single-pass form (needs Dev::tr): scatter e += A^T (y / (A f + r)) row by
    // row into e (zeroed beforehand), then the f-update from e (which it clears)
    int n_scatter;
    void (*scatter[kMaxVariants])(const Dev &, const void *f, void *e, cudaStream_t);
    const char *scatter_name[kMaxVariants];
    int scatter_bufs[kMaxVariants];  // staging-sized shared-memory buffers the variant needs (with the f stage)
    int scatter_sp[kMaxVariants];    // 1: reads the single-pass row stream (Dev::sp)
    void (*fupdate)(const Dev &, const Geom &, void *e, const void *f, void *f_new, cudaStream_t);
    int n_pers;                      // persistent one-launch iterations (need Dev::tr and Dev::tc)
    PersistentFn pers[8];
    const char *pers_name[8];
    void (*backproject)(const Dev &, const void *v, void *out, cudaStream_t);
    void (*colsum)(const Dev &, cudaStream_t);
    void (*wgrad)(const Dev &, const Geom &, const void *f, void *out, cudaStream_t);
    // c = theta * tau * d_s / |d_s| per group (0 where d_s = 0), from Dev::d
    void (*dual_rule)(const Dev &, const Geom &, double theta, cudaStream_t);
    void (*fill)(int64_t n, void *a, double val, cudaStream_t);
    void (*ratio_out)(int64_t n, const void *num, const void *den, float *out, cudaStream_t);
    void (*load_image)(int64_t n, const float *src, void *f, int *flag, cudaStream_t);
    void (*load_vec)(int64_t n, const float *src, void *a, int *flag, cudaStream_t);  // no clamp
    // FP64 reductions: results land in d.red[...] (device)
    void (*sum)(const Dev &, int64_t n, const void *a, int slot, cudaStream_t);
    // deviance over measurements [i0, i1); tv over sites [s0, s1)
    void (*deviance)(const Dev &, const void *f, int64_t i0, int64_t i1, int slot, cudaStream_t);
    void (*tv)(const Dev &, const Geom &, const void *f, const void *dsplit, int64_t s0, int64_t s1, int slot,
               cudaStream_t);
    void (*kkt)(const Dev &, const Geom &, const void *f, int slot, cudaStream_t);
    // red[slot] = ||rho (w.G)^T (d - d_prev)||^2, red[slot + 1] = ||rho (w.G)^T c||^2
    void (*dual_res)(const Dev &, const Geom &, int slot, cudaStream_t);
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

// Tiled local-index set-up (sgtv_tli.cu). Indices must be strictly ascending
// inside each segment. tile_range: per tile min / max index (empty tile:
// min = INT32_MAX, max = -1). window_lidx: lidx = idx - wbase[tile].
// list_count / list_build: per tile unique indices through a shared-memory
// bitmap of max_words 32-bit words, swept over [tmin, tmax] in chunks.
void tli_tile_range(const int64_t *ptr, const int32_t *idx, int64_t nseg, int64_t ntiles, int32_t *tmin,
                    int32_t *tmax, cudaStream_t st);
void tli_window_lidx(const int64_t *ptr, const int32_t *idx, int64_t nseg, const int32_t *wbase,
                     const int32_t *wlen, uint16_t *lidx, int sm_count, cudaStream_t st);
int tli_list_max_words();
void tli_check(const int64_t *ptr, int64_t nseg, const uint16_t *lidx, const int32_t *wlen, const int64_t *uoff,
               const int32_t *uidx, int64_t n_dense, int *flag, int sm_count, cudaStream_t st);
cudaError_t tli_list_count(const int64_t *ptr, const int32_t *idx, int64_t nseg, int64_t ntiles,
                           const int32_t *tmin, const int32_t *tmax, int max_words, int32_t *ucnt,
                           cudaStream_t st);
cudaError_t tli_list_build(const int64_t *ptr, const int32_t *idx, int64_t nseg, int64_t ntiles,
                           const int32_t *tmin, const int32_t *tmax, const int32_t *wlen, int max_words,
                           const int64_t *uoff, int32_t *uidx, uint16_t *lidx, cudaStream_t st);

// Single-pass row stream (sgtv_sp.cu) from the tiled CSR form: sp_rp (device,
// [I + 1], row starts padded to multiples of 4) given; writes sp_lidx, sp_val
// and checks the result (flag bit 32 if a row is not a padded permutation).
cudaError_t sp_build(int64_t I, const int64_t *rowptr, const uint16_t *lidx, const void *val, int val_bytes,
                     const int64_t *sp_rp, const int32_t *wlen, const int64_t *uoff, uint16_t *sp_lidx, void *sp_val,
                     int *flag, int sm_count, cudaStream_t st);

// a[k] += off for k < n (offsetting one scan's indices inside a batch).
void add_offset_i32(int32_t *a, int64_t n, int32_t off, cudaStream_t st);
void add_offset_i64(int64_t *a, int64_t n, int64_t off, cudaStream_t st);

// Reduce the field-major partials of `nfields` fields (nblocks each) in a fixed
// order; field k is a max if bit k of max_mask is set, else a sum.
void finalize(const double *part, int nblocks, int nfields, unsigned max_mask, double *out,
              cudaStream_t st);

}  // namespace sgtv
