/*
 * sgtv.h -- C ABI of the GB300 (sm_103a) spectrally grouped TV reconstruction
 * library (libsgtv.so).
 *
 * Method: Odinaka et al., "Spectrally Grouped Total Variation Reconstruction
 * for Scatter Imaging Using ADMM" (IEEE NSS/MIC 2015).
 *   Measurement model (Sec. II, Eq. 1): y_i ~ Poisson((A f)_i + r_i), A >= 0,
 *   I measurements, J = S * Q hyper-voxels (S spatial bins, Q q-bins).
 *   Regulariser (Sec. II, Eq. 2): group TV, one L2 norm per spatial bin over
 *   all q-bins and all neighbour directions.
 *   Solver (Sec. III, Eqs. 4-7): ADMM / split Bregman on d_p = w_p . G_p f with
 *   the f-subproblem (Eq. 5) solved by one closed-form step of optimisation
 *   transfer (EM surrogate + De Pierro's convexity split), group soft-threshold
 *   for d (Eq. 6) and the scaled dual update for c (Eq. 7).
 *
 * Symbol map: the API's `lambda` is the paper's regularisation weight beta
 * (Eq. 4); the API's `rho` is the paper's ADMM penalty lambda (Eqs. 5-7).
 *
 * Layouts (all arrays dense, C order):
 *   hyper-voxel index j = (x * Nz + z) * Nq + q  (q fastest), J = Nx * Nz * Nq;
 *   directions: n_dirs = 4 -> p = 0:+x, 1:-x, 2:+z, 3:-z; n_dirs = 2 -> 0:+x, 1:+z;
 *   (G_p f)_j = f_j - f_{neighbour in direction p}, a neighbour outside the
 *   domain being a zero ghost (Dirichlet, Sec. III);
 *   d and c are direction-major: element (p, j) at p * J + j.
 *
 * Errors: every call returns SGTV_OK (0) or a negative SGTV_ERR_* code. An
 * error is sticky on its handle (later calls return SGTV_ERR_STATE) and its
 * text is available from sgtv_last_error. Calls on one handle are not
 * thread-safe; separate handles are independent.
 *
 * Execution: the handle owns its device memory (cudaMalloc, or the allocator
 * given in sgtv_opts) and issues its work on one CUDA stream (its own, or the
 * one given in sgtv_opts). Inside sgtv_iterate the group shrink and dual
 * update of each iteration (Eqs. 6-7), which only the next iteration's
 * f-update reads, run on a second stream the handle owns, overlapping the
 * next forward pass (unless SGTV_FLAG_SERIAL); it is joined back into the
 * handle's stream before that f-update and at the end of every call, so the
 * work of each call is ordered on the handle's stream. sgtv_iterate only enqueues work; the calls that
 * return data (sgtv_get_*, sgtv_objective, sgtv_residuals, sgtv_sync) wait for
 * the stream and report a non-finite value met by an earlier iteration.
 */
#ifndef SGTV_H
#define SGTV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgtv_ctx *sgtv_t;

enum {
    SGTV_OK = 0,
    SGTV_ERR_ARG = -1,       /* null pointer, bad size, J != Nx*Nz*Nq, bad option */
    SGTV_ERR_DOMAIN = -2,    /* negative / non-finite data, CSR and CSC disagree,
                                rho <= 0 or lambda < 0, ybar_i can be 0 with y_i > 0 */
    SGTV_ERR_CUDA = -3,      /* a CUDA runtime call failed */
    SGTV_ERR_OOM = -4,       /* device allocation failed */
    SGTV_ERR_STATE = -5,     /* wrong call order, or the handle holds an earlier error */
    SGTV_ERR_TIMEOUT = -6,   /* a bounded device-side wait (a tile's bulk copy, a grid barrier) gave up */
    SGTV_ERR_NONFINITE = -7  /* NaN or Inf appeared in the iterate */
};

enum { SGTV_PREC_FP32 = 0,    /* FP32 A values, vectors and accumulation */
       SGTV_PREC_BF16VAL = 1, /* A values rounded to BF16 (nearest even), FP32 rest */
       SGTV_PREC_FP64 = 2 };  /* FP64 everywhere (checking mode) */

enum { SGTV_FLAG_ALLOW_RHO0 = 1,    /* accept rho = 0: every iteration is one MLEM step */
       SGTV_FLAG_NO_AUTOTUNE = 2,   /* keep the default SpMV variants (no timing at set-up) */
       SGTV_FLAG_PERSISTENT = 4,    /* one cooperative launch per iteration (grid-wide barriers
                                       between its three phases; needs both tiled forms and
                                       n_inner = 1, else SGTV_ERR_ARG at set-up) */
       SGTV_FLAG_GRAPH = 8,         /* sgtv_iterate replays CUDA graphs of 8 captured iterations */
       SGTV_FLAG_SINGLE_PASS = 16, /* stream A once per surrogate step, by rows: each row's ratio is
                                       formed and its a_ij * ratio_i scattered into e at once, then an
                                       elementwise f-update. Same iteration; e's sums are formed in an
                                       order set by atomic adds, so results vary between runs at the
                                       rounding level. Needs the tiled row form with room for two
                                       staging buffers and no SGTV_FLAG_PERSISTENT, else SGTV_ERR_ARG
                                       at set-up. */
       SGTV_FLAG_STANDARD_TV = 32,  /* the standard isotropic TV of the paper's comparison instead
                                       of the group TV of Eq. 2: one group per (site, q-bin), the
                                       sum over q outside the square root; Eq. 6 shrinks each such
                                       group over the directions p, and the objective's R and the
                                       warm start's dual follow */
       SGTV_FLAG_SERIAL = 64 };     /* issue every kernel on the handle's stream, one after the other:
                                       no second stream for the shrink (for profiler captures and
                                       per-kernel timings that must not overlap) */

/* Kernel identifiers for sgtv_profile_read. */
enum { SGTV_K_FORWARD = 0,    /* ybar = A f + r, ratio = y / ybar (CSR) */
       SGTV_K_BACK_UPDATE = 1,/* e = A^T ratio (CSC) fused with the f-update */
       SGTV_K_SHRINK = 2,     /* v = w.G f + c, group shrink (d), dual update (c) */
       SGTV_K_ITERATION = 3,  /* a whole iteration: the persistent launch, or half a graph launch */
       SGTV_K_SCATTER = 4,    /* single-pass form: forward projection + ratio + scatter into e (CSR) */
       SGTV_K_FUPDATE = 5,    /* single-pass form: the f-update from e */
       SGTV_K_COUNT = 6 };

typedef void *(*sgtv_alloc_fn)(size_t bytes, void *user);
typedef void (*sgtv_free_fn)(void *ptr, void *user);

typedef struct {
    double w[4];          /* per-direction weights w_p (Eq. 2); default 1 */
    int32_t n_dirs;       /* 4 (default) or 2 */
    int32_t n_inner;      /* surrogate steps per ADMM iteration with u fixed; default 1 */
    int32_t precision;    /* SGTV_PREC_*; default FP32 */
    int32_t flags;        /* SGTV_FLAG_*; default 0 */
    void *stream;         /* cudaStream_t to issue work on; NULL = a stream the handle owns */
    sgtv_alloc_fn alloc;  /* device allocator; NULL = cudaMalloc */
    sgtv_free_fn free_;   /* paired with alloc */
    void *alloc_user;     /* passed to alloc / free_ */
} sgtv_opts;

/* Fill *o with the defaults listed above. */
void sgtv_default_opts(sgtv_opts *o);

/*
 * Create a handle for one reconstruction problem and initialise the ADMM state
 * (f0 = kappa everywhere, kappa = sum(y - r) / sum(A); d0 = w.G f0; c0 = 0).
 *
 * A is given twice, as CSR (rows = measurements, for the forward projection)
 * and as CSC (columns = hyper-voxels, for the backprojection); the two must
 * hold the same nonzeros. All pointers are HOST pointers; the library copies
 * them and the caller keeps ownership.
 *   I, J, nnz            : measurements, hyper-voxels, nonzeros (I, J < 2^31)
 *   csr_rowptr[I+1]      : int64, csr_rowptr[0] = 0, nondecreasing, [I] = nnz
 *   csr_col[nnz]         : int32 in [0, J)
 *   csr_val[nnz]         : float, >= 0 and finite
 *   csc_colptr[J+1], csc_row[nnz], csc_val[nnz] : the same matrix by columns
 *   Nx, Nz, Nq           : image shape, J = Nx * Nz * Nq
 *   y[I]                 : counts (float, >= 0)
 *   b[b_len]             : background r, b_len = 1 (scalar) or I, >= 0
 *   lambda               : regularisation weight beta >= 0 (Eq. 4)
 *   rho                  : ADMM penalty > 0 (Eqs. 5-7)
 *   opts                 : NULL for the defaults
 * On failure *out is set to NULL and no memory is kept.
 */
int sgtv_setup(sgtv_t *out, int64_t I, int64_t J, int64_t nnz,
               const int64_t *csr_rowptr, const int32_t *csr_col, const float *csr_val,
               const int64_t *csc_colptr, const int32_t *csc_row, const float *csc_val,
               int32_t Nx, int32_t Nz, int32_t Nq,
               const float *y, const float *b, int64_t b_len,
               double lambda, double rho, const sgtv_opts *opts);

/*
 * A batch of independent scans in one handle (the batched form). Each scan is
 * described exactly as in sgtv_setup (host pointers, copied; lambda = its
 * beta, rho = its ADMM penalty); all scans share the options (stencil,
 * weights, precision). The scans are concatenated: hyper-voxels, sites and
 * measurements back to back in scan order, so images, states, objectives and
 * residuals of the handle cover all scans (sgtv_batch_info gives the
 * offsets; sgtv_objective_scan one scan's objective). The total I and J must
 * stay below 2^31; the total nnz may exceed it. Each iteration runs the same
 * kernels as a one-scan handle over the block-diagonal system.
 */
typedef struct {
    int64_t I, J, nnz;
    const int64_t *csr_rowptr;
    const int32_t *csr_col;
    const float *csr_val;
    const int64_t *csc_colptr;
    const int32_t *csc_row;
    const float *csc_val;
    int32_t Nx, Nz, Nq;
    const float *y;
    const float *b;
    int64_t b_len;
    double lambda, rho;
} sgtv_scan;

int sgtv_setup_batch(sgtv_t *out, int32_t nscans, const sgtv_scan *scans, const sgtv_opts *opts);

/* Scan count and per-scan offsets (each array, if not NULL, holds nscans + 1
 * values; the last is the total): hyper-voxels, measurements, spatial sites. */
int sgtv_batch_info(sgtv_t h, int32_t *nscans, int64_t *vox_off, int64_t *meas_off, int64_t *site_off);

/* sgtv_objective restricted to scan k (0 <= k < nscans); SGTV_ERR_ARG (not
 * sticky) for k out of range. */
int sgtv_objective_scan(sgtv_t h, int32_t k, double *phi, double *dev, double *tv);

/* Enqueue n >= 0 ADMM iterations (Eqs. 5-7) on the handle's stream. Each
 * iteration launches three kernels: forward projection with the ratio y/ybar,
 * backprojection fused with the closed-form f-update, and the group shrink
 * fused with the dual update -- with SGTV_FLAG_SINGLE_PASS the first two are
 * one pass over the rows that scatters into e, then the f-update -- or, with
 * SGTV_FLAG_PERSISTENT, one cooperative
 * kernel doing the three phases between grid-wide barriers (each wait is
 * bounded: a barrier that does not complete within about 1 s records
 * SGTV_ERR_TIMEOUT, reported by the next sgtv_sync). With SGTV_FLAG_GRAPH,
 * runs of 8 iterations are captured once into CUDA graphs (one per buffer
 * order of the image and the split variable) and replayed, the remainder
 * launched directly; the graphs are rebuilt after the variants change. The
 * first graph use captures the handle's stream: do not call it while that
 * stream is itself being captured. Does not wait for the GPU. */
int sgtv_iterate(sgtv_t h, int32_t n);

/* Wait for the stream; returns SGTV_ERR_NONFINITE if an iteration produced a
 * NaN or Inf since the last check. */
int sgtv_sync(sgtv_t h);

/* Objective at the current f, reduced in FP64 (Eq. 4 with the Poisson
 * deviance as L): phi = dev + lambda * tv, dev = sum_i [ybar - y + y log(y/ybar)]
 * (0 log 0 = 0), tv = R(w.G f) of Eq. 2. For a batch the sums run over all
 * scans and phi = dev + sum_k lambda_k tv_k. Any output pointer may be NULL. */
int sgtv_objective(sgtv_t h, double *phi, double *dev, double *tv);

/* Convergence measures of the ADMM state (Sec. III, Eqs. 5-7, with the
 * constraint d = w.G f of Eq. 4), reduced in FP64:
 *   primal = ||w.G f - d||_2 / max(1, ||d||_2)
 *   dual   = ||rho (w.G)^T (d - d_prev)||_2 / max(1, ||rho (w.G)^T c||_2),
 *            d_prev = d before the last iteration's Eq. 6 step (rho per scan
 *            in a batch). It reads 0 before the first iteration after set-up
 *            and after any call that replaces the state (sgtv_set_state_f64,
 *            sgtv_set_data, sgtv_warm_start, sgtv_warm_start_dual).
 *   kkt    = ||min(f, g)||_inf / max(1, ||s||_inf),
 *            g = s - A^T(y / (A f + r)) + rho (w.G)^T c,  s = A^T 1.
 * Any output pointer may be NULL. */
int sgtv_residuals(sgtv_t h, double *primal, double *dual, double *kkt);

/* Copy f (len must equal J) to the host buffer out. */
int sgtv_get_image(sgtv_t h, float *out, int64_t len);

/* Copy the ADMM state (f [J], d [n_dirs*J], c [n_dirs*J]) to host buffers,
 * converted to double. Any pointer may be NULL to skip that array. */
int sgtv_get_state_f64(sgtv_t h, double *f, double *d, double *c);

/* Replace the state from host buffers (checkpoint resume / warm start).
 * f [J] must be >= 0 and finite. If d and c are both NULL, d = w.G f and
 * c = 0 (the initialisation rule applied to the given f). */
int sgtv_set_state_f64(sgtv_t h, const double *f, const double *d, const double *c);

/* SpMV autotuner. The forward projection and the fused backprojection come
 * in several tilings (segments per warp, prefetch depth, pipelining, register
 * cap). Variants of one element order give bit-identical results; the
 * 4-wide forms ("v4" in the name) split a segment among lanes differently and
 * round differently (equally deterministic), so with the autotuner on, the
 * chosen pair decides the last bits; pin the variants (SGTV_FLAG_NO_AUTOTUNE +
 * sgtv_set_variants) for bit-reproducible runs. sgtv_autotune times every variant
 * `reps` times on the handle's own problem (writing only scratch buffers, the
 * ADMM state is untouched) and keeps the fastest; sgtv_setup runs it with
 * reps = 10 unless SGTV_FLAG_NO_AUTOTUNE is set. In persistent mode it also
 * times the fused kernel's forms (the four tile-form pairs, with and without a
 * register cap) and selects the tiled variants ("tli_u8" / "tli_v4x2") of the
 * fastest; sgtv_set_variants then picks the pair and keeps the register cap.
 * With SGTV_FLAG_SINGLE_PASS it also times the single-pass scatter's forms
 * (one accumulator per block with shared-memory atomic adds, or one per warp
 * summed in a fixed order; prefetch depth; register cap) that fit in shared
 * memory. kernel is SGTV_K_FORWARD, SGTV_K_BACK_UPDATE or SGTV_K_SCATTER (the
 * latter in sgtv_variant_count / _name and sgtv_get_variant / sgtv_set_variant
 * only). The set functions return SGTV_ERR_ARG (not sticky) for an index out
 * of range or a form that does not fit; sgtv_variant_name returns "" for one. */
int sgtv_autotune(sgtv_t h, int32_t reps);
int sgtv_get_variants(sgtv_t h, int32_t *fwd, int32_t *back);
int sgtv_set_variants(sgtv_t h, int32_t fwd, int32_t back);
int sgtv_get_variant(sgtv_t h, int32_t kernel, int32_t *v);
int sgtv_set_variant(sgtv_t h, int32_t kernel, int32_t v);
int sgtv_variant_count(sgtv_t h, int32_t kernel);
const char *sgtv_variant_name(sgtv_t h, int32_t kernel, int32_t v);

/* Tiled local-index forms built at set-up for the CSR (index 0) and CSC
 * (index 1) copies: tiles of 64 rows (columns) carry 16-bit local indices into
 * a staging buffer that is, per tile, the tile's 16-byte-aligned index window
 * (staged by one bulk copy) or its unique-index list (staged by a gather).
 * fmt = 0 not built (plain kernels only), 1 all list, 2 all window, 3 mixed;
 * list_entries = unique-index entries stored over all list tiles;
 * window_elems = window elements summed over all window tiles; max_stage = the
 * largest tile's staging buffer in elements. Each non-NULL pointer must hold
 * 2 values. */
int sgtv_tli_info(sgtv_t h, int32_t *fmt, int64_t *list_entries, int64_t *window_elems,
                  int64_t *max_stage);

/* Replace the counts y [I], the background b [b_len] (b_len as at set-up) and
 * the regularisation weight lambda of a one-scan handle, keeping A, and
 * re-initialise the state by the set-up rule (host pointers, copied). Many
 * measurements of one instrument then share one resident A. SGTV_ERR_DOMAIN
 * (not sticky, nothing changed) for negative or non-finite data. */
int sgtv_set_data(sgtv_t h, const float *y, const float *b, int64_t b_len, double lambda);

/* The normalised backprojection A^T y / A^T 1 (0 where A^T 1 = 0), J floats,
 * written to a device buffer (out_on_device = 1) or a host buffer (0). */
int sgtv_normalized_backprojection(sgtv_t h, float *out, int32_t out_on_device);

/* Warm start: f = max(f0, 0) from J floats in device (on_device = 1) or host
 * (0) memory, then d = w.G f and the scaled dual
 *   c_s = dual_scale * tau * d_s / |d_s|   per spatial group s (0 where d_s = 0),
 * tau = beta / rho of the scan. dual_scale = 0 is the initialisation rule of
 * the method applied to f0 (c = 0); dual_scale = 1 is the dual that the group
 * shrink of Eq. 6 leaves unchanged when f0 is a fixed point (a group with
 * d_s != 0 satisfies d_s = shrink(d_s + c_s) exactly for that c_s). The
 * iteration itself is unchanged either way. dual_scale outside [0, 1] gives
 * SGTV_ERR_ARG; a non-finite f0 gives SGTV_ERR_NONFINITE. */
int sgtv_warm_start(sgtv_t h, const float *f0, int32_t on_device, double dual_scale);

/* Warm start with a given dual: f = max(f0, 0) (J floats), d = w.G f and
 * c = c0 (n_dirs * J floats, direction-major [p][J], in the scaled-dual units
 * of Eq. 7), from device (on_device = 1) or host (0) memory. The iteration
 * itself is unchanged. A start that carries a dual close to the solution's
 * shortens the solve where an image alone does not: the dual restarts from
 * zero otherwise and sets the pace of convergence. A non-finite f0 or c0
 * gives SGTV_ERR_NONFINITE. */
int sgtv_warm_start_dual(sgtv_t h, const float *f0, const float *c0, int32_t on_device);

/* Problem sizes of a handle (any pointer may be NULL). */
int sgtv_info(sgtv_t h, int64_t *I, int64_t *J, int64_t *nnz, int32_t *n_dirs,
              int32_t *precision, int64_t *device_bytes);

/* Kernel timing with CUDA events on the handle's stream. enable = 1 clears
 * the counters and brackets every later launch with events; enable = 0 stops.
 * sgtv_profile_read waits for the stream and writes, for the first n_kernels
 * kernel identifiers (SGTV_K_*), the summed device milliseconds and the launch
 * counts since profiling was enabled. */
int sgtv_profile(sgtv_t h, int32_t enable);
int sgtv_profile_read(sgtv_t h, double *ms, int64_t *launches, int32_t n_kernels);

/* Bound, in nanoseconds, on each wait of a block in the grid-wide barriers
 * of the persistent launch (SGTV_FLAG_PERSISTENT); 1 s by default. A block
 * that waits longer gives up: the launch returns early, the iterate is left
 * incomplete, and the next call that waits for the stream (sgtv_sync and the
 * calls that return data) fails with SGTV_ERR_TIMEOUT, which is sticky. 0
 * gives up at the first look, so a grid of more than one block always times
 * out: a way to test the failure path without a fault. The bound of the bulk
 * copies' waits stays 1 s (a block never leaves a copy into its shared memory
 * in flight). ns < 0 gives SGTV_ERR_ARG (not sticky). Takes effect for the
 * launches enqueued after the call. */
int sgtv_set_wait_limit(sgtv_t h, int64_t ns);

/* Turns SGTV_FLAG_SERIAL on (on != 0) or off for the iterations enqueued
 * after the call: on, every kernel runs on the handle's stream, one after the
 * other, so that sgtv_profile times each kernel alone; off, the shrink runs on
 * the second stream, overlapping the next forward pass. A shrink already
 * queued on the second stream is joined first; CUDA graphs captured in the
 * other mode are dropped. The iterate is the same either way. */
int sgtv_set_serial(sgtv_t h, int32_t on);

/* The CUDA stream the handle issues work on (a cudaStream_t). */
int sgtv_get_stream(sgtv_t h, void **stream);

/*
 * KKT residual of a given state without any device allocation.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc -- code that runs while its stream is being captured into a
 * CUDA graph (allocation is not a capturable operation), code under an
 * external device-memory budget or allocator it must not bypass, and
 * real-time loops that must never stall in the allocator. It computes the
 * numerator and denominator of the KKT measure of sgtv_residuals from state
 * the caller already holds on the device, in FP32 with FP64 reductions:
 *   out[0] = max_j |min(f_j, g_j)|,  g = s - A^T(y / (A f + r)) + rho (w.G)^T c
 *   out[1] = max_j s_j               (kkt = out[0] / max(1, out[1]))
 * Every pointer is a DEVICE pointer on the current device, owned by the
 * caller: the CSR and CSC copies of A (as for sgtv_setup, float values, and
 * already valid: pointers nondecreasing from 0 to nnz, indices in range; the
 * call does not check them, so an index out of range reads out of bounds --
 * pass arrays that passed sgtv_setup's checks), y [I],
 * b [b_len] (1 or I), s = A^T 1 [J], f [J], c [n_dirs * J] (direction-major),
 * w [n_dirs] is a HOST array, out receives 2 doubles. stream is a
 * cudaStream_t (NULL = the legacy default stream). The call only enqueues
 * work; read out after the stream has finished.
 *
 * The scratch it needs (the ratio, the backprojection and the reduction
 * partials) is one fixed array in the library's device memory, about 8 MB,
 * held by every GPU that loads the library until the process exits. Hence the
 * limits I <= SGTV_NOALLOC_MAX_I and J <= SGTV_NOALLOC_MAX_J; larger problems
 * get SGTV_ERR_ARG (text from sgtv_noalloc_last_error). All calls share that
 * array: calls whose kernels may overlap on the GPU (on unordered streams)
 * race and give wrong results; issue them in order on one stream. The first
 * call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture. It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 */
#define SGTV_NOALLOC_MAX_I (1 << 20)
#define SGTV_NOALLOC_MAX_J (1 << 20)
int sgtv_kkt_residual_noalloc(int64_t I, int64_t J, const int64_t *csr_rowptr, const int32_t *csr_col,
                              const float *csr_val, const int64_t *csc_colptr, const int32_t *csc_row,
                              const float *csc_val, int32_t Nx, int32_t Nz, int32_t Nq, int32_t n_dirs,
                              const double *w, const float *y, const float *b, int64_t b_len, const float *s,
                              const float *f, const float *c, double rho, double *out, void *stream);

/* Text of the last sgtv_kkt_residual_noalloc failure on this thread ("" if none). */
const char *sgtv_noalloc_last_error(void);

/* Free everything the handle owns. h may be NULL. */
int sgtv_destroy(sgtv_t h);

/* Text of the handle's last error ("" if none); h = NULL gives the text of the
 * last sgtv_setup failure on this thread. The pointer stays valid until the
 * next call on the same handle. */
const char *sgtv_last_error(sgtv_t h);

/* Name of an SGTV_* code. */
const char *sgtv_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SGTV_H */
