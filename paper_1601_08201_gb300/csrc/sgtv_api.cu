// sgtv_api.cu -- host side of the C ABI declared in include/sgtv.h.
//
// One handle = one reconstruction problem resident on one GPU: A as CSR and CSC,
// y, r, the sensitivity s = A^T 1, the ADMM state (f double-buffered, d, c) and
// scratch for the ratio, the backprojection and the FP64 reductions. All work
// runs on the handle's stream; only the calls that return data synchronise.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/sgtv.h"
#include "sgtv_internal.h"

using namespace sgtv;

namespace {

thread_local std::string g_setup_error;

// Bound of the persistent kernel's grid-barrier waits unless sgtv_set_wait_limit
// sets another: far beyond any healthy phase of an iteration.
constexpr unsigned long long kDefaultWaitNs = 1000000000ull;

struct ProfRec {
    int kernel;
    cudaEvent_t a, b;
};

}  // namespace

struct sgtv_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the shrink (Eqs. 6-7) of iteration k feeds only the f-update of
    // iteration k + 1: it runs on a second stream, forked after the f-update
    // and joined before the next one, so it overlaps the next forward pass
    cudaStream_t side = nullptr;
    cudaEvent_t ev_f = nullptr, ev_shrink = nullptr;
    bool shrink_pending = false;  // a shrink on `side` not yet joined into `stream`
    sgtv_alloc_fn alloc = nullptr;
    sgtv_free_fn free_ = nullptr;
    void *alloc_user = nullptr;
    std::vector<void *> blocks;
    int64_t bytes = 0;

    Geom g{};
    Dev d{};
    const KernelSet *ks = nullptr;
    int precision = SGTV_PREC_FP32;
    int n_inner = 1;
    int flags = 0;
    double beta = 0, rho = 1;   // of scan 0
    bool any_rho = true;        // some scan has rho > 0 (else no shrink is needed)
    int32_t nscans = 1;
    std::vector<int64_t> I_off, J_off, S_off;  // per-scan offsets (nscans + 1)
    std::vector<Scan> scan_tab;
    int v_fwd = 0, v_back = 0;  // chosen SpMV variants (see sgtv_autotune)
    bool persistent = false;    // one cooperative launch per iteration
    int v_pers = 0;             // its variant (KernelSet::pers)
    bool use_graph = false;     // iterations replayed from captured CUDA graphs
    bool single_pass = false;   // A streamed once per surrogate step (scatter + f-update)
    void *e_acc = nullptr;      // its accumulator of e (all zero between iterations)
    int v_scatter = 0;          // its scatter variant (KernelSet::scatter)
    int64_t max_warp_span = 0;  // most nonzeros in kTliTile / 8 consecutive rows
    int64_t max_sp_span = 0;    // the same in the single-pass row stream (padded rows)
    GridBar *bar = nullptr;     // grid barrier of the persistent kernel
    void *bufA = nullptr;       // the first image buffer (graph parity)
    void *dbufA = nullptr;      // the first buffer of d (graph parity)
    // two captured iterations, keyed by the buffer order they start from:
    // index = (f is bufA ? 0 : 1) + 2 * (d is dbufA ? 0 : 1)
    cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};  // kGraphIters iterations each

    int sticky = SGTV_OK;
    std::string err;

    bool prof = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    double prof_ms[SGTV_K_COUNT] = {};
    int64_t prof_n[SGTV_K_COUNT] = {};
};

namespace {

int fail(sgtv_t h, int code, const std::string &msg)
{
    if (h) {
        if (h->sticky == SGTV_OK) {
            h->sticky = code;
            h->err = msg;
        }
    } else {
        g_setup_error = msg;
    }
    return code;
}

int cuda_fail(sgtv_t h, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? SGTV_ERR_OOM : SGTV_ERR_CUDA, m);
}

#define CK(h, call)                                        \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

void *dev_alloc(sgtv_t h, size_t bytes, cudaError_t *err)
{
    if (bytes < 16) bytes = 16;
    void *p = nullptr;
    if (h->alloc) {
        p = h->alloc(bytes, h->alloc_user);
        *err = p ? cudaSuccess : cudaErrorMemoryAllocation;
    } else {
        *err = cudaMalloc(&p, bytes);
        if (*err != cudaSuccess) p = nullptr;
    }
    if (p) {
        h->blocks.push_back(p);
        h->bytes += int64_t(bytes);
    }
    return p;
}

void dev_free(sgtv_t h, void *p)
{
    if (!p) return;
    for (size_t k = 0; k < h->blocks.size(); k++)
        if (h->blocks[k] == p) {
            h->blocks.erase(h->blocks.begin() + k);
            break;
        }
    if (h->free_) h->free_(p, h->alloc_user);
    else cudaFree(p);
}

void release(sgtv_t h)
{
    if (!h) return;
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto &r : h->recs) {
        if (r.kernel < 0) continue;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
    for (auto &ge : h->gexec)
        if (ge) cudaGraphExecDestroy(ge);
    for (void *p : h->blocks) {
        if (h->free_) h->free_(p, h->alloc_user);
        else cudaFree(p);
    }
    h->blocks.clear();
    if (h->ev_f) cudaEventDestroy(h->ev_f);
    if (h->ev_shrink) cudaEventDestroy(h->ev_shrink);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Iterations captured in one CUDA graph (even: the image and split-variable
// buffers are back in their starting order after it).
constexpr int kGraphIters = 8;

// Order the pending shrink before later work on the handle's stream.
cudaError_t join_shrink(sgtv_t h)
{
    if (!h->shrink_pending) return cudaSuccess;
    h->shrink_pending = false;
    return cudaStreamWaitEvent(h->stream, h->ev_shrink, 0);
}

int check_live(sgtv_t h)
{
    if (!h) return SGTV_ERR_ARG;
    if (h->sticky != SGTV_OK) return SGTV_ERR_STATE;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    return SGTV_OK;
}

// Whether an SpMV variant can run on this handle (its tiled form was built
// and, for the TMA pipelines, NS stages fit in shared memory).
bool variant_ok(const TliMat &m, int need)
{
    if (need == 0) return true;
    if (m.fmt == 0) return false;
    if (need == 1) return true;
    return m.tma_stage_bytes > 0 && int64_t(need) * m.tma_stage_bytes <= m.smem_optin - 1024;
}

// The persistent kernel's tile forms follow the chosen tiled variants
// ("tli_u8" -> strided, "tli_v4x2" -> 4-wide); -1 if either is another form.
int pers_index(sgtv_t h, int fwd, int back)
{
    auto form = [](const char *name) {
        const std::string n(name);
        return n == "tli_u8" ? 0 : (n == "tli_v4x2" ? 1 : -1);
    };
    const int a = form(h->ks->fwd_name[fwd]), b = form(h->ks->back_name[back]);
    return (a < 0 || b < 0) ? -1 : 2 * a + b;
}

void drop_graphs(sgtv_t h)
{
    for (auto &ge : h->gexec)
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
}

cudaEvent_t take_event(sgtv_t h)
{
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch `fn` (on stream st) bracketed by events when profiling is on.
template <typename F>
void timed_on(sgtv_t h, cudaStream_t st, int kernel, F &&fn)
{
    if (!h->prof) {
        fn();
        return;
    }
    ProfRec r{kernel, take_event(h), take_event(h)};
    cudaEventRecord(r.a, st);
    fn();
    cudaEventRecord(r.b, st);
    h->recs.push_back(r);
}

template <typename F>
void timed(sgtv_t h, int kernel, F &&fn)
{
    timed_on(h, h->stream, kernel, fn);
}

bool finite_nonneg(double v) { return v >= 0.0 && isfinite(v); }

int validate_ptr(sgtv_t h, const int64_t *ptr, int64_t n, int64_t nnz, const char *name)
{
    (void)h;
    if (ptr[0] != 0) return fail(nullptr, SGTV_ERR_DOMAIN, std::string(name) + "[0] != 0");
    for (int64_t k = 0; k < n; k++)
        if (ptr[k + 1] < ptr[k])
            return fail(nullptr, SGTV_ERR_DOMAIN, std::string(name) + " is not nondecreasing");
    if (ptr[n] != nnz) return fail(nullptr, SGTV_ERR_DOMAIN, std::string(name) + "[n] != nnz");
    return SGTV_OK;
}

// A single-pass scatter form fits when its staging-sized buffers (f and the
// accumulators) fit in the opt-in shared memory of one block.
bool scatter_fits(sgtv_t h, int v)
{
    const TliMat &m = h->d.tr;
    if (m.fmt == 0 || h->max_warp_span >= (int64_t(1) << 31)) return false;
    const bool sp = h->ks->scatter_sp[v] != 0;
    if (sp && (!h->d.sp.built || h->max_sp_span >= (int64_t(1) << 31))) return false;
    // the row-stream forms keep one more slot (the padding's dummy entry)
    const int64_t cap = sp ? ((int64_t(m.max_stage) + 2) & ~int64_t(1)) : ((int64_t(m.max_stage) + 1) & ~int64_t(1));
    return int64_t(h->ks->scatter_bufs[v]) * cap * h->ks->elem_size <= h->d.smem_optin - 1024;
}

// d and d_prev trade places after each shrink: d^{k+1} was written over d^{k-1}.
void swap_d(Dev &d)
{
    void *t = d.d;
    d.d = d.d_prev;
    d.d_prev = t;
}

// d_prev = d: a state set from outside has no previous split variable, so
// its dual residual reads 0 until the next iteration. Also u = d - c, the
// single-pass f-update's operand that the shrink otherwise keeps.
cudaError_t copy_d_to_prev(sgtv_t h)
{
    cudaError_t e = cudaMemcpyAsync(h->d.d_prev, h->d.d, size_t(h->ks->elem_size) * h->d.J * h->g.n_dirs,
                                    cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && h->d.u) {
        h->ks->sub(h->d.J * h->g.n_dirs, h->d.d, h->d.c, h->d.u, h->stream);
        e = cudaGetLastError();
    }
    return e;
}

// One ADMM iteration: n_inner surrogate steps with d, c fixed, then shrink +
// dual; in persistent mode all of it is one cooperative launch.
cudaError_t enqueue_iteration(sgtv_t h)
{
    Dev &d = h->d;
    if (h->persistent) {
        cudaError_t e = join_shrink(h);
        if (e != cudaSuccess) return e;
        const int pv = h->v_pers;
        timed(h, SGTV_K_ITERATION,
              [&] { e = h->ks->pers[pv](d, h->g, d.f, d.f_next, h->any_rho ? 1 : 0, h->bar, h->stream); });
        void *t = d.f;
        d.f = d.f_next;
        d.f_next = t;
        if (h->any_rho) swap_d(d);
        return e;
    }
    for (int k = 0; k < h->n_inner; k++) {
        if (h->single_pass) {
            timed(h, SGTV_K_SCATTER, [&] { h->ks->scatter[h->v_scatter](d, d.f, h->e_acc, h->stream); });
            cudaError_t e = join_shrink(h);  // the previous shrink's u
            if (e != cudaSuccess) return e;
            timed(h, SGTV_K_FUPDATE, [&] { h->ks->fupdate(d, h->g, h->e_acc, d.f, d.f_next, h->stream); });
            void *t = d.f;
            d.f = d.f_next;
            d.f_next = t;
            continue;
        }
        timed(h, SGTV_K_FORWARD, [&] { h->ks->fwd[h->v_fwd](d, d.f, d.ratio, h->stream); });
        cudaError_t e = join_shrink(h);  // the previous shrink's d and c
        if (e != cudaSuccess) return e;
        timed(h, SGTV_K_BACK_UPDATE, [&] { h->ks->back[h->v_back](d, h->g, d.f, d.f_next, h->stream); });
        void *t = d.f;
        d.f = d.f_next;
        d.f_next = t;
    }
    if (h->any_rho && (h->flags & SGTV_FLAG_SERIAL)) {
        timed(h, SGTV_K_SHRINK, [&] { h->ks->shrink(d, h->g, d.f, d.d_prev, h->stream); });
        swap_d(d);
    } else if (h->any_rho) {
        // fork: the shrink of this iteration's image on the second stream
        cudaError_t e = cudaEventRecord(h->ev_f, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_f, 0);
        if (e != cudaSuccess) return e;
        timed_on(h, h->side, SGTV_K_SHRINK, [&] { h->ks->shrink(d, h->g, d.f, d.d_prev, h->side); });
        e = cudaEventRecord(h->ev_shrink, h->side);
        if (e != cudaSuccess) return e;
        h->shrink_pending = true;
        swap_d(d);
    }
    return cudaGetLastError();
}

// Capture two iterations (starting from the current image buffer) into a
// CUDA graph; replaying it leaves the buffers in the same order.
cudaError_t capture_pair(sgtv_t h, cudaGraphExec_t *out)
{
    const bool prof = h->prof;
    h->prof = false;  // events are recorded around graph launches instead
    cudaGraph_t graph = nullptr;
    cudaError_t e = join_shrink(h);  // nothing from before the capture is waited on inside it
    if (e == cudaSuccess) e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaError_t e1 = cudaSuccess;
        for (int k = 0; k < kGraphIters && e1 == cudaSuccess; k++) e1 = enqueue_iteration(h);
        if (e1 == cudaSuccess) e1 = join_shrink(h);  // the graph ends with every shrink joined
        e = cudaStreamEndCapture(h->stream, &graph);
        if (e == cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    h->prof = prof;
    return e;
}

int read_red(sgtv_t h, double *host, int n)
{
    CK(h, cudaMemcpyAsync(host, h->d.red, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return SGTV_OK;
}

// Build the tiled local-index form of one compressed matrix (ptr, idx with
// nseg segments). Each tile whose 16-byte-aligned index window fits the
// staging cap becomes a window tile; every other tile a list tile, which needs
// its unique index count to fit the cap (else fmt stays 0: plain kernels only).
int build_tli(sgtv_t h, const int64_t *ptr, const int64_t *host_ptr, const int32_t *idx, int64_t nseg,
              int64_t nnz_pad, int64_t n_dense, TliMat &m)
{
    m = TliMat{};
    m.smem_optin = h->d.smem_optin;
    cudaStream_t st = h->stream;
    const int64_t ntiles = (nseg + kTliTile - 1) / kTliTile;
    const int esz = h->ks->elem_size;
    const int64_t cap = (96 * 1024) / esz < 65536 ? (96 * 1024) / esz : 65536;
    cudaError_t ae;
    std::vector<void *> tmp;
    auto cleanup = [&]() {
        for (void *p : tmp) dev_free(h, p);
    };
    auto talloc = [&](size_t bytes) {
        void *p = dev_alloc(h, bytes, &ae);
        if (p) tmp.push_back(p);
        return p;
    };
    int32_t *tmin = static_cast<int32_t *>(talloc(sizeof(int32_t) * ntiles));
    int32_t *tmax = static_cast<int32_t *>(talloc(sizeof(int32_t) * ntiles));
    if (!tmin || !tmax) { cleanup(); return cuda_fail(h, ae, "device allocation"); }
    tli_tile_range(ptr, idx, nseg, ntiles, tmin, tmax, st);
    std::vector<int32_t> hmin(ntiles), hmax(ntiles);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hmin.data(), tmin, sizeof(int32_t) * ntiles, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hmax.data(), tmax, sizeof(int32_t) * ntiles, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(h, e, "tile ranges"); }
    const int64_t align = 16 / esz;
    std::vector<int32_t> wb(ntiles, 0), wl(ntiles, 0);
    int64_t max_stage = 0, max_list_range = 0, n_list = 0, n_win = 0, max_win = 0;
    for (int64_t t = 0; t < ntiles; t++) {
        if (hmax[t] < 0) continue;  // empty tile: nothing to stage
        const int64_t b = (int64_t(hmin[t]) / align) * align;
        const int64_t en = ((int64_t(hmax[t]) + 1 + align - 1) / align) * align;
        if (en - b <= cap) {
            wb[t] = int32_t(b);
            wl[t] = int32_t(en - b);
            if (en - b > max_stage) max_stage = en - b;
            if (en - b > max_win) max_win = en - b;
            n_win++;
        } else {
            n_list++;
            if (int64_t(hmax[t]) - hmin[t] + 1 > max_list_range) max_list_range = int64_t(hmax[t]) - hmin[t] + 1;
        }
    }
    // bitmap words of the list build (a wider tile range is processed in chunks)
    const int words = int((max_list_range + 31) / 32 < tli_list_max_words() ? (max_list_range + 31) / 32
                                                                             : tli_list_max_words());
    std::vector<int64_t> off(ntiles + 1, 0);
    if (n_list > 0) {
        int32_t *ucnt = static_cast<int32_t *>(talloc(sizeof(int32_t) * ntiles));
        if (!ucnt) { cleanup(); return cuda_fail(h, ae, "device allocation"); }
        // tile ranges of window tiles may exceed the bitmap: count list tiles only
        std::vector<int32_t> lmax(hmax);
        for (int64_t t = 0; t < ntiles; t++)
            if (wl[t] > 0) lmax[t] = -1;
        int32_t *tmax_l = static_cast<int32_t *>(talloc(sizeof(int32_t) * ntiles));
        if (!tmax_l) { cleanup(); return cuda_fail(h, ae, "device allocation"); }
        e = cudaMemcpyAsync(tmax_l, lmax.data(), sizeof(int32_t) * ntiles, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = tli_list_count(ptr, idx, nseg, ntiles, tmin, tmax_l, words, ucnt, st);
        std::vector<int32_t> hc(ntiles);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), ucnt, sizeof(int32_t) * ntiles, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(h, e, "tile unique counts"); }
        for (int64_t t = 0; t < ntiles; t++) {
            const int64_t c = (wl[t] > 0 || hmax[t] < 0) ? 0 : hc[t];
            off[t + 1] = off[t] + c;
            if (c > max_stage) max_stage = c;
        }
        if (max_stage > cap) { cleanup(); return SGTV_OK; }  // fmt 0
        tmax = tmax_l;
    }
    m.lidx = static_cast<uint16_t *>(dev_alloc(h, sizeof(uint16_t) * nnz_pad, &ae));
    m.wbase = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * ntiles, &ae));
    m.wlen = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * ntiles, &ae));
    m.uoff = static_cast<int64_t *>(dev_alloc(h, sizeof(int64_t) * (ntiles + 1), &ae));
    m.uidx = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (off[ntiles] + 8), &ae));
    if (!m.lidx || !m.wbase || !m.wlen || !m.uoff || !m.uidx) {
        cleanup();
        return cuda_fail(h, ae, "device allocation");
    }
    e = cudaMemsetAsync(m.lidx, 0, sizeof(uint16_t) * nnz_pad, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.uidx, 0, sizeof(int32_t) * (off[ntiles] + 8), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.wbase, wb.data(), sizeof(int32_t) * ntiles, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.wlen, wl.data(), sizeof(int32_t) * ntiles, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.uoff, off.data(), sizeof(int64_t) * (ntiles + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_win > 0) {
        tli_window_lidx(ptr, idx, nseg, m.wbase, m.wlen, m.lidx, h->d.sm_count, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n_list > 0)
        e = tli_list_build(ptr, idx, nseg, ntiles, tmin, tmax, m.wlen, words, m.uoff, m.uidx, m.lidx, st);
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d.flag, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        tli_check(ptr, nseg, m.lidx, m.wlen, m.uoff, m.uidx, n_dense, h->d.flag, h->d.sm_count, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, h->d.flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(h, e, "tiled index build");
    if (hflag) return fail(h, SGTV_ERR_CUDA, "internal: a tiled local index fell outside its staging buffer");
    m.ntiles = ntiles;
    m.max_stage = int(max_stage);
    m.fmt = (n_list > 0 && n_win > 0) ? 3 : (n_win > 0 ? 2 : 1);
    // One stage of the TMA pipeline: segment pointers, local indices and
    // values of the largest tile (plus 16-byte alignment slack), its list
    // entries and its staging buffer.
    int64_t max_nnz = 0, max_list = 0;
    for (int64_t t = 0; t < ntiles; t++) {
        const int64_t a = host_ptr[t * kTliTile];
        const int64_t b = host_ptr[(t + 1) * kTliTile < nseg ? (t + 1) * kTliTile : nseg];
        if (b - a > max_nnz) max_nnz = b - a;
        if (off[t + 1] - off[t] > max_list) max_list = off[t + 1] - off[t];
    }
    // A window tile stages its window; a list tile its values and, behind
    // them, its list (the two never share a tile, so they share the region).
    auto r128 = [](int64_t v) { return (v + 127) & ~int64_t(127); };
    const int64_t vsz = h->ks->val_size;
    const int64_t b_ptr = r128((kTliTile + 2) * 8);
    const int64_t b_lidx = r128((max_nnz + 16) * 2);
    const int64_t b_val = r128((max_nnz + 2 * (16 / vsz)) * vsz);
    const int64_t off_xs = b_ptr + b_lidx + b_val;
    const int64_t b_list = max_list > 0 ? r128(max_list * esz) + r128((max_list + 8) * 4) : 0;
    const int64_t b_region = r128(max_win * esz) > b_list ? r128(max_win * esz) : b_list;
    const int64_t stage = off_xs + b_region;
    if (stage * 3 <= h->d.smem_optin - 1024) {
        m.tma_off_lidx = int(b_ptr);
        m.tma_off_val = int(b_ptr + b_lidx);
        m.tma_off_xs = int(off_xs);
        m.tma_off_uidx = int(off_xs + r128(max_list * esz));
        m.tma_stage_bytes = int(stage);
    }
    return SGTV_OK;
}

}  // namespace

extern "C" {

void sgtv_default_opts(sgtv_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    for (int p = 0; p < 4; p++) o->w[p] = 1.0;
    o->n_dirs = 4;
    o->n_inner = 1;
    o->precision = SGTV_PREC_FP32;
}

// Set-up of one or more independent scans (sgtv_setup is the one-scan case).
// The scans are concatenated: hyper-voxels, sites and measurements back to
// back in scan order, A block-diagonal with each scan's column (row) indices
// offset by the hyper-voxels (measurements) of the scans before it.
static int setup_impl(sgtv_t *out, int32_t nscans, const sgtv_scan *sc, const sgtv_opts *opts_in)
{
    g_setup_error.clear();
    if (!out) return fail(nullptr, SGTV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nscans < 1 || !sc) return fail(nullptr, SGTV_ERR_ARG, "need at least one scan");
    sgtv_opts opts;
    if (opts_in) opts = *opts_in;
    else sgtv_default_opts(&opts);

    // ---- host-side validation (no CUDA call before this passes) ----
    if (opts.n_dirs != 4 && opts.n_dirs != 2) return fail(nullptr, SGTV_ERR_ARG, "n_dirs must be 4 or 2");
    if (opts.n_inner < 1) return fail(nullptr, SGTV_ERR_ARG, "n_inner must be >= 1");
    if (opts.flags & ~int32_t(127)) return fail(nullptr, SGTV_ERR_ARG, "unknown flag bits");
    if (opts.precision < SGTV_PREC_FP32 || opts.precision > SGTV_PREC_FP64)
        return fail(nullptr, SGTV_ERR_ARG, "unknown precision");
    if ((opts.alloc == nullptr) != (opts.free_ == nullptr))
        return fail(nullptr, SGTV_ERR_ARG, "alloc and free_ must be given together");
    for (int p = 0; p < opts.n_dirs; p++)
        if (!finite_nonneg(opts.w[p])) return fail(nullptr, SGTV_ERR_DOMAIN, "weights must be finite and >= 0");
    std::vector<int64_t> I_off(nscans + 1, 0), J_off(nscans + 1, 0), N_off(nscans + 1, 0), S_off(nscans + 1, 0);
    std::vector<double> sum_y(nscans, 0.0), sum_r(nscans, 0.0);
    bool any_rho = false;
    for (int32_t k = 0; k < nscans; k++) {
        const sgtv_scan &q = sc[k];
        const std::string who = nscans > 1 ? "scan " + std::to_string(k) + ": " : "";
        if (!q.csr_rowptr || !q.csr_col || !q.csr_val || !q.csc_colptr || !q.csc_row || !q.csc_val || !q.y || !q.b)
            return fail(nullptr, SGTV_ERR_ARG, who + "a required pointer is NULL");
        if (q.I < 1 || q.J < 1 || q.nnz < 0 || q.I >= (int64_t(1) << 31) || q.J >= (int64_t(1) << 31))
            return fail(nullptr, SGTV_ERR_ARG, who + "I and J must be in [1, 2^31), nnz >= 0");
        if (q.Nx < 1 || q.Nz < 1 || q.Nq < 1 || int64_t(q.Nx) * q.Nz * q.Nq != q.J)
            return fail(nullptr, SGTV_ERR_ARG, who + "J != Nx * Nz * Nq");
        if (q.b_len != 1 && q.b_len != q.I) return fail(nullptr, SGTV_ERR_ARG, who + "b_len must be 1 or I");
        if (!(q.lambda >= 0.0) || !isfinite(q.lambda))
            return fail(nullptr, SGTV_ERR_DOMAIN, who + "lambda must be finite and >= 0");
        if (!isfinite(q.rho) || q.rho < 0.0 || (q.rho == 0.0 && !(opts.flags & SGTV_FLAG_ALLOW_RHO0)))
            return fail(nullptr, SGTV_ERR_DOMAIN, who + "rho must be finite and > 0");
        any_rho |= q.rho > 0.0;
        int rc;
        if ((rc = validate_ptr(nullptr, q.csr_rowptr, q.I, q.nnz, "csr_rowptr")) != SGTV_OK) return rc;
        if ((rc = validate_ptr(nullptr, q.csc_colptr, q.J, q.nnz, "csc_colptr")) != SGTV_OK) return rc;
        for (int64_t i = 0; i < q.I; i++) {
            if (!finite_nonneg(q.y[i])) return fail(nullptr, SGTV_ERR_DOMAIN, who + "y must be finite and >= 0");
            sum_y[k] += q.y[i];
        }
        for (int64_t i = 0; i < q.b_len; i++)
            if (!finite_nonneg(q.b[i])) return fail(nullptr, SGTV_ERR_DOMAIN, who + "b must be finite and >= 0");
        for (int64_t i = 0; i < q.I; i++) {
            const double ri = q.b[q.b_len == 1 ? 0 : i];
            sum_r[k] += ri;
            if (ri == 0.0 && q.y[i] > 0.0 && q.csr_rowptr[i + 1] == q.csr_rowptr[i])
                return fail(nullptr, SGTV_ERR_DOMAIN, who + "an empty row with y > 0 and r = 0 has ybar = 0");
        }
        I_off[k + 1] = I_off[k] + q.I;
        J_off[k + 1] = J_off[k] + q.J;
        N_off[k + 1] = N_off[k] + q.nnz;
        S_off[k + 1] = S_off[k] + int64_t(q.Nx) * q.Nz;
    }
    const int64_t I = I_off[nscans], J = J_off[nscans], nnz = N_off[nscans];
    if (I >= (int64_t(1) << 31) || J >= (int64_t(1) << 31))
        return fail(nullptr, SGTV_ERR_ARG, "the scans' total I and J must be below 2^31");
    const bool r_scalar = nscans == 1 && sc[0].b_len == 1;

    // ---- device set-up ----
    sgtv_t h = new sgtv_ctx();
    h->alloc = opts.alloc;
    h->free_ = opts.free_;
    h->alloc_user = opts.alloc_user;
    h->precision = opts.precision;
    h->n_inner = opts.n_inner;
    h->flags = opts.flags;
    h->persistent = (opts.flags & SGTV_FLAG_PERSISTENT) != 0;
    h->use_graph = (opts.flags & SGTV_FLAG_GRAPH) != 0;
    h->single_pass = (opts.flags & SGTV_FLAG_SINGLE_PASS) != 0;
    h->beta = sc[0].lambda;
    h->rho = sc[0].rho;
    h->any_rho = any_rho;
    h->nscans = nscans;
    h->I_off = I_off;
    h->J_off = J_off;
    h->S_off = S_off;
    h->ks = opts.precision == SGTV_PREC_FP64 ? &kset_f64
          : opts.precision == SGTV_PREC_BF16VAL ? &kset_bf16 : &kset_f32;
    Geom &g = h->g;
    g.n_dirs = opts.n_dirs;
    g.per_bin = (opts.flags & SGTV_FLAG_STANDARD_TV) ? 1 : 0;
    g.nscans = nscans;
    g.max_nq = 0;
    for (int32_t k = 0; k < nscans; k++) g.max_nq = sc[k].Nq > g.max_nq ? sc[k].Nq : g.max_nq;
    g.J = J;
    g.S = S_off[nscans];
    static const int dx4[4] = {+1, -1, 0, 0}, dz4[4] = {0, 0, +1, -1};
    static const int dx2[4] = {+1, 0, 0, 0}, dz2[4] = {0, +1, 0, 0};
    for (int p = 0; p < 4; p++) {
        g.dx[p] = opts.n_dirs == 4 ? dx4[p] : dx2[p];
        g.dz[p] = opts.n_dirs == 4 ? dz4[p] : dz2[p];
        g.w[p] = p < opts.n_dirs ? opts.w[p] : 0.0;
        g.wf[p] = float(g.w[p]);
    }

    auto bail = [&](int code) {
        g_setup_error = h->err.empty() ? std::string(sgtv_strerror(code)) : h->err;
        release(h);
        return code;
    };
#define SK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return bail(cuda_fail(h, e_, #call)); \
    } while (0)

    SK(cudaGetDevice(&h->device));
    int sms = 0;
    SK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    int optin = 0;
    SK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    if (opts.stream) {
        h->stream = static_cast<cudaStream_t>(opts.stream);
    } else {
        SK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    SK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    SK(cudaEventCreateWithFlags(&h->ev_f, cudaEventDisableTiming));
    SK(cudaEventCreateWithFlags(&h->ev_shrink, cudaEventDisableTiming));
    cudaStream_t st = h->stream;
    Dev &d = h->d;
    d.I = I; d.J = J; d.nnz = nnz;
    d.sm_count = sms;
    d.smem_optin = optin;
    d.red_blocks = 2 * sms;

    const size_t T = h->ks->elem_size, V = h->ks->val_size;
    // index/value arrays: zero padding past nnz for aligned vector and bulk copies
    const int64_t nnz_pad = ((nnz + 15) & ~int64_t(15)) + 16;
    // segment pointers: padded with nnz (empty segments) to whole tiles + 2
    const int64_t I_ptr = ((I + kTliTile - 1) / kTliTile) * kTliTile + 2;
    const int64_t J_ptr = ((J + kTliTile - 1) / kTliTile) * kTliTile + 2;
    cudaError_t ae;
#define ALLOC(ptr, bytes)                                         \
    do {                                                          \
        ptr = dev_alloc(h, (bytes), &ae);                         \
        if (!ptr) return bail(cuda_fail(h, ae, "device allocation")); \
    } while (0)
    void *p_rowptr, *p_colptr, *p_col, *p_row, *p_rval, *p_cval, *p_y, *p_r;
    ALLOC(p_rowptr, sizeof(int64_t) * I_ptr);
    ALLOC(p_colptr, sizeof(int64_t) * J_ptr);
    ALLOC(p_col, sizeof(int32_t) * nnz_pad);
    ALLOC(p_row, sizeof(int32_t) * nnz_pad);
    ALLOC(p_rval, V * nnz_pad);
    ALLOC(p_cval, V * nnz_pad);
    ALLOC(p_y, T * I);
    ALLOC(p_r, T * (r_scalar ? 1 : I));
    ALLOC(d.s, T * J);
    // f and ratio are staged by 16-byte-aligned tile windows: pad to 16 elements
    const int64_t J_pad = (J + 15) & ~int64_t(15), I_pad = (I + 15) & ~int64_t(15);
    ALLOC(d.f, T * J_pad);
    ALLOC(d.f_next, T * J_pad);
    h->bufA = d.f;
    ALLOC(d.ratio, T * I_pad);
    SK(cudaMemsetAsync(d.f, 0, T * J_pad, st));
    SK(cudaMemsetAsync(d.f_next, 0, T * J_pad, st));
    SK(cudaMemsetAsync(d.ratio, 0, T * I_pad, st));
    ALLOC(d.e, T * J);
    ALLOC(d.d, T * J * g.n_dirs);
    ALLOC(d.d_prev, T * J * g.n_dirs);
    h->dbufA = d.d;
    ALLOC(d.c, T * J * g.n_dirs);
    void *p_part, *p_red, *p_flag, *p_scans, *p_voff, *p_soff;
    ALLOC(p_part, sizeof(double) * 4 * d.red_blocks);
    ALLOC(p_red, sizeof(double) * 8);
    ALLOC(p_flag, sizeof(int) * 4);
    ALLOC(p_scans, sizeof(Scan) * nscans);
    void *p_bar;
    ALLOC(p_bar, sizeof(GridBar));
    {
        static GridBar bar0 = {0u, 0u, kDefaultWaitNs};
        SK(cudaMemcpyAsync(p_bar, &bar0, sizeof(GridBar), cudaMemcpyHostToDevice, st));
    }
    h->bar = static_cast<GridBar *>(p_bar);
    ALLOC(p_voff, sizeof(int64_t) * (nscans + 1));
    ALLOC(p_soff, sizeof(int64_t) * (nscans + 1));
    d.rowptr = static_cast<int64_t *>(p_rowptr);
    d.colptr = static_cast<int64_t *>(p_colptr);
    d.col = static_cast<int32_t *>(p_col);
    d.row = static_cast<int32_t *>(p_row);
    d.rval = p_rval;
    d.cval = p_cval;
    d.y = p_y;
    d.r = p_r;
    d.r_scalar = r_scalar;
    d.part = static_cast<double *>(p_part);
    d.red = static_cast<double *>(p_red);
    d.flag = static_cast<int *>(p_flag);
    g.scans = static_cast<Scan *>(p_scans);
    g.vox_off = static_cast<int64_t *>(p_voff);
    g.site_off = static_cast<int64_t *>(p_soff);
    {
        std::vector<Scan> tab(nscans);
        for (int32_t k = 0; k < nscans; k++) {
            tab[k].vox0 = J_off[k];
            tab[k].site0 = S_off[k];
            tab[k].Nx = sc[k].Nx;
            tab[k].Nz = sc[k].Nz;
            tab[k].Nq = sc[k].Nq;
            tab[k].pad_ = 0;
            tab[k].rho = sc[k].rho;
            tab[k].tau = sc[k].rho > 0.0 ? sc[k].lambda / sc[k].rho : 0.0;
            tab[k].beta = sc[k].lambda;
            tab[k].rhof = float(tab[k].rho);
            tab[k].tauf = float(tab[k].tau);
        }
        h->scan_tab = tab;
        SK(cudaMemcpyAsync(p_scans, h->scan_tab.data(), sizeof(Scan) * nscans, cudaMemcpyHostToDevice, st));
        SK(cudaMemcpyAsync(p_voff, h->J_off.data(), sizeof(int64_t) * (nscans + 1), cudaMemcpyHostToDevice, st));
        SK(cudaMemcpyAsync(p_soff, h->S_off.data(), sizeof(int64_t) * (nscans + 1), cudaMemcpyHostToDevice, st));
    }

    // Upload. Padding past nnz is zeroed (index 0, value 0): the aligned vector
    // and bulk loads of the SpMVs may touch it but never use it.
    SK(cudaMemsetAsync(p_col, 0, sizeof(int32_t) * nnz_pad, st));
    SK(cudaMemsetAsync(p_row, 0, sizeof(int32_t) * nnz_pad, st));
    std::vector<int64_t> tail(size_t(kTliTile + 2), nnz);
    SK(cudaMemcpyAsync(static_cast<int64_t *>(p_rowptr) + I, tail.data(), sizeof(int64_t) * (I_ptr - I),
                       cudaMemcpyHostToDevice, st));
    SK(cudaMemcpyAsync(static_cast<int64_t *>(p_colptr) + J, tail.data(), sizeof(int64_t) * (J_ptr - J),
                       cudaMemcpyHostToDevice, st));
    // Values arrive as float; the FP32 mode keeps them, the others convert.
    float *fr = nullptr, *fc = nullptr;
    void *tmp_r = nullptr, *tmp_c = nullptr;
    if (h->precision == SGTV_PREC_FP32) {
        fr = static_cast<float *>(p_rval);
        fc = static_cast<float *>(p_cval);
        SK(cudaMemsetAsync(p_rval, 0, V * nnz_pad, st));
        SK(cudaMemsetAsync(p_cval, 0, V * nnz_pad, st));
    } else {
        ALLOC(tmp_r, sizeof(float) * nnz_pad);
        ALLOC(tmp_c, sizeof(float) * nnz_pad);
        SK(cudaMemsetAsync(tmp_r, 0, sizeof(float) * nnz_pad, st));
        SK(cudaMemsetAsync(tmp_c, 0, sizeof(float) * nnz_pad, st));
        fr = static_cast<float *>(tmp_r);
        fc = static_cast<float *>(tmp_c);
    }
    SK(cudaMemsetAsync(d.flag, 0, sizeof(int) * 4, st));
    for (int32_t k = 0; k < nscans; k++) {
        const sgtv_scan &q = sc[k];
        int64_t *rp = static_cast<int64_t *>(p_rowptr) + I_off[k];
        int64_t *cp = static_cast<int64_t *>(p_colptr) + J_off[k];
        SK(cudaMemcpyAsync(rp, q.csr_rowptr, sizeof(int64_t) * q.I, cudaMemcpyHostToDevice, st));
        SK(cudaMemcpyAsync(cp, q.csc_colptr, sizeof(int64_t) * q.J, cudaMemcpyHostToDevice, st));
        if (q.nnz > 0) {
            int32_t *cl = static_cast<int32_t *>(p_col) + N_off[k];
            int32_t *rw = static_cast<int32_t *>(p_row) + N_off[k];
            SK(cudaMemcpyAsync(cl, q.csr_col, sizeof(int32_t) * q.nnz, cudaMemcpyHostToDevice, st));
            SK(cudaMemcpyAsync(rw, q.csc_row, sizeof(int32_t) * q.nnz, cudaMemcpyHostToDevice, st));
            SK(cudaMemcpyAsync(fr + N_off[k], q.csr_val, sizeof(float) * q.nnz, cudaMemcpyHostToDevice, st));
            SK(cudaMemcpyAsync(fc + N_off[k], q.csc_val, sizeof(float) * q.nnz, cudaMemcpyHostToDevice, st));
            // each scan's indices must stay inside its own block
            validate_indices(cl, q.nnz, q.J, d.flag, st);
            validate_indices(rw, q.nnz, q.I, d.flag, st);
            if (nscans > 1) {
                add_offset_i32(cl, q.nnz, int32_t(J_off[k]), st);
                add_offset_i32(rw, q.nnz, int32_t(I_off[k]), st);
            }
        }
        if (nscans > 1) {
            add_offset_i64(rp, q.I, N_off[k], st);
            add_offset_i64(cp, q.J, N_off[k], st);
        }
    }
    validate_values(fr, nnz, d.flag, st);
    validate_values(fc, nnz, d.flag, st);
    SK(cudaGetLastError());
    int hflag = 0;
    SK(cudaMemcpyAsync(&hflag, d.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SK(cudaStreamSynchronize(st));
    if (hflag & 1) return bail(fail(h, SGTV_ERR_DOMAIN, "an index of A is out of range"));
    if (hflag & 2) return bail(fail(h, SGTV_ERR_DOMAIN, "A has a negative or non-finite value"));
    validate_sorted(d.rowptr, d.col, I, d.flag, sms, st);
    validate_sorted(d.colptr, d.row, J, d.flag, sms, st);
    SK(cudaGetLastError());
    SK(cudaMemcpyAsync(&hflag, d.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SK(cudaStreamSynchronize(st));
    if (hflag & 8)
        return bail(fail(h, SGTV_ERR_DOMAIN, "indices must be strictly ascending inside each row and column"));
    validate_match(I, d.rowptr, d.col, fr, d.colptr, d.row, fc, d.flag, sms, st);
    SK(cudaGetLastError());
    SK(cudaMemcpyAsync(&hflag, d.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    SK(cudaStreamSynchronize(st));
    if (hflag & 4) return bail(fail(h, SGTV_ERR_DOMAIN, "the CSR and CSC copies of A differ"));
    std::vector<int64_t> hrp, hcp;
    if (nnz > 0) {
        // host copies of the (global) segment pointers for the tile bookkeeping
        hrp.resize(I + 1);
        hcp.resize(J + 1);
        SK(cudaMemcpyAsync(hrp.data(), d.rowptr, sizeof(int64_t) * (I + 1), cudaMemcpyDeviceToHost, st));
        SK(cudaMemcpyAsync(hcp.data(), d.colptr, sizeof(int64_t) * (J + 1), cudaMemcpyDeviceToHost, st));
        SK(cudaStreamSynchronize(st));
        for (int64_t i0 = 0; i0 < I; i0 += kTliTile / 8) {  // nonzeros of one warp's rows (single pass)
            const int64_t span = hrp[i0 + kTliTile / 8 < I ? i0 + kTliTile / 8 : I] - hrp[i0];
            if (span > h->max_warp_span) h->max_warp_span = span;
        }
        int trc = build_tli(h, d.rowptr, hrp.data(), d.col, I, nnz_pad, J, d.tr);
        if (trc == SGTV_OK) trc = build_tli(h, d.colptr, hcp.data(), d.row, J, nnz_pad, I, d.tc);
        if (trc != SGTV_OK) return bail(trc);
    }
    if (h->persistent && (d.tr.fmt == 0 || d.tc.fmt == 0 || h->n_inner != 1))
        return bail(fail(h, SGTV_ERR_ARG, "the persistent iteration needs both tiled forms and n_inner = 1"));
    if (h->single_pass) {
        if (h->persistent) return bail(fail(h, SGTV_ERR_ARG, "the single-pass form has no persistent launch"));
        if (!scatter_fits(h, 0))
            return bail(fail(h, SGTV_ERR_ARG,
                             "the single-pass form needs the tiled row form with room for two staging buffers"));
        ALLOC(h->e_acc, T * J_pad);
        SK(cudaMemsetAsync(h->e_acc, 0, T * J_pad, st));
        ALLOC(d.u, T * J * g.n_dirs);
    }
    if (h->persistent) {
        // start from the fused strided forms until the autotuner picks
        for (int v = 0; v < h->ks->n_fwd; v++)
            if (std::string(h->ks->fwd_name[v]) == "tli_u8") h->v_fwd = v;
        for (int v = 0; v < h->ks->n_back; v++)
            if (std::string(h->ks->back_name[v]) == "tli_u8") h->v_back = v;
    }
    if (h->precision == SGTV_PREC_BF16VAL) {
        convert_values_bf16(fr, p_rval, nnz_pad, st);
        convert_values_bf16(fc, p_cval, nnz_pad, st);
    } else if (h->precision == SGTV_PREC_FP64) {
        convert_values_f64(fr, p_rval, nnz_pad, st);
        convert_values_f64(fc, p_cval, nnz_pad, st);
    }
    if (h->single_pass && nnz > 0) {
        // the bank-dealt row stream of the single-pass scatter (sgtv_sp.cu)
        std::vector<int64_t> srp(I + 1);
        srp[0] = 0;
        for (int64_t i = 0; i < I; i++) srp[i + 1] = srp[i] + ((hrp[i + 1] - hrp[i] + 3) & ~int64_t(3));
        for (int64_t i0 = 0; i0 < I; i0 += kTliTile / 8) {
            const int64_t span = srp[i0 + kTliTile / 8 < I ? i0 + kTliTile / 8 : I] - srp[i0];
            if (span > h->max_sp_span) h->max_sp_span = span;
        }
        const int64_t nsp = srp[I] + 16;
        void *p_srp, *p_sli, *p_sval;
        ALLOC(p_srp, sizeof(int64_t) * (I + 1));
        ALLOC(p_sli, sizeof(uint16_t) * nsp);
        ALLOC(p_sval, V * nsp);
        SK(cudaMemcpyAsync(p_srp, srp.data(), sizeof(int64_t) * (I + 1), cudaMemcpyHostToDevice, st));
        SK(cudaMemsetAsync(p_sli, 0xFF, sizeof(uint16_t) * nsp, st));  // an unwritten slot fails the check
        SK(cudaMemsetAsync(p_sval, 0, V * nsp, st));
        d.sp.rp = static_cast<int64_t *>(p_srp);
        d.sp.lidx = static_cast<uint16_t *>(p_sli);
        d.sp.val = p_sval;
        SK(cudaMemsetAsync(d.flag, 0, sizeof(int), st));
        SK(sp_build(I, d.rowptr, d.tr.lidx, d.rval, int(V), d.sp.rp, d.tr.wlen, d.tr.uoff, d.sp.lidx, d.sp.val,
                    d.flag, sms, st));
        SK(cudaMemcpyAsync(&hflag, d.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        SK(cudaStreamSynchronize(st));
        if (hflag & 32) return bail(fail(h, SGTV_ERR_CUDA, "the single-pass row stream failed its set-up check"));
        d.sp.built = 1;
    }
    // y and r (expanded to one value per measurement unless a single scalar)
    {
        std::vector<double> yd(I), rd(r_scalar ? 1 : I);
        for (int32_t k = 0; k < nscans; k++) {
            for (int64_t i = 0; i < sc[k].I; i++) yd[I_off[k] + i] = sc[k].y[i];
            if (r_scalar) rd[0] = sc[k].b[0];
            else
                for (int64_t i = 0; i < sc[k].I; i++) rd[I_off[k] + i] = sc[k].b[sc[k].b_len == 1 ? 0 : i];
        }
        if (T == sizeof(float)) {
            std::vector<float> yf(yd.begin(), yd.end()), rf(rd.begin(), rd.end());
            SK(cudaMemcpyAsync(p_y, yf.data(), sizeof(float) * yf.size(), cudaMemcpyHostToDevice, st));
            SK(cudaMemcpyAsync(p_r, rf.data(), sizeof(float) * rf.size(), cudaMemcpyHostToDevice, st));
            SK(cudaStreamSynchronize(st));
        } else {
            SK(cudaMemcpyAsync(p_y, yd.data(), sizeof(double) * yd.size(), cudaMemcpyHostToDevice, st));
            SK(cudaMemcpyAsync(p_r, rd.data(), sizeof(double) * rd.size(), cudaMemcpyHostToDevice, st));
            SK(cudaStreamSynchronize(st));
        }
    }
    SK(cudaStreamSynchronize(st));
    if (tmp_r) { dev_free(h, tmp_r); tmp_r = nullptr; }
    if (tmp_c) { dev_free(h, tmp_c); tmp_c = nullptr; }

    // Sensitivity and the initial state per scan (f0 = kappa_k, d0 = w.G f0, c0 = 0).
    h->ks->colsum(d, st);
    SK(cudaGetLastError());
    for (int32_t k = 0; k < nscans; k++) {
        h->ks->sum(d, sc[k].J, static_cast<const char *>(d.s) + T * J_off[k], 0, st);
        SK(cudaGetLastError());
        double ss = 0.0;
        SK(cudaMemcpyAsync(&ss, d.red, sizeof(double), cudaMemcpyDeviceToHost, st));
        SK(cudaStreamSynchronize(st));
        const double syr = sum_y[k] - sum_r[k];
        const double num = syr > 0.0 ? syr : (sum_y[k] > 0.0 ? sum_y[k] : 1.0);
        const double kappa = ss > 0.0 ? num / ss : 0.0;
        h->ks->fill(sc[k].J, static_cast<char *>(d.f) + T * J_off[k], kappa, st);
    }
    h->ks->wgrad(d, g, d.f, d.d, st);
    SK(cudaMemsetAsync(d.c, 0, T * J * g.n_dirs, st));
    SK(copy_d_to_prev(h));
    SK(cudaMemsetAsync(d.flag, 0, sizeof(int) * 4, st));
    SK(cudaGetLastError());
    SK(cudaStreamSynchronize(st));
#undef SK
#undef ALLOC
    if (!(opts.flags & SGTV_FLAG_NO_AUTOTUNE)) {
        int rc2 = sgtv_autotune(h, 10);
        if (rc2 != SGTV_OK) {
            g_setup_error = h->err;
            release(h);
            return rc2;
        }
    }
    *out = h;
    return SGTV_OK;
}

int sgtv_setup(sgtv_t *out, int64_t I, int64_t J, int64_t nnz, const int64_t *csr_rowptr,
               const int32_t *csr_col, const float *csr_val, const int64_t *csc_colptr,
               const int32_t *csc_row, const float *csc_val, int32_t Nx, int32_t Nz, int32_t Nq,
               const float *y, const float *b, int64_t b_len, double lambda, double rho,
               const sgtv_opts *opts)
{
    sgtv_scan one;
    one.I = I;
    one.J = J;
    one.nnz = nnz;
    one.csr_rowptr = csr_rowptr;
    one.csr_col = csr_col;
    one.csr_val = csr_val;
    one.csc_colptr = csc_colptr;
    one.csc_row = csc_row;
    one.csc_val = csc_val;
    one.Nx = Nx;
    one.Nz = Nz;
    one.Nq = Nq;
    one.y = y;
    one.b = b;
    one.b_len = b_len;
    one.lambda = lambda;
    one.rho = rho;
    return setup_impl(out, 1, &one, opts);
}

int sgtv_setup_batch(sgtv_t *out, int32_t nscans, const sgtv_scan *scans, const sgtv_opts *opts)
{
    return setup_impl(out, nscans, scans, opts);
}

int sgtv_batch_info(sgtv_t h, int32_t *nscans, int64_t *vox_off, int64_t *meas_off, int64_t *site_off)
{
    if (!h) return SGTV_ERR_ARG;
    if (nscans) *nscans = h->nscans;
    for (int32_t k = 0; k <= h->nscans; k++) {
        if (vox_off) vox_off[k] = h->J_off[k];
        if (meas_off) meas_off[k] = h->I_off[k];
        if (site_off) site_off[k] = h->S_off[k];
    }
    return SGTV_OK;
}

int sgtv_objective_scan(sgtv_t h, int32_t k, double *phi, double *dev, double *tv)
{
    int rc = sgtv_sync(h);
    if (rc) return rc;
    if (k < 0 || k >= h->nscans) return SGTV_ERR_ARG;  // not sticky
    h->ks->deviance(h->d, h->d.f, h->I_off[k], h->I_off[k + 1], 0, h->stream);
    h->ks->tv(h->d, h->g, h->d.f, nullptr, h->S_off[k], h->S_off[k + 1], 1, h->stream);
    CK(h, cudaGetLastError());
    double r[3];
    if ((rc = read_red(h, r, 3))) return rc;
    if (dev) *dev = r[0];
    if (tv) *tv = r[1];
    if (phi) *phi = r[0] + r[2];
    return SGTV_OK;
}

int sgtv_iterate(sgtv_t h, int32_t n)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (n < 0) return fail(h, SGTV_ERR_ARG, "n must be >= 0");
    int32_t k = 0;
    if (h->use_graph) {
        for (; k + kGraphIters <= n; k += kGraphIters) {
            CK(h, join_shrink(h));
            const int parity = (h->d.f == h->bufA ? 0 : 1) + (h->d.d == h->dbufA ? 0 : 2);
            if (!h->gexec[parity]) CK(h, capture_pair(h, &h->gexec[parity]));
            if (h->prof) {
                ProfRec r{SGTV_K_ITERATION, take_event(h), take_event(h)};
                cudaEventRecord(r.a, h->stream);
                CK(h, cudaGraphLaunch(h->gexec[parity], h->stream));
                cudaEventRecord(r.b, h->stream);
                h->recs.push_back(r);
                for (int m = 1; m < kGraphIters; m++)
                    h->recs.push_back(ProfRec{-1, nullptr, nullptr});  // the graph's other iterations
            } else {
                CK(h, cudaGraphLaunch(h->gexec[parity], h->stream));
            }
        }
    }
    for (; k < n; k++) CK(h, enqueue_iteration(h));
    // every call leaves its work ordered on the handle's stream
    CK(h, join_shrink(h));
    CK(h, cudaGetLastError());
    return SGTV_OK;
}

int sgtv_sync(sgtv_t h)
{
    int rc = check_live(h);
    if (rc) return rc;
    CK(h, join_shrink(h));
    int flag = 0;
    CK(h, cudaMemcpyAsync(&flag, h->d.flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (flag & 2) return fail(h, SGTV_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (flag & 1) return fail(h, SGTV_ERR_NONFINITE, "a NaN or Inf appeared in the iterate");
    return SGTV_OK;
}

int sgtv_objective(sgtv_t h, double *phi, double *dev, double *tv)
{
    int rc = sgtv_sync(h);
    if (rc) return rc;
    h->ks->deviance(h->d, h->d.f, 0, h->d.I, 0, h->stream);
    h->ks->tv(h->d, h->g, h->d.f, nullptr, 0, h->g.S, 1, h->stream);
    CK(h, cudaGetLastError());
    double r[3];
    if ((rc = read_red(h, r, 3))) return rc;
    if (dev) *dev = r[0];
    if (tv) *tv = r[1];
    if (phi) *phi = r[0] + r[2];  // r[2] = sum over scans of beta_k * R_k
    return SGTV_OK;
}

int sgtv_residuals(sgtv_t h, double *primal, double *dual, double *kkt)
{
    int rc = sgtv_sync(h);
    if (rc) return rc;
    Dev &d = h->d;
    h->ks->tv(d, h->g, d.f, d.d, 0, h->g.S, 0, h->stream);  // red[0] = ||wGf - d||^2, red[1] = ||d||^2
    h->ks->fwd[h->v_fwd](d, d.f, d.ratio, h->stream);
    h->ks->backproject(d, d.ratio, d.e, h->stream);
    h->ks->kkt(d, h->g, d.f, 2, h->stream);                  // red[2] = max |min(f, g)|, red[3] = max s
    h->ks->dual_res(d, h->g, 4, h->stream);                  // red[4] = ||rho (wG)^T dd||^2, red[5] = ||rho (wG)^T c||^2
    CK(h, cudaGetLastError());
    double r[6];
    if ((rc = read_red(h, r, 6))) return rc;
    if (primal) *primal = sqrt(r[0]) / fmax(1.0, sqrt(r[1]));
    if (dual) *dual = sqrt(r[4]) / fmax(1.0, sqrt(r[5]));
    if (kkt) *kkt = r[2] / fmax(1.0, r[3]);
    return SGTV_OK;
}

int sgtv_get_image(sgtv_t h, float *out, int64_t len)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (!out || len != h->d.J) return fail(h, SGTV_ERR_ARG, "out must hold exactly J floats");
    if ((rc = sgtv_sync(h))) return rc;
    if (h->ks->elem_size == sizeof(float)) {
        CK(h, cudaMemcpyAsync(out, h->d.f, sizeof(float) * len, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    } else {
        std::vector<double> tmp(len);
        CK(h, cudaMemcpyAsync(tmp.data(), h->d.f, sizeof(double) * len, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        for (int64_t k = 0; k < len; k++) out[k] = float(tmp[k]);
    }
    return SGTV_OK;
}

int sgtv_get_state_f64(sgtv_t h, double *f, double *dsplit, double *c)
{
    int rc = sgtv_sync(h);
    if (rc) return rc;
    const int64_t J = h->d.J, ND = J * h->g.n_dirs;
    const void *src[3] = {h->d.f, h->d.d, h->d.c};
    double *dst[3] = {f, dsplit, c};
    const int64_t n[3] = {J, ND, ND};
    for (int k = 0; k < 3; k++) {
        if (!dst[k]) continue;
        if (h->ks->elem_size == sizeof(double)) {
            CK(h, cudaMemcpyAsync(dst[k], src[k], sizeof(double) * n[k], cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        } else {
            std::vector<float> tmp(n[k]);
            CK(h, cudaMemcpyAsync(tmp.data(), src[k], sizeof(float) * n[k], cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            for (int64_t i = 0; i < n[k]; i++) dst[k][i] = tmp[i];
        }
    }
    return SGTV_OK;
}

int sgtv_set_state_f64(sgtv_t h, const double *f, const double *dsplit, const double *c)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (!f) return fail(h, SGTV_ERR_ARG, "f is NULL");
    if ((dsplit == nullptr) != (c == nullptr)) return fail(h, SGTV_ERR_ARG, "give both d and c, or neither");
    const int64_t J = h->d.J, ND = J * h->g.n_dirs;
    for (int64_t j = 0; j < J; j++)
        if (!finite_nonneg(f[j])) return SGTV_ERR_DOMAIN;  // not sticky: the state is unchanged
    if (dsplit)
        for (int64_t k = 0; k < ND; k++)
            if (!isfinite(dsplit[k]) || !isfinite(c[k])) return SGTV_ERR_DOMAIN;
    if ((rc = sgtv_sync(h))) return rc;
    const double *src[3] = {f, dsplit, c};
    void *dst[3] = {h->d.f, h->d.d, h->d.c};
    const int64_t n[3] = {J, ND, ND};
    for (int k = 0; k < 3; k++) {
        if (!src[k]) continue;
        if (h->ks->elem_size == sizeof(double)) {
            CK(h, cudaMemcpyAsync(dst[k], src[k], sizeof(double) * n[k], cudaMemcpyHostToDevice, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        } else {
            std::vector<float> tmp(src[k], src[k] + n[k]);
            CK(h, cudaMemcpyAsync(dst[k], tmp.data(), sizeof(float) * n[k], cudaMemcpyHostToDevice, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        }
    }
    if (!dsplit) {
        h->ks->wgrad(h->d, h->g, h->d.f, h->d.d, h->stream);
        CK(h, cudaMemsetAsync(h->d.c, 0, size_t(h->ks->elem_size) * ND, h->stream));
        CK(h, cudaGetLastError());
    }
    CK(h, copy_d_to_prev(h));
    CK(h, cudaStreamSynchronize(h->stream));
    return SGTV_OK;
}

int sgtv_set_data(sgtv_t h, const float *y, const float *b, int64_t b_len, double lambda)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (h->nscans != 1) return fail(h, SGTV_ERR_ARG, "sgtv_set_data needs a one-scan handle");
    if (!y || !b) return fail(h, SGTV_ERR_ARG, "y and b are required");
    const int64_t I = h->d.I;
    if (b_len != (h->d.r_scalar ? 1 : I)) return fail(h, SGTV_ERR_ARG, "b_len must match the handle's background");
    if (!(lambda >= 0.0) || !isfinite(lambda)) return SGTV_ERR_DOMAIN;  // not sticky: data unchanged
    double sy = 0.0, sr = 0.0;
    for (int64_t i = 0; i < I; i++) {
        if (!finite_nonneg(y[i])) return SGTV_ERR_DOMAIN;
        sy += y[i];
    }
    for (int64_t i = 0; i < b_len; i++)
        if (!finite_nonneg(b[i])) return SGTV_ERR_DOMAIN;
    for (int64_t i = 0; i < I; i++) sr += b[b_len == 1 ? 0 : i];
    if ((rc = sgtv_sync(h))) return rc;
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    const size_t T = h->ks->elem_size;
    if (T == sizeof(float)) {
        CK(h, cudaMemcpyAsync(const_cast<void *>(d.y), y, sizeof(float) * I, cudaMemcpyHostToDevice, st));
        CK(h, cudaMemcpyAsync(const_cast<void *>(d.r), b, sizeof(float) * b_len, cudaMemcpyHostToDevice, st));
        CK(h, cudaStreamSynchronize(st));
    } else {
        std::vector<double> yd(y, y + I), rd(b, b + b_len);
        CK(h, cudaMemcpyAsync(const_cast<void *>(d.y), yd.data(), sizeof(double) * I, cudaMemcpyHostToDevice, st));
        CK(h, cudaMemcpyAsync(const_cast<void *>(d.r), rd.data(), sizeof(double) * b_len, cudaMemcpyHostToDevice, st));
        CK(h, cudaStreamSynchronize(st));
    }
    h->beta = lambda;
    h->scan_tab[0].beta = lambda;
    h->scan_tab[0].tau = h->scan_tab[0].rho > 0.0 ? lambda / h->scan_tab[0].rho : 0.0;
    h->scan_tab[0].tauf = float(h->scan_tab[0].tau);
    CK(h, cudaMemcpyAsync(const_cast<Scan *>(h->g.scans), h->scan_tab.data(), sizeof(Scan), cudaMemcpyHostToDevice, st));
    // the initialisation rule for the new counts
    h->ks->sum(d, d.J, d.s, 0, st);
    double ss = 0.0;
    CK(h, cudaMemcpyAsync(&ss, d.red, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    const double syr = sy - sr;
    const double num = syr > 0.0 ? syr : (sy > 0.0 ? sy : 1.0);
    h->ks->fill(d.J, d.f, ss > 0.0 ? num / ss : 0.0, st);
    h->ks->wgrad(d, h->g, d.f, d.d, st);
    CK(h, cudaMemsetAsync(d.c, 0, T * d.J * h->g.n_dirs, st));
    CK(h, copy_d_to_prev(h));
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(st));
    return SGTV_OK;
}

int sgtv_normalized_backprojection(sgtv_t h, float *out, int32_t out_on_device)
{
    int rc = sgtv_sync(h);
    if (rc) return rc;
    if (!out) return fail(h, SGTV_ERR_ARG, "out is NULL");
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    h->ks->backproject(d, d.y, d.e, st);  // e = A^T y (scratch)
    float *dst = out;
    void *tmp = nullptr;
    if (!out_on_device) {
        cudaError_t ae;
        tmp = dev_alloc(h, sizeof(float) * d.J, &ae);
        if (!tmp) return cuda_fail(h, ae, "device allocation");
        dst = static_cast<float *>(tmp);
    }
    h->ks->ratio_out(d.J, d.e, d.s, dst, st);
    CK(h, cudaGetLastError());
    if (!out_on_device) {
        CK(h, cudaMemcpyAsync(out, dst, sizeof(float) * d.J, cudaMemcpyDeviceToHost, st));
        CK(h, cudaStreamSynchronize(st));
        dev_free(h, tmp);
    } else {
        CK(h, cudaStreamSynchronize(st));
    }
    return SGTV_OK;
}

int sgtv_warm_start(sgtv_t h, const float *f0, int32_t on_device, double dual_scale)
{
    int rc = sgtv_sync(h);
    if (rc) return rc;
    if (!f0) return fail(h, SGTV_ERR_ARG, "f0 is NULL");
    if (!(dual_scale >= 0.0 && dual_scale <= 1.0)) return fail(h, SGTV_ERR_ARG, "dual_scale must be in [0, 1]");
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    const float *src = f0;
    void *tmp = nullptr;
    if (!on_device) {
        cudaError_t ae;
        tmp = dev_alloc(h, sizeof(float) * d.J, &ae);
        if (!tmp) return cuda_fail(h, ae, "device allocation");
        CK(h, cudaMemcpyAsync(tmp, f0, sizeof(float) * d.J, cudaMemcpyHostToDevice, st));
        src = static_cast<const float *>(tmp);
    }
    h->ks->load_image(d.J, src, d.f, d.flag, st);
    h->ks->wgrad(d, h->g, d.f, d.d, st);
    if (dual_scale > 0.0)
        h->ks->dual_rule(d, h->g, dual_scale, st);
    else
        CK(h, cudaMemsetAsync(d.c, 0, size_t(h->ks->elem_size) * d.J * h->g.n_dirs, st));
    CK(h, copy_d_to_prev(h));
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(st));
    if (tmp) dev_free(h, tmp);
    return sgtv_sync(h);  // a non-finite image is reported here
}

int sgtv_warm_start_dual(sgtv_t h, const float *f0, const float *c0, int32_t on_device)
{
    int rc = sgtv_sync(h);
    if (rc) return rc;
    if (!f0 || !c0) return fail(h, SGTV_ERR_ARG, "f0 or c0 is NULL");
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    const int64_t ND = d.J * h->g.n_dirs;
    const float *sf = f0, *sc = c0;
    void *tmp = nullptr;
    if (!on_device) {
        cudaError_t ae;
        tmp = dev_alloc(h, sizeof(float) * (d.J + ND), &ae);
        if (!tmp) return cuda_fail(h, ae, "device allocation");
        float *tf = static_cast<float *>(tmp);
        CK(h, cudaMemcpyAsync(tf, f0, sizeof(float) * d.J, cudaMemcpyHostToDevice, st));
        CK(h, cudaMemcpyAsync(tf + d.J, c0, sizeof(float) * ND, cudaMemcpyHostToDevice, st));
        sf = tf;
        sc = tf + d.J;
    }
    h->ks->load_image(d.J, sf, d.f, d.flag, st);
    h->ks->wgrad(d, h->g, d.f, d.d, st);
    h->ks->load_vec(ND, sc, d.c, d.flag, st);
    CK(h, copy_d_to_prev(h));
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(st));
    if (tmp) dev_free(h, tmp);
    return sgtv_sync(h);  // a non-finite f0 or c0 is reported here
}

int sgtv_autotune(sgtv_t h, int32_t reps)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (reps < 1) return fail(h, SGTV_ERR_ARG, "reps must be >= 1");
    Dev &d = h->d;
    cudaStream_t st = h->stream;
    cudaEvent_t a, b;
    CK(h, cudaEventCreate(&a));
    CK(h, cudaEventCreate(&b));
    auto time_it = [&](auto &&launch, float *ms) -> cudaError_t {
        launch();  // warm-up (also the first-launch occupancy query)
        cudaError_t e = cudaEventRecord(a, st);
        for (int k = 0; k < reps; k++) launch();
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
        if (e == cudaSuccess) e = cudaGetLastError();
        return e;
    };
    // Only scratch is written (ratio, f_next): the ADMM state is untouched.
    // The single-pass form times only its scatter forms (the two-pass
    // products serve it only for the KKT measure).
    float best = 3.4e38f;
    int best_v = 0;
    for (int v = 0; v < h->ks->n_fwd && !h->single_pass; v++) {
        if (!variant_ok(d.tr, h->ks->fwd_need[v])) continue;
        float ms = 0;
        cudaError_t e = time_it([&] { h->ks->fwd[v](d, d.f, d.ratio, st); }, &ms);
        if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(h, e, "autotune forward"); }
        if (ms < best) { best = ms; best_v = v; }
    }
    h->v_fwd = best_v;
    h->ks->fwd[h->v_fwd](d, d.f, d.ratio, st);
    best = 3.4e38f;
    best_v = 0;
    for (int v = 0; v < h->ks->n_back && !h->single_pass; v++) {
        if (!variant_ok(d.tc, h->ks->back_need[v])) continue;
        float ms = 0;
        cudaError_t e = time_it([&] { h->ks->back[v](d, h->g, d.f, d.f_next, st); }, &ms);
        if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(h, e, "autotune backprojection"); }
        if (ms < best) { best = ms; best_v = v; }
    }
    h->v_back = best_v;
    if (h->single_pass) {
        // the scatter accumulates into e_acc: cleared again after the timing
        float bests = 3.4e38f;
        for (int v = 0; v < h->ks->n_scatter; v++) {
            if (!scatter_fits(h, v)) continue;
            float ms = 0;
            cudaError_t e = time_it([&] { h->ks->scatter[v](d, d.f, h->e_acc, st); }, &ms);
            if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(h, e, "autotune scatter"); }
            if (ms < bests) { bests = ms; h->v_scatter = v; }
        }
        CK(h, cudaMemsetAsync(h->e_acc, 0, size_t(h->ks->elem_size) * ((d.J + 15) & ~int64_t(15)), st));
    }
    if (h->persistent) {
        // time the fused forms (no shrink, image written to scratch) and
        // select the tiled variants they correspond to
        int fv[2] = {-1, -1}, bv[2] = {-1, -1};
        for (int v = 0; v < h->ks->n_fwd; v++) {
            const std::string nm(h->ks->fwd_name[v]);
            if (nm == "tli_u8") fv[0] = v;
            if (nm == "tli_v4x2") fv[1] = v;
        }
        for (int v = 0; v < h->ks->n_back; v++) {
            const std::string nm(h->ks->back_name[v]);
            if (nm == "tli_u8") bv[0] = v;
            if (nm == "tli_v4x2") bv[1] = v;
        }
        float bestp = 3.4e38f;
        for (int pv = 0; pv < h->ks->n_pers; pv++) {
            float ms = 0;
            cudaError_t lerr = cudaSuccess;
            cudaError_t e = time_it([&] { lerr = h->ks->pers[pv](d, h->g, d.f, d.f_next, 0, h->bar, st); }, &ms);
            if (e == cudaSuccess) e = lerr;
            if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(h, e, "autotune persistent"); }
            if (ms < bestp) {
                bestp = ms;
                h->v_pers = pv;
                h->v_fwd = fv[(pv >> 1) & 1];
                h->v_back = bv[pv & 1];
            }
        }
    }
    drop_graphs(h);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    int fl = 0;
    CK(h, cudaMemcpy(&fl, h->d.flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (fl & 2) return fail(h, SGTV_ERR_TIMEOUT, "a bounded device-side wait gave up");
    return SGTV_OK;
}

int sgtv_get_variants(sgtv_t h, int32_t *fwd, int32_t *back)
{
    if (!h) return SGTV_ERR_ARG;
    if (fwd) *fwd = h->v_fwd;
    if (back) *back = h->v_back;
    return SGTV_OK;
}

int sgtv_set_variants(sgtv_t h, int32_t fwd, int32_t back)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (fwd < 0 || fwd >= h->ks->n_fwd || back < 0 || back >= h->ks->n_back)
        return SGTV_ERR_ARG;  // not sticky: the handle keeps its variants
    if (!variant_ok(h->d.tr, h->ks->fwd_need[fwd]) || !variant_ok(h->d.tc, h->ks->back_need[back]))
        return SGTV_ERR_ARG;  // that tiled form was not built for this matrix
    if (h->persistent && pers_index(h, fwd, back) < 0)
        return SGTV_ERR_ARG;  // the persistent kernel fuses only the tli_u8 / tli_v4x2 forms
    if (h->persistent) h->v_pers = (h->v_pers & 4) | pers_index(h, fwd, back);
    h->v_fwd = fwd;
    h->v_back = back;
    drop_graphs(h);
    return SGTV_OK;
}

const char *sgtv_variant_name(sgtv_t h, int32_t kernel, int32_t v)
{
    if (!h) return "";
    if (kernel == SGTV_K_FORWARD && v >= 0 && v < h->ks->n_fwd) return h->ks->fwd_name[v];
    if (kernel == SGTV_K_BACK_UPDATE && v >= 0 && v < h->ks->n_back) return h->ks->back_name[v];
    if (kernel == SGTV_K_SCATTER && v >= 0 && v < h->ks->n_scatter) return h->ks->scatter_name[v];
    return "";
}

int sgtv_variant_count(sgtv_t h, int32_t kernel)
{
    if (!h) return 0;
    if (kernel == SGTV_K_FORWARD) return h->ks->n_fwd;
    if (kernel == SGTV_K_BACK_UPDATE) return h->ks->n_back;
    if (kernel == SGTV_K_SCATTER) return h->ks->n_scatter;
    return 0;
}

int sgtv_get_variant(sgtv_t h, int32_t kernel, int32_t *v)
{
    if (!h || !v) return SGTV_ERR_ARG;
    if (kernel == SGTV_K_FORWARD) *v = h->v_fwd;
    else if (kernel == SGTV_K_BACK_UPDATE) *v = h->v_back;
    else if (kernel == SGTV_K_SCATTER) *v = h->v_scatter;
    else return SGTV_ERR_ARG;
    return SGTV_OK;
}

int sgtv_set_variant(sgtv_t h, int32_t kernel, int32_t v)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (kernel == SGTV_K_FORWARD) return sgtv_set_variants(h, v, h->v_back);
    if (kernel == SGTV_K_BACK_UPDATE) return sgtv_set_variants(h, h->v_fwd, v);
    if (kernel != SGTV_K_SCATTER || v < 0 || v >= h->ks->n_scatter) return SGTV_ERR_ARG;
    if (!h->single_pass || !scatter_fits(h, v)) return SGTV_ERR_ARG;
    h->v_scatter = v;
    drop_graphs(h);
    return SGTV_OK;
}

int sgtv_tli_info(sgtv_t h, int32_t *fmt, int64_t *list_entries, int64_t *window_elems, int64_t *max_stage)
{
    if (!h) return SGTV_ERR_ARG;
    const TliMat *m[2] = {&h->d.tr, &h->d.tc};
    for (int k = 0; k < 2; k++) {
        if (fmt) fmt[k] = m[k]->fmt;
        if (max_stage) max_stage[k] = m[k]->max_stage;
        int64_t nl = 0, nw = 0;
        if (m[k]->fmt != 0 && (list_entries || window_elems)) {
            CK(h, cudaMemcpy(&nl, m[k]->uoff + m[k]->ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost));
            std::vector<int32_t> wl(m[k]->ntiles);
            CK(h, cudaMemcpy(wl.data(), m[k]->wlen, sizeof(int32_t) * m[k]->ntiles, cudaMemcpyDeviceToHost));
            for (int32_t v : wl) nw += v;
        }
        if (list_entries) list_entries[k] = nl;
        if (window_elems) window_elems[k] = nw;
    }
    return SGTV_OK;
}

int sgtv_info(sgtv_t h, int64_t *I, int64_t *J, int64_t *nnz, int32_t *n_dirs, int32_t *precision,
              int64_t *device_bytes)
{
    if (!h) return SGTV_ERR_ARG;
    if (I) *I = h->d.I;
    if (J) *J = h->d.J;
    if (nnz) *nnz = h->d.nnz;
    if (n_dirs) *n_dirs = h->g.n_dirs;
    if (precision) *precision = h->precision;
    if (device_bytes) *device_bytes = h->bytes;
    return SGTV_OK;
}

int sgtv_profile(sgtv_t h, int32_t enable)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (enable) {
        CK(h, cudaStreamSynchronize(h->stream));
        for (auto &r : h->recs) {
            if (r.kernel < 0) continue;
            h->pool.push_back(r.a);
            h->pool.push_back(r.b);
        }
        h->recs.clear();
        for (int k = 0; k < SGTV_K_COUNT; k++) {
            h->prof_ms[k] = 0;
            h->prof_n[k] = 0;
        }
    }
    h->prof = enable != 0;
    return SGTV_OK;
}

int sgtv_profile_read(sgtv_t h, double *ms, int64_t *launches, int32_t n_kernels)
{
    int rc = check_live(h);
    if (rc) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto &r : h->recs) {
        if (r.kernel < 0) {  // second iteration of a graph launch (timed with the first)
            h->prof_n[SGTV_K_ITERATION] += 1;
            continue;
        }
        float t = 0.f;
        CK(h, cudaEventElapsedTime(&t, r.a, r.b));
        h->prof_ms[r.kernel] += t;
        h->prof_n[r.kernel] += 1;
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->recs.clear();
    for (int k = 0; k < n_kernels && k < SGTV_K_COUNT; k++) {
        if (ms) ms[k] = h->prof_ms[k];
        if (launches) launches[k] = h->prof_n[k];
    }
    return SGTV_OK;
}

int sgtv_set_wait_limit(sgtv_t h, int64_t ns)
{
    int rc = check_live(h);
    if (rc) return rc;
    if (ns < 0) return SGTV_ERR_ARG;  // not sticky
    const unsigned long long v = ns == 0 ? 0ull : static_cast<unsigned long long>(ns);
    // after the launches already queued on the stream, before later ones
    CK(h, cudaMemcpyAsync(&h->bar->limit_ns, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return SGTV_OK;
}

int sgtv_set_serial(sgtv_t h, int32_t on)
{
    int rc = check_live(h);
    if (rc) return rc;
    CK(h, join_shrink(h));
    if (on)
        h->flags |= SGTV_FLAG_SERIAL;
    else
        h->flags &= ~SGTV_FLAG_SERIAL;
    drop_graphs(h);
    return SGTV_OK;
}

int sgtv_get_stream(sgtv_t h, void **stream)
{
    if (!h || !stream) return SGTV_ERR_ARG;
    *stream = h->stream;
    return SGTV_OK;
}

int sgtv_destroy(sgtv_t h)
{
    if (!h) return SGTV_OK;
    cudaSetDevice(h->device);
    release(h);
    return SGTV_OK;
}

const char *sgtv_last_error(sgtv_t h)
{
    return h ? h->err.c_str() : g_setup_error.c_str();
}

const char *sgtv_strerror(int code)
{
    switch (code) {
    case SGTV_OK: return "SGTV_OK";
    case SGTV_ERR_ARG: return "SGTV_ERR_ARG";
    case SGTV_ERR_DOMAIN: return "SGTV_ERR_DOMAIN";
    case SGTV_ERR_CUDA: return "SGTV_ERR_CUDA";
    case SGTV_ERR_OOM: return "SGTV_ERR_OOM";
    case SGTV_ERR_STATE: return "SGTV_ERR_STATE";
    case SGTV_ERR_TIMEOUT: return "SGTV_ERR_TIMEOUT";
    case SGTV_ERR_NONFINITE: return "SGTV_ERR_NONFINITE";
    default: return "SGTV_ERR_UNKNOWN";
    }
}

}  // extern "C"
