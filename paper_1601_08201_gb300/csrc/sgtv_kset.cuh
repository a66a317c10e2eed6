// sgtv_kset.cuh -- launchers of one precision (T = vector type, V = type of A's
// values); each kset_*.cu file instantiates one.
#pragma once

#include "sgtv_kernels.cuh"

namespace sgtv {

constexpr int kThreads = 256;

inline int grid_for(int64_t warps_needed, int grid_cap)
{
    int64_t blocks = (warps_needed + (kThreads / 32) - 1) / (kThreads / 32);
    if (blocks < 1) blocks = 1;
    return int(blocks < grid_cap ? blocks : grid_cap);
}

// Resident blocks per SM of a kernel (queried once per instantiation): the
// SpMV grids are sized to fill every SM exactly once and then grid-stride.
template <typename K>
inline int resident_blocks(K kernel)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads, 0) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

// Forward projection variant: SPW rows per warp task, U-deep prefetch, PIPE
// = next row's stream issued before this row's gathers, MINB = blocks per SM
// requested from the register allocator.
template <typename T, typename V, int SPW, int U, bool PIPE, int MINB>
struct Fwd {
    static void launch(const Dev &d, const void *f, void *ratio, cudaStream_t st)
    {
        static const int nb = resident_blocks(k_forward<T, V, SPW, U, PIPE, MINB>);
        const int64_t tasks = (d.I + SPW - 1) / SPW;
        k_forward<T, V, SPW, U, PIPE, MINB><<<grid_for(tasks, nb * d.sm_count), kThreads, 0, st>>>(
            d.I, d.rowptr, d.col, static_cast<const V *>(d.rval), static_cast<const T *>(f),
            static_cast<const T *>(d.r), d.r_scalar, static_cast<const T *>(d.y),
            static_cast<T *>(ratio));
    }
};

template <typename T, typename V, int SPW, int U, bool PIPE, int MINB>
struct Back {
    static void launch(const Dev &d, const Geom &g, const void *f, void *f_new, cudaStream_t st)
    {
        static const int nb = resident_blocks(k_back_update<T, V, SPW, U, PIPE, MINB>);
        const int64_t tasks = (d.J + SPW - 1) / SPW;
        k_back_update<T, V, SPW, U, PIPE, MINB><<<grid_for(tasks, nb * d.sm_count), kThreads, 0, st>>>(
            g, d.colptr, d.row, static_cast<const V *>(d.cval), static_cast<const T *>(d.ratio),
            static_cast<const T *>(d.s), static_cast<const T *>(f), static_cast<const T *>(d.d),
            static_cast<const T *>(d.c), static_cast<T *>(f_new));
    }
};

// Launch a TLI kernel with `smem` bytes of dynamic shared memory, raising the
// kernel's opt-in limit the first time a launch needs more than 48 KB.
template <typename K>
inline void ensure_smem(K kernel, int smem, int &granted)
{
    if (smem > 48 * 1024 && smem > granted) {
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess)
            granted = smem;
    }
}

inline TliTiles tiles_of(const TliMat &m)
{
    return TliTiles{m.lidx, m.uoff, m.uidx, m.wbase, m.wlen};
}

// TLI forward projection: one block per tile of 8 * SPW (= kTliTile) rows.
template <typename T, typename V, int SPW, int U, bool PIPE, int UV = 0, int MINB = 1, bool L2PF = false>
struct FwdTli {
    static_assert(8 * SPW == kTliTile, "tile = 8 warps x SPW rows");
    static void launch(const Dev &d, const void *f, void *ratio, cudaStream_t st)
    {
        static int granted = 48 * 1024;
        auto kern = k_forward_tli<T, V, SPW, U, PIPE, UV, MINB, L2PF>;
        const int smem = d.tr.max_stage * int(sizeof(T));
        ensure_smem(kern, smem, granted);
        kern<<<unsigned(d.tr.ntiles), kThreads, smem, st>>>(
            d.I, d.rowptr, tiles_of(d.tr), static_cast<const V *>(d.rval), static_cast<const T *>(f),
            static_cast<const T *>(d.r), d.r_scalar, static_cast<const T *>(d.y), static_cast<T *>(ratio),
            d.flag);
    }
};

template <typename T, typename V, int SPW, int U, bool PIPE, int UV = 0, int MINB = 1, bool L2PF = false>
struct BackTli {
    static_assert(8 * SPW == kTliTile, "tile = 8 warps x SPW columns");
    static void launch(const Dev &d, const Geom &g, const void *f, void *f_new, cudaStream_t st)
    {
        static int granted = 48 * 1024;
        auto kern = k_back_update_tli<T, V, SPW, U, PIPE, UV, MINB, L2PF>;
        if (MINB > 1) {  // several large staged windows per SM: all on-chip memory as shared memory
            static const bool carved =
                cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess;
            (void)carved;
        }
        const int smem = d.tc.max_stage * int(sizeof(T));
        ensure_smem(kern, smem, granted);
        kern<<<unsigned(d.tc.ntiles), kThreads, smem, st>>>(
            g, d.colptr, tiles_of(d.tc), static_cast<const V *>(d.cval), static_cast<const T *>(d.ratio),
            static_cast<const T *>(d.s), static_cast<const T *>(f), static_cast<const T *>(d.d),
            static_cast<const T *>(d.c), static_cast<T *>(f_new), d.flag);
    }
};

// Single-pass forward + scatter: one block per tile of 8 * SPW rows, the
// staged f and the scatter accumulator side by side in shared memory.
template <typename T, typename V, int SPW, int U, bool PRIV, bool KEEP, int MINB>
struct Scatter {
    static_assert(8 * SPW == kTliTile, "tile = 8 warps x SPW rows");
    static constexpr int kBufs = PRIV ? 9 : 2;
    static void launch(const Dev &d, const void *f, void *e, cudaStream_t st)
    {
        static int granted = 48 * 1024;
        auto kern = k_project_scatter_tli<T, V, SPW, U, PRIV, KEEP, MINB>;
        // all of the SM's on-chip memory as shared memory: the gathers and the
        // scatter hit shared memory and the stream bypasses L1, so the
        // carve-out decides how many blocks fit
        static const bool carved =
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess;
        (void)carved;
        const int cap = (d.tr.max_stage + 1) & ~1;
        const int smem = kBufs * cap * int(sizeof(T));
        ensure_smem(kern, smem, granted);
        kern<<<unsigned(d.tr.ntiles), kThreads, smem, st>>>(
            d.I, d.J, d.rowptr, tiles_of(d.tr), static_cast<const V *>(d.rval), static_cast<const T *>(f),
            static_cast<const T *>(d.r), d.r_scalar, static_cast<const T *>(d.y), cap, static_cast<T *>(e),
            d.flag);
    }
};

// 4-wide single-pass scatter (same shared-memory layout as Scatter).
template <typename T, typename V, int SPW, int UV, bool PRIV, int MINB, bool L2PF = false>
struct ScatterV4 {
    static_assert(8 * SPW == kTliTile, "tile = 8 warps x SPW rows");
    static void launch(const Dev &d, const void *f, void *e, cudaStream_t st)
    {
        static int granted = 48 * 1024;
        auto kern = k_project_scatter_tli_v4<T, V, SPW, UV, PRIV, MINB, L2PF>;
        static const bool carved =
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess;
        (void)carved;
        const int cap = (d.tr.max_stage + 1) & ~1;
        const int smem = (PRIV ? 9 : 2) * cap * int(sizeof(T));
        ensure_smem(kern, smem, granted);
        kern<<<unsigned(d.tr.ntiles), kThreads, smem, st>>>(
            d.I, d.J, d.rowptr, tiles_of(d.tr), static_cast<const V *>(d.rval), static_cast<const T *>(f),
            static_cast<const T *>(d.r), d.r_scalar, static_cast<const T *>(d.y), cap, static_cast<T *>(e),
            d.flag);
    }
};

// Single-pass scatter over the bank-dealt row stream (Dev::sp): staged f and
// one accumulator per warp in shared memory.
template <typename T, typename V, int UV, int MINB, bool L2PF = false, bool PRIV = true, bool PF = true,
          int OPT = 0>
struct ScatterSp {
    static constexpr int kBufs = PRIV ? 9 : 2;
    static void launch(const Dev &d, const void *f, void *e, cudaStream_t st)
    {
        static int granted = 48 * 1024;
        auto kern = k_scatter_sp<T, V, UV, MINB, L2PF, PRIV, PF, OPT>;
        static const bool carved =
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess;
        (void)carved;
        const int cap = (d.tr.max_stage + 2) & ~1;  // the staging buffer and its dummy slot
        const int smem = kBufs * cap * int(sizeof(T));
        ensure_smem(kern, smem, granted);
        kern<<<unsigned(d.tr.ntiles), kThreads, smem, st>>>(
            d.I, d.J, d.sp.rp, d.sp.lidx, static_cast<const V *>(d.sp.val), tiles_of(d.tr),
            static_cast<const T *>(f), static_cast<const T *>(d.r), d.r_scalar, static_cast<const T *>(d.y), cap,
            static_cast<T *>(e), d.flag);
    }
};

inline TmaMat tma_mat(const TliMat &m, const int64_t *ptr, int64_t nseg)
{
    return TmaMat{ptr, m.lidx, m.wbase, m.wlen, m.uoff, m.uidx, nseg, m.ntiles};
}

inline TmaLayout tma_layout(const TliMat &m)
{
    return TmaLayout{m.tma_off_lidx, m.tma_off_val, m.tma_off_uidx, m.tma_off_xs, m.tma_stage_bytes};
}

// Persistent grid of a TMA-pipeline kernel: resident CTAs (at this shared
// memory size) on every SM, at most one per tile.
template <typename K>
inline int tma_grid(K kernel, int threads, int smem, int sm_count, int64_t ntiles, int &granted, int &cached_smem,
                    int &cached_nb)
{
    ensure_smem(kernel, smem, granted);
    if (cached_smem != smem) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) nb = 1;
        cached_nb = nb;
        cached_smem = smem;
    }
    const int64_t g = int64_t(cached_nb) * sm_count;
    return int(g < ntiles ? g : (ntiles > 0 ? ntiles : 1));
}

template <typename T, typename V, int NS, int NW>
struct FwdTma {
    static void launch(const Dev &d, const void *f, void *ratio, cudaStream_t st)
    {
        static int granted = 48 * 1024, cs = -1, nb = 1;
        auto kern = k_forward_tma<T, V, NS, NW>;
        const int smem = NS * d.tr.tma_stage_bytes;
        const int grid = tma_grid(kern, 32 * (NW + 1), smem, d.sm_count, d.tr.ntiles, granted, cs, nb);
        kern<<<grid, 32 * (NW + 1), smem, st>>>(tma_mat(d.tr, d.rowptr, d.I), tma_layout(d.tr),
                                            static_cast<const V *>(d.rval), static_cast<const T *>(f),
                                            static_cast<const T *>(d.r), d.r_scalar, static_cast<const T *>(d.y),
                                            static_cast<T *>(ratio), d.flag);
    }
};

template <typename T, typename V, int NS, int NW>
struct BackTma {
    static void launch(const Dev &d, const Geom &g, const void *f, void *f_new, cudaStream_t st)
    {
        static int granted = 48 * 1024, cs = -1, nb = 1;
        auto kern = k_back_update_tma<T, V, NS, NW>;
        const int smem = NS * d.tc.tma_stage_bytes;
        const int grid = tma_grid(kern, 32 * (NW + 1), smem, d.sm_count, d.tc.ntiles, granted, cs, nb);
        kern<<<grid, 32 * (NW + 1), smem, st>>>(tma_mat(d.tc, d.colptr, d.J), tma_layout(d.tc), g,
                                            static_cast<const V *>(d.cval), static_cast<const T *>(d.ratio),
                                            static_cast<const T *>(d.s), static_cast<const T *>(f),
                                            static_cast<const T *>(d.d), static_cast<const T *>(d.c),
                                            static_cast<T *>(f_new), d.flag);
    }
};

// Persistent one-launch iteration: a cooperative grid of every block that
// fits (at the staging size of the larger tiled form) on every SM.
template <typename T, typename V, int UVF, int UVB, int MINB>
struct Pers {
    static cudaError_t launch(const Dev &d, const Geom &g, const void *f, void *f_new, int do_shrink, GridBar *bar,
                              cudaStream_t st)
    {
        static int granted = 48 * 1024, cached_smem = -1, nb = 1;
        auto kern = k_iteration<T, V, UVF, UVB, MINB>;
        const int smem = int(sizeof(T)) * (d.tr.max_stage > d.tc.max_stage ? d.tr.max_stage : d.tc.max_stage);
        ensure_smem(kern, smem, granted);
        if (cached_smem != smem) {
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads, smem) != cudaSuccess || n < 1) n = 1;
            nb = n;
            cached_smem = smem;
        }
        int64_t ntr = d.tr.ntiles, ntc = d.tc.ntiles;
        int64_t want = ntr > ntc ? ntr : ntc;
        const int grid = int(want < int64_t(nb) * d.sm_count ? want : int64_t(nb) * d.sm_count);
        TliTiles tr = tiles_of(d.tr), tc = tiles_of(d.tc);
        int64_t I = d.I;
        const int64_t *rowptr = d.rowptr, *colptr = d.colptr;
        const V *rval = static_cast<const V *>(d.rval), *cval = static_cast<const V *>(d.cval);
        const T *r = static_cast<const T *>(d.r), *y = static_cast<const T *>(d.y), *s = static_cast<const T *>(d.s);
        T *ratio = static_cast<T *>(d.ratio), *cc = static_cast<T *>(d.c);
        const T *dd = static_cast<const T *>(d.d);
        T *dout = static_cast<T *>(d.d_prev);
        const T *fc = static_cast<const T *>(f);
        T *fn = static_cast<T *>(f_new);
        int r_scalar = d.r_scalar;
        Geom gg = g;
        int *flag = d.flag;
        void *args[] = {&I, &rowptr, &tr, &ntr, &rval, &r, &r_scalar, &y, &ratio, &gg, &colptr, &tc, &ntc, &cval,
                        &s, &fc, &fn, &dd, &dout, &cc, &do_shrink, &bar, &flag};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(grid));
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = size_t(smem);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void *>(kern), args);
    }
};

template <typename T, typename V>
struct Impl {
    template <int QPL>
    static void shrink_q(const Dev &d, const Geom &g, const void *f, void *d_out, cudaStream_t st)
    {
        static const int nb = resident_blocks(k_shrink<T, QPL>);
        k_shrink<T, QPL><<<grid_for(g.S, d.sm_count * nb), kThreads, 0, st>>>(
            g, static_cast<const T *>(f), static_cast<T *>(d_out), static_cast<T *>(d.c), d.flag,
            static_cast<T *>(d.u));
    }
    template <int QPL, bool ONE>
    static void shrink_lean(const Dev &d, const Geom &g, const void *f, void *d_out, cudaStream_t st)
    {
        static const int nb = resident_blocks(k_shrink_lean<T, QPL, ONE>);
        k_shrink_lean<T, QPL, ONE><<<grid_for(g.S, d.sm_count * nb), kThreads, 0, st>>>(
            g, static_cast<const T *>(f), static_cast<T *>(d_out), static_cast<T *>(d.c), d.flag,
            static_cast<T *>(d.u));
    }
    template <bool ONE>
    static void shrink_lean_q(const Dev &d, const Geom &g, const void *f, void *d_out, cudaStream_t st)
    {
        if (g.max_nq <= 32) shrink_lean<1, ONE>(d, g, f, d_out, st);
        else if (g.max_nq <= 64) shrink_lean<2, ONE>(d, g, f, d_out, st);
        else shrink_lean<4, ONE>(d, g, f, d_out, st);
    }
    // v kept in registers for Nq up to 128 (the lean form under the group TV,
    // same bits); larger q-ranges sweep twice
    static void shrink(const Dev &d, const Geom &g, const void *f, void *d_out, cudaStream_t st)
    {
        if (!g.per_bin && g.max_nq <= 128) {
            if (g.nscans == 1) shrink_lean_q<true>(d, g, f, d_out, st);
            else shrink_lean_q<false>(d, g, f, d_out, st);
            return;
        }
        if (g.max_nq <= 32) shrink_q<1>(d, g, f, d_out, st);
        else if (g.max_nq <= 64) shrink_q<2>(d, g, f, d_out, st);
        else if (g.max_nq <= 128) shrink_q<4>(d, g, f, d_out, st);
        else shrink_q<0>(d, g, f, d_out, st);
    }
    static void dual_rule(const Dev &d, const Geom &g, double theta, cudaStream_t st)
    {
        k_dual_rule<T><<<grid_for(g.S, d.sm_count * 8), kThreads, 0, st>>>(
            g, static_cast<const T *>(d.d), static_cast<T *>(d.c), theta);
    }
    template <int QB>
    static void fupdate_site(const Dev &d, const Geom &g, void *e, const void *f, void *f_new, cudaStream_t st)
    {
        static const int nb = resident_blocks(k_fupdate_site<T, QB>);
        k_fupdate_site<T, QB><<<grid_for(g.S, d.sm_count * nb), kThreads, 0, st>>>(
            g, static_cast<T *>(e), static_cast<const T *>(d.s), static_cast<const T *>(f),
            static_cast<const T *>(d.u), static_cast<T *>(f_new));
    }
    static void sub(int64_t n, const void *a, const void *b, void *out, cudaStream_t st)
    {
        int blocks = int((n + kThreads - 1) / kThreads);
        blocks = blocks > 4096 ? 4096 : (blocks < 1 ? 1 : blocks);
        k_sub<T><<<blocks, kThreads, 0, st>>>(n, static_cast<const T *>(a), static_cast<const T *>(b),
                                              static_cast<T *>(out));
    }
    static void fupdate(const Dev &d, const Geom &g, void *e, const void *f, void *f_new, cudaStream_t st)
    {
        if (g.max_nq >= 16 && d.u) {  // a warp per site: lanes over q-bins
            if (g.max_nq <= 32) fupdate_site<1>(d, g, e, f, f_new, st);
            else fupdate_site<2>(d, g, e, f, f_new, st);
            return;
        }
        int64_t blocks = (d.J + kThreads - 1) / kThreads;  // one hyper-voxel per thread
        blocks = blocks > (int64_t(1) << 30) ? (int64_t(1) << 30) : (blocks < 1 ? 1 : blocks);
        k_fupdate<T><<<unsigned(blocks), kThreads, 0, st>>>(g, static_cast<T *>(e), static_cast<const T *>(d.s),
                                                  static_cast<const T *>(f), static_cast<const T *>(d.d),
                                                  static_cast<const T *>(d.c), static_cast<T *>(f_new));
    }
    static void backproject(const Dev &d, const void *v, void *out, cudaStream_t st)
    {
        k_backproject<T, V><<<grid_for(d.J, d.sm_count * 8), kThreads, 0, st>>>(
            d.J, d.colptr, d.row, static_cast<const V *>(d.cval), static_cast<const T *>(v),
            static_cast<T *>(out));
    }
    static void colsum(const Dev &d, cudaStream_t st)
    {
        k_colsum<T, V><<<grid_for(d.J, d.sm_count * 8), kThreads, 0, st>>>(
            d.J, d.colptr, static_cast<const V *>(d.cval), static_cast<T *>(d.s));
    }
    static void wgrad(const Dev &d, const Geom &g, const void *f, void *out, cudaStream_t st)
    {
        k_wgrad<T><<<d.sm_count * 4, kThreads, 0, st>>>(g, static_cast<const T *>(f), static_cast<T *>(out));
    }
    static void fill(int64_t n, void *a, double val, cudaStream_t st)
    {
        int blocks = int((n + kThreads - 1) / kThreads);
        if (blocks > 4096) blocks = 4096;
        if (blocks < 1) blocks = 1;
        k_fill<T><<<blocks, kThreads, 0, st>>>(n, static_cast<T *>(a), val);
    }
    static void ratio_out(int64_t n, const void *num, const void *den, float *out, cudaStream_t st)
    {
        int blocks = int((n + kThreads - 1) / kThreads);
        blocks = blocks > 4096 ? 4096 : (blocks < 1 ? 1 : blocks);
        k_ratio_out<T><<<blocks, kThreads, 0, st>>>(n, static_cast<const T *>(num), static_cast<const T *>(den), out);
    }
    static void load_image(int64_t n, const float *src, void *f, int *flag, cudaStream_t st)
    {
        int blocks = int((n + kThreads - 1) / kThreads);
        blocks = blocks > 4096 ? 4096 : (blocks < 1 ? 1 : blocks);
        k_load_image<T><<<blocks, kThreads, 0, st>>>(n, src, static_cast<T *>(f), flag);
    }
    static void load_vec(int64_t n, const float *src, void *a, int *flag, cudaStream_t st)
    {
        int blocks = int((n + kThreads - 1) / kThreads);
        blocks = blocks > 4096 ? 4096 : (blocks < 1 ? 1 : blocks);
        k_load_vec<T><<<blocks, kThreads, 0, st>>>(n, src, static_cast<T *>(a), flag);
    }
    static void sum(const Dev &d, int64_t n, const void *a, int slot, cudaStream_t st)
    {
        k_sum_partials<T><<<d.red_blocks, kThreads, 0, st>>>(n, static_cast<const T *>(a), d.part);
        finalize(d.part, d.red_blocks, 1, 0u, d.red + slot, st);
    }
    static void deviance(const Dev &d, const void *f, int64_t i0, int64_t i1, int slot, cudaStream_t st)
    {
        k_dev_partials<T, V><<<d.red_blocks, kThreads, 0, st>>>(
            i1 - i0, d.rowptr + i0, d.col, static_cast<const V *>(d.rval), static_cast<const T *>(f),
            static_cast<const T *>(d.r) + (d.r_scalar ? 0 : i0), d.r_scalar, static_cast<const T *>(d.y) + i0,
            d.part);
        finalize(d.part, d.red_blocks, 1, 0u, d.red + slot, st);
    }
    static void tv(const Dev &d, const Geom &g, const void *f, const void *dsplit, int64_t s0, int64_t s1, int slot,
                   cudaStream_t st)
    {
        k_tv_partials<T><<<d.red_blocks, kThreads, 0, st>>>(g, static_cast<const T *>(f),
                                                            static_cast<const T *>(dsplit), s0, s1, d.part);
        finalize(d.part, d.red_blocks, 2, 0u, d.red + slot, st);
    }
    static void kkt(const Dev &d, const Geom &g, const void *f, int slot, cudaStream_t st)
    {
        k_kkt_partials<T><<<d.red_blocks, kThreads, 0, st>>>(
            g, static_cast<const T *>(f), static_cast<const T *>(d.e), static_cast<const T *>(d.s),
            static_cast<const T *>(d.c), d.part);
        finalize(d.part, d.red_blocks, 2, 3u, d.red + slot, st);
    }
    static void dual_res(const Dev &d, const Geom &g, int slot, cudaStream_t st)
    {
        k_dual_partials<T><<<d.red_blocks, kThreads, 0, st>>>(
            g, static_cast<const T *>(d.d), static_cast<const T *>(d.d_prev), static_cast<const T *>(d.c), d.part);
        finalize(d.part, d.red_blocks, 2, 0u, d.red + slot, st);
    }
    static KernelSet make()
    {
        KernelSet k{};
        int n = 0;
        k.fwd[n] = Fwd<T, V, 8, 8, false, 8>::launch;  k.fwd_name[n++] = "rows8_u8_min8";
        k.fwd[n] = FwdTli<T, V, kTliTile / 8, 8, false>::launch;  k.fwd_name[n] = "tli_u8"; k.fwd_need[n++] = 1;
        k.fwd[n] = FwdTli<T, V, kTliTile / 8, 8, false, 2>::launch; k.fwd_name[n] = "tli_v4x2"; k.fwd_need[n++] = 1;
        k.fwd[n] = FwdTli<T, V, kTliTile / 8, 8, false, 3>::launch; k.fwd_name[n] = "tli_v4x3"; k.fwd_need[n++] = 1;
        k.fwd[n] = FwdTli<T, V, kTliTile / 8, 8, false, 2, 8>::launch; k.fwd_name[n] = "tli_v4x2_min8";
        k.fwd_need[n++] = 1;
        k.fwd[n] = FwdTli<T, V, kTliTile / 8, 8, false, 3, 6>::launch; k.fwd_name[n] = "tli_v4x3_min6";
        k.fwd_need[n++] = 1;
        // the same forms with the block's tile stream bulk-prefetched into L2 at its start
        k.fwd[n] = FwdTli<T, V, kTliTile / 8, 8, false, 3, 1, true>::launch; k.fwd_name[n] = "tli_v4x3_l2pf";
        k.fwd_need[n++] = 1;
        k.fwd[n] = FwdTli<T, V, kTliTile / 8, 8, false, 2, 8, true>::launch; k.fwd_name[n] = "tli_v4x2_min8_l2pf";
        k.fwd_need[n++] = 1;
        k.fwd[n] = FwdTli<T, V, kTliTile / 8, 8, false, 3, 6, true>::launch; k.fwd_name[n] = "tli_v4x3_min6_l2pf";
        k.fwd_need[n++] = 1;
        k.fwd[n] = FwdTma<T, V, 3, 16>::launch;  k.fwd_name[n] = "tma_ns3_w16"; k.fwd_need[n++] = 3;
        k.fwd[n] = FwdTma<T, V, 3, 8>::launch;   k.fwd_name[n] = "tma_ns3_w8"; k.fwd_need[n++] = 3;
        k.fwd[n] = FwdTma<T, V, 4, 16>::launch;  k.fwd_name[n] = "tma_ns4_w16"; k.fwd_need[n++] = 4;
        k.n_fwd = n;
        n = 0;
        k.back[n] = Back<T, V, 8, 8, false, 8>::launch;  k.back_name[n++] = "cols8_u8_min8";
        k.back[n] = BackTli<T, V, kTliTile / 8, 8, false>::launch;  k.back_name[n] = "tli_u8"; k.back_need[n++] = 1;
        k.back[n] = BackTli<T, V, kTliTile / 8, 8, false, 2>::launch; k.back_name[n] = "tli_v4x2"; k.back_need[n++] = 1;
        k.back[n] = BackTli<T, V, kTliTile / 8, 8, false, 3>::launch; k.back_name[n] = "tli_v4x3"; k.back_need[n++] = 1;
        k.back[n] = BackTli<T, V, kTliTile / 8, 8, false, 0, 6>::launch; k.back_name[n] = "tli_u8_min6";
        k.back_need[n++] = 1;
        k.back[n] = BackTli<T, V, kTliTile / 8, 8, false, 2, 6>::launch; k.back_name[n] = "tli_v4x2_min6";
        k.back_need[n++] = 1;
        k.back[n] = BackTli<T, V, kTliTile / 8, 8, false, 2, 6, true>::launch; k.back_name[n] = "tli_v4x2_min6_l2pf";
        k.back_need[n++] = 1;
        k.back[n] = BackTli<T, V, kTliTile / 8, 8, false, 2, 1, true>::launch; k.back_name[n] = "tli_v4x2_l2pf";
        k.back_need[n++] = 1;
        k.back[n] = BackTli<T, V, kTliTile / 8, 8, false, 0, 6, true>::launch; k.back_name[n] = "tli_u8_min6_l2pf";
        k.back_need[n++] = 1;
        k.back[n] = BackTma<T, V, 3, 16>::launch;  k.back_name[n] = "tma_ns3_w16"; k.back_need[n++] = 3;
        k.back[n] = BackTma<T, V, 3, 8>::launch;   k.back_name[n] = "tma_ns3_w8"; k.back_need[n++] = 3;
        k.back[n] = BackTma<T, V, 4, 16>::launch;  k.back_name[n] = "tma_ns4_w16"; k.back_need[n++] = 4;
        k.n_back = n;
        // index = 4 * (register cap) + 2 * (forward 4-wide) + (back 4-wide)
        k.n_pers = 8;
        k.pers[0] = Pers<T, V, 0, 0, 1>::launch;  k.pers_name[0] = "persistent_tli_u8";
        k.pers[1] = Pers<T, V, 0, 2, 1>::launch;  k.pers_name[1] = "persistent_tli_u8_v4x2";
        k.pers[2] = Pers<T, V, 2, 0, 1>::launch;  k.pers_name[2] = "persistent_tli_v4x2_u8";
        k.pers[3] = Pers<T, V, 2, 2, 1>::launch;  k.pers_name[3] = "persistent_tli_v4x2";
        k.pers[4] = Pers<T, V, 0, 0, 6>::launch;  k.pers_name[4] = "persistent_tli_u8_min6";
        k.pers[5] = Pers<T, V, 0, 2, 6>::launch;  k.pers_name[5] = "persistent_tli_u8_v4x2_min6";
        k.pers[6] = Pers<T, V, 2, 0, 6>::launch;  k.pers_name[6] = "persistent_tli_v4x2_u8_min6";
        k.pers[7] = Pers<T, V, 2, 2, 6>::launch;  k.pers_name[7] = "persistent_tli_v4x2_min6";
        k.shrink = shrink;
        n = 0;
        k.scatter[n] = Scatter<T, V, kTliTile / 8, 8, false, true, 4>::launch;
        k.scatter_name[n] = "tli_u8_atomic_keep"; k.scatter_bufs[n++] = 2;
        k.scatter[n] = Scatter<T, V, kTliTile / 8, 8, true, true, 4>::launch;
        k.scatter_name[n] = "tli_u8_private_keep"; k.scatter_bufs[n++] = 9;
        k.scatter[n] = ScatterV4<T, V, kTliTile / 8, 3, true, 4>::launch;
        k.scatter_name[n] = "tli_v4x3_private_min4"; k.scatter_bufs[n++] = 9;
        k.scatter[n] = ScatterV4<T, V, kTliTile / 8, 2, true, 5>::launch;
        k.scatter_name[n] = "tli_v4x2_private_min5"; k.scatter_bufs[n++] = 9;
        k.scatter[n] = ScatterV4<T, V, kTliTile / 8, 2, true, 5, true>::launch;
        k.scatter_name[n] = "tli_v4x2_private_min5_l2pf"; k.scatter_bufs[n++] = 9;
        k.scatter[n] = ScatterSp<T, V, 3, 3, true>::launch;
        k.scatter_name[n] = "sp_v4x3_min3_l2pf"; k.scatter_sp[n] = 1; k.scatter_bufs[n++] = 9;
        // one block-shared accumulator (2 staging-sized buffers): the form that still fits when the
        // per-warp accumulators do not (large staging, FP64)
        k.scatter[n] = ScatterSp<T, V, 2, 4, false, false>::launch;
        k.scatter_name[n] = "sp_v4x2_atomic_min4"; k.scatter_sp[n] = 1; k.scatter_bufs[n++] = 2;
        // no register prefetch (the L2 prefetch hides the stream's latency): fewer registers, more warps
        k.scatter[n] = ScatterSp<T, V, 2, 5, true, true, false>::launch;
        k.scatter_name[n] = "sp_v4x2_nopf_min5_l2pf"; k.scatter_sp[n] = 1; k.scatter_bufs[n++] = 9;
        k.scatter[n] = ScatterSp<T, V, 3, 4, true, true, false>::launch;
        k.scatter_name[n] = "sp_v4x3_nopf_min4_l2pf"; k.scatter_sp[n] = 1; k.scatter_bufs[n++] = 9;
        // each chunk's accumulator reads ahead of its writes; no zero-fill past a row's end
        k.scatter[n] = ScatterSp<T, V, 2, 5, true, true, false, kSpBatch4 | kSpLean>::launch;
        k.scatter_name[n] = "sp_v4x2_batch_min5_l2pf"; k.scatter_sp[n] = 1; k.scatter_bufs[n++] = 9;
        k.scatter[n] = ScatterSp<T, V, 2, 4, true, true, false, kSpBatch4 | kSpLean>::launch;
        k.scatter_name[n] = "sp_v4x2_batch_min4_l2pf"; k.scatter_sp[n] = 1; k.scatter_bufs[n++] = 9;
        k.scatter[n] = ScatterSp<T, V, 3, 4, true, true, false, kSpBatch4 | kSpLean>::launch;
        k.scatter_name[n] = "sp_v4x3_batch_min4_l2pf"; k.scatter_sp[n] = 1; k.scatter_bufs[n++] = 9;
        k.n_scatter = n;
        k.fupdate = fupdate;
        k.backproject = backproject;
        k.colsum = colsum;
        k.wgrad = wgrad;
        k.dual_rule = dual_rule;
        k.fill = fill;
        k.ratio_out = ratio_out;
        k.load_image = load_image;
        k.load_vec = load_vec;
        k.sum = sum;
        k.deviance = deviance;
        k.tv = tv;
        k.kkt = kkt;
        k.dual_res = dual_res;
        k.sub = sub;
        k.elem_size = sizeof(T);
        k.val_size = sizeof(V);
        return k;
    }
};

}  // namespace sgtv
