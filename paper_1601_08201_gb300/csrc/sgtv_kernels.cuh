// sgtv_kernels.cuh -- sm_103a kernels of one ADMM iteration of spectrally
// grouped TV reconstruction (Sec. III, Eqs. 5-7) and its FP64 reductions.
//
// Three launches per iteration:
//   k_forward      ybar_i = sum_j a_ij f_j + r_i, ratio_i = y_i / ybar_i   (Eq. 1; CSR)
//   k_back_update  e_j = sum_i a_ij ratio_i (CSC) and, in the same warp, the
//                  closed-form hyper-voxel update of Eq. 5 (EM surrogate +
//                  De Pierro split), writing f^{k+1} to a second buffer
//   k_shrink       v = w.G f^{k+1} + c^k, group soft-threshold per spatial bin
//                  (Eq. 6, grouping of Eq. 2), c^{k+1} = v - d^{k+1} (Eq. 7)
//
// Both sparse products are warp-per-row (warp-per-column) streams with
// coalesced, lane-strided index and value loads (see seg_dot) and gathers of
// the dense operand (f or ratio, both L2-resident) through the read-only path.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgtv_internal.h"

namespace sgtv {

// ---------------------------------------------------------------------------------------
// loads

__device__ __forceinline__ double to_f64(float v) { return double(v); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 v) { return double(__bfloat162float(v)); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Dot product of the sparse segment [start, end) of (idx, val) with the dense
// vector x, accumulated in T by one warp; every lane returns its partial.
// Lane k takes elements start + k, start + k + 32, ...: every index and value
// load is one fully coalesced 128-byte (64-byte for BF16) warp access, and one
// gather instruction touches the few cache lines that 32 consecutive nonzeros
// of a row (or column) fall in, instead of one line per lane. U loads of each
// array are issued before the first gather, so a warp keeps 32 * U indices
// and values in flight.
__device__ __forceinline__ int32_t ld_idx(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ int32_t ld_idx(const uint16_t *p)
{
    return int32_t(__ldcs(reinterpret_cast<const unsigned short *>(p)));
}

// The dense operand: global memory through the read-only path, or a
// shared-memory tile (SX = true) staged by the tiled kernels.
template <bool SX, typename T>
__device__ __forceinline__ T ld_x(const T *x, int32_t c)
{
    if (SX) return x[c];
    return __ldg(x + c);
}
__device__ __forceinline__ float ld_val(const float *p) { return __ldcs(p); }
__device__ __forceinline__ double ld_val(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16 *p)
{
    return __uint_as_float(uint32_t(__ldcs(reinterpret_cast<const unsigned short *>(p))) << 16);
}

template <int U, typename T, typename V, typename IdxT = int32_t, bool SX = false>
__device__ __forceinline__ T seg_dot(int64_t start, int64_t end, const IdxT *__restrict__ idx,
                                     const V *__restrict__ val, const T *__restrict__ x, int lane)
{
    T acc = T(0);
    for (int64_t p = start + lane; p < end; p += 32 * U) {
        int32_t c[U];
        T v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int64_t q = p + 32 * u;
            c[u] = 0;
            v[u] = T(0);
            if (q < end) {
                c[u] = ld_idx(idx + q);
                v[u] = T(ld_val(val + q));
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (p + 32 * u < end) acc = fma(v[u], ld_x<SX>(x, c[u]), acc);
    }
    return acc;
}

// Vector form of seg_dot for 16-bit local indices and a shared-memory dense
// operand: lane k loads 4 consecutive indices (8 bytes) and 4 consecutive
// values (16 bytes for FP32) from a 4-aligned position and masks the elements
// outside the segment; UV such 4-element chunks (128 elements per warp each)
// are in flight before the first gather. Each lane still adds its elements
// in increasing position order, but the partition of elements among lanes
// differs from seg_dot's, so the two forms round differently (both are
// deterministic).
__device__ __forceinline__ void ld_idx4(const uint16_t *p, int32_t (&c)[4])
{
    const uint2 u = __ldcs(reinterpret_cast<const uint2 *>(p));
    c[0] = int32_t(u.x & 0xFFFFu);
    c[1] = int32_t(u.x >> 16);
    c[2] = int32_t(u.y & 0xFFFFu);
    c[3] = int32_t(u.y >> 16);
}

__device__ __forceinline__ void ld_val4(const float *p, float (&v)[4])
{
    const float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

__device__ __forceinline__ void ld_val4(const double *p, double (&v)[4])
{
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(p + 2));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ void ld_val4(const __nv_bfloat16 *p, float (&v)[4])
{
    const uint2 u = __ldcs(reinterpret_cast<const uint2 *>(p));
    v[0] = __uint_as_float(u.x << 16);
    v[1] = __uint_as_float(u.x & 0xFFFF0000u);
    v[2] = __uint_as_float(u.y << 16);
    v[3] = __uint_as_float(u.y & 0xFFFF0000u);
}

template <int UV, typename T, typename V>
__device__ __forceinline__ T seg_dot_v4(int64_t start, int64_t end, const uint16_t *__restrict__ idx,
                                        const V *__restrict__ val, const T *xs, int lane)
{
    T acc = T(0);
    for (int64_t p = (start & ~int64_t(3)) + 4 * lane; p < end; p += 128 * UV) {
        int32_t c[UV][4];
        T v[UV][4];
#pragma unroll
        for (int u = 0; u < UV; u++) {
            const int64_t q = p + 128 * u;
            if (q < end) {
                ld_idx4(idx + q, c[u]);
                ld_val4(val + q, v[u]);
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) { c[u][k] = 0; v[u][k] = T(0); }
            }
        }
#pragma unroll
        for (int u = 0; u < UV; u++)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int64_t q = p + 128 * u + k;
                if (q >= start && q < end) acc = fma(v[u][k], xs[c[u][k]], acc);
            }
    }
    return acc;
}

template <int UV, typename T, typename V>
__device__ __forceinline__ T warp_segments_v4(const int64_t *__restrict__ ptr, int64_t seg0, int nseg,
                                              const uint16_t *__restrict__ idx, const V *__restrict__ val,
                                              const T *xs, int lane)
{
    const int64_t bound = (lane <= nseg) ? ptr[seg0 + lane] : 0;
    T mine = T(0);
#pragma unroll 1
    for (int k = 0; k < nseg; k++) {
        const int64_t s = __shfl_sync(0xffffffffu, bound, k);
        const int64_t e = __shfl_sync(0xffffffffu, bound, k + 1);
        const T acc = warp_sum(seg_dot_v4<UV, T, V>(s, e, idx, val, xs, lane));
        if (lane == k) mine = acc;
    }
    return mine;
}

// One warp reduces nseg (<= 31) consecutive segments (rows or columns)
// seg0 .. seg0+nseg-1 and lane k returns segment k's dot product. The segment
// bounds are loaded once, lane-parallel. With PIPE the first 32 * U indices and
// values of segment k+1 are loaded before segment k's gathers, so the warp has
// the next segment's stream in flight while it waits on the current gathers
// and reduction.
template <int U, typename T, typename V, typename IdxT>
__device__ __forceinline__ void load_chunk(int64_t p, int64_t end, const IdxT *__restrict__ idx,
                                           const V *__restrict__ val, int32_t (&c)[U], T (&v)[U])
{
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int64_t q = p + 32 * u;
        c[u] = 0;
        v[u] = T(0);
        if (q < end) {
            c[u] = ld_idx(idx + q);
            v[u] = T(ld_val(val + q));
        }
    }
}

template <int U, typename T, typename V, bool PIPE, typename IdxT = int32_t, bool SX = false>
__device__ __forceinline__ T warp_segments(const int64_t *__restrict__ ptr, int64_t seg0, int nseg,
                                           const IdxT *__restrict__ idx, const V *__restrict__ val,
                                           const T *__restrict__ x, int lane)
{
    const int64_t bound = (lane <= nseg) ? ptr[seg0 + lane] : 0;
    if (!PIPE) {  // one segment at a time, no prefetch
        T mine = T(0);
#pragma unroll 1
        for (int k = 0; k < nseg; k++) {
            const int64_t s = __shfl_sync(0xffffffffu, bound, k);
            const int64_t e = __shfl_sync(0xffffffffu, bound, k + 1);
            const T acc = warp_sum(seg_dot<U, T, V, IdxT, SX>(s, e, idx, val, x, lane));
            if (lane == k) mine = acc;
        }
        return mine;
    }
    int64_t s = __shfl_sync(0xffffffffu, bound, 0);
    int64_t e = __shfl_sync(0xffffffffu, bound, 1);
    int32_t c0[U];
    T v0[U];
    load_chunk<U, T, V, IdxT>(s + lane, e, idx, val, c0, v0);
    T mine = T(0);
#pragma unroll 1
    for (int k = 0; k < nseg; k++) {
        int32_t c1[U];
        T v1[U];
        int64_t s1 = 0, e1 = 0;
        if (k + 1 < nseg) {
            s1 = __shfl_sync(0xffffffffu, bound, k + 1);
            e1 = __shfl_sync(0xffffffffu, bound, k + 2);
            load_chunk<U, T, V, IdxT>(s1 + lane, e1, idx, val, c1, v1);
        } else {
#pragma unroll
            for (int u = 0; u < U; u++) { c1[u] = 0; v1[u] = T(0); }
        }
        T acc = T(0);
        const int64_t p0 = s + lane;
#pragma unroll
        for (int u = 0; u < U; u++)
            if (p0 + 32 * u < e) acc = fma(v0[u], ld_x<SX>(x, c0[u]), acc);
        if (s + 32 * U < e) acc += seg_dot<U, T, V, IdxT, SX>(s + 32 * U, e, idx, val, x, lane);
        acc = warp_sum(acc);
        if (lane == k) mine = acc;
#pragma unroll
        for (int u = 0; u < U; u++) { c0[u] = c1[u]; v0[u] = v1[u]; }
        s = s1;
        e = e1;
    }
    return mine;
}

// Same stream, summing the values only (column sums s = A^T 1).
template <typename T, typename V>
__device__ __forceinline__ T seg_sum(int64_t start, int64_t end, const V *__restrict__ val, int lane)
{
    T acc = T(0);
    for (int64_t p = start + lane; p < end; p += 32) acc += T(ld_val(val + p));
    return acc;
}

// ---------------------------------------------------------------------------------------
// a1: forward projection with the ratio epilogue (Eq. 1; EM surrogate input)

template <typename T, typename V, int RPW, int U, bool PIPE, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_forward(int64_t I, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
          const V *__restrict__ val, const T *__restrict__ f, const T *__restrict__ r,
          int r_scalar, const T *__restrict__ y, T *__restrict__ ratio)
{
    const int lane = threadIdx.x & 31;
    const int64_t ntask = (I + RPW - 1) / RPW;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t t = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; t < ntask; t += nwarps) {
        const int64_t i0 = t * RPW;
        const int n = int(I - i0 < RPW ? I - i0 : RPW);
        const T acc = warp_segments<U, T, V, PIPE>(rowptr, i0, n, col, val, f, lane);
        const int64_t i = i0 + lane;
        if (lane < n) {
            const T yb = acc + (r_scalar ? r[0] : r[i]);
            const T yi = y[i];
            ratio[i] = (yi == T(0)) ? T(0) : yi / yb;
        }
    }
}

// ---------------------------------------------------------------------------------------
// a4: the closed-form hyper-voxel update (Eq. 5)
//
// Separable surrogate of Eq. 5's objective at f (all sums over directions p):
//   EM part (De Pierro's EM surrogate of the Poisson NLL): s_j t - f_j e_j log t
//   quadratic part: each term (a, p) of rho/2 (u_{a,p} - w_p (t_a - t_b))^2 with
//     b = nbr_p(a) inside the domain is split 1/2-1/2 around f, adding rho w^2 to
//     the t^2 coefficient alpha of both a and b and rho w (w (f_a + f_b) +- u)
//     (+ for a, - for b) to the -t coefficient gamma; a ghost term (b outside)
//     adds rho w^2 / 2 to alpha_a and rho w u to gamma_a.
// Voxel j meets the terms (j, p) and the terms (a, p) with a = j - step_p.
// Minimiser on t >= 0: the root of 2 alpha t^2 + (s - gamma) t - f e = 0.
template <typename T>
__device__ __forceinline__ T sgtv_root(T alpha, T B, T E, T s)
{
    if (alpha == T(0)) return (s > T(0)) ? E / s : T(0);
    T disc = sqrt(B * B + T(8) * alpha * E);
    if (B >= T(0)) {
        T den = B + disc;
        return (den > T(0)) ? T(2) * E / den : T(0);
    }
    return (-B + disc) / (T(4) * alpha);
}

// Scan holding hyper-voxel (or site) v: the last k with off[k] <= v.
__device__ __forceinline__ int scan_of(const int64_t *__restrict__ off, int nscans, int64_t v)
{
    int lo = 0, hi = nscans - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Position of hyper-voxel j inside its scan.
struct Loc {
    int32_t Nx, Nz, Nq, x, z;
    double rho, tau, beta;
    float rhof, tauf;
};

// The stencil weight w_p, the penalty rho and the threshold tau as operands
// of type T: FP32 values rounded once on the host (no per-element FP64-to-FP32
// conversion), FP64 values as given.
template <typename T> __device__ __forceinline__ T wgt(const Geom &g, int p);
template <> __device__ __forceinline__ float wgt<float>(const Geom &g, int p) { return g.wf[p]; }
template <> __device__ __forceinline__ double wgt<double>(const Geom &g, int p) { return g.w[p]; }
template <typename T> __device__ __forceinline__ T lrho(const Loc &L);
template <> __device__ __forceinline__ float lrho<float>(const Loc &L) { return L.rhof; }
template <> __device__ __forceinline__ double lrho<double>(const Loc &L) { return L.rho; }
template <typename T> __device__ __forceinline__ T ltau(const Loc &L);
template <> __device__ __forceinline__ float ltau<float>(const Loc &L) { return L.tauf; }
template <> __device__ __forceinline__ double ltau<double>(const Loc &L) { return L.tau; }

__device__ __forceinline__ Loc locate_voxel(const Geom &g, int64_t j)
{
    const Scan &sc = g.scans[scan_of(g.vox_off, g.nscans, j)];
    Loc L;
    L.Nx = sc.Nx;
    L.Nz = sc.Nz;
    L.Nq = sc.Nq;
    // J < 2^31 (checked at set-up): 32-bit unsigned divisions are exact
    const uint32_t site = uint32_t(j - sc.vox0) / uint32_t(sc.Nq);
    L.x = int32_t(site / uint32_t(sc.Nz));
    L.z = int32_t(site - uint32_t(L.x) * uint32_t(sc.Nz));
    L.rho = sc.rho;
    L.tau = sc.tau;
    L.beta = sc.beta;
    L.rhof = sc.rhof;
    L.tauf = sc.tauf;
    return L;
}

__device__ __forceinline__ bool inside(const Loc &L, int32_t x, int32_t z)
{
    return x >= 0 && x < L.Nx && z >= 0 && z < L.Nz;
}

__device__ __forceinline__ int64_t step_of(const Geom &g, const Loc &L, int p)
{
    return (int64_t(g.dx[p]) * L.Nz + g.dz[p]) * L.Nq;
}

// PRE = false: each direction's neighbour loads sit behind its inside test
// (inside the fused backprojection this is the faster form); PRE = true: every
// load first, a neighbour outside the scan reading the voxel itself (unused),
// so a stand-alone elementwise pass has them all in flight together. Both
// forms do the same arithmetic in the same order.
template <typename T, bool PRE = false>
__device__ __forceinline__ T voxel_update_at(const Geom &g, const Loc &L, int64_t j, T e, const T *__restrict__ s,
                                             const T *__restrict__ f, const T *__restrict__ d,
                                             const T *__restrict__ c)
{
    const T fj = f[j];
    T alpha = T(0), gamma = T(0);
    if (!PRE) {
#pragma unroll
        for (int p = 0; p < 4; p++) {
            if (p >= g.n_dirs) break;
            const int dx = g.dx[p], dz = g.dz[p];
            const T w = wgt<T>(g, p);
            const T w2 = w * w;
            const int64_t step = step_of(g, L, p);
            const int64_t pj = int64_t(p) * g.J + j;
            const T u_jp = d[pj] - c[pj];
            if (inside(L, L.x + dx, L.z + dz)) {
                alpha += w2;
                gamma += w * (w * (fj + f[j + step]) + u_jp);
            } else {
                alpha += T(0.5) * w2;
                gamma += w * u_jp;
            }
            if (inside(L, L.x - dx, L.z - dz)) {
                const T u_ap = d[pj - step] - c[pj - step];
                alpha += w2;
                gamma += w * (w * (f[j - step] + fj) - u_ap);
            }
        }
    } else {
        T fF[4], fB[4], uF[4], uB[4];
        bool inF[4], inB[4];
#pragma unroll
        for (int p = 0; p < 4; p++) {
            fF[p] = fB[p] = uF[p] = uB[p] = T(0);
            inF[p] = inB[p] = false;
            if (p < g.n_dirs) {
                const int64_t step = step_of(g, L, p);
                const int64_t pj = int64_t(p) * g.J + j;
                inF[p] = inside(L, L.x + g.dx[p], L.z + g.dz[p]);
                inB[p] = inside(L, L.x - g.dx[p], L.z - g.dz[p]);
                const int64_t sf = inF[p] ? step : 0, sb = inB[p] ? step : 0;
                fF[p] = f[j + sf];
                fB[p] = f[j - sb];
                uF[p] = d[pj] - c[pj];
                uB[p] = d[pj - sb] - c[pj - sb];
            }
        }
#pragma unroll
        for (int p = 0; p < 4; p++) {
            if (p >= g.n_dirs) break;
            const T w = wgt<T>(g, p);
            const T w2 = w * w;
            if (inF[p]) {
                alpha += w2;
                gamma += w * (w * (fj + fF[p]) + uF[p]);
            } else {
                alpha += T(0.5) * w2;
                gamma += w * uF[p];
            }
            if (inB[p]) {
                alpha += w2;
                gamma += w * (w * (fB[p] + fj) - uB[p]);
            }
        }
    }
    const T rho = lrho<T>(L);
    alpha *= rho;
    gamma *= rho;
    const T sj = s[j];
    return sgtv_root<T>(alpha, sj - gamma, fj * e, sj);
}

template <typename T, bool PRE = false>
__device__ __forceinline__ T voxel_update(const Geom &g, int64_t j, T e, const T *__restrict__ s,
                                          const T *__restrict__ f, const T *__restrict__ d,
                                          const T *__restrict__ c)
{
    return voxel_update_at<T, PRE>(g, locate_voxel(g, j), j, e, s, f, d, c);
}

// a2 + a4: backprojection fused with the f-update. One warp owns CPW
// consecutive columns: it reduces each column's dot product in turn (lane k
// keeps column k's e, see warp_segments), then CPW lanes update their
// hyper-voxels side by side, so the epilogue's loads are coalesced across
// neighbouring q-bins.
template <typename T, typename V, int CPW, int U, bool PIPE, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_back_update(Geom g, const int64_t *__restrict__ colptr, const int32_t *__restrict__ row,
              const V *__restrict__ val, const T *__restrict__ ratio, const T *__restrict__ s,
              const T *__restrict__ f, const T *__restrict__ d, const T *__restrict__ c,
              T *__restrict__ f_new)
{
    const int lane = threadIdx.x & 31;
    const int64_t ntask = (g.J + CPW - 1) / CPW;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t t = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; t < ntask; t += nwarps) {
        const int64_t j0 = t * CPW;
        const int n = int(g.J - j0 < CPW ? g.J - j0 : CPW);
        const T my_e = warp_segments<U, T, V, PIPE>(colptr, j0, n, row, val, ratio, lane);
        const int64_t j = j0 + lane;
        if (lane < n) f_new[j] = voxel_update<T>(g, j, my_e, s, f, d, c);
    }
}

// Backprojection alone: out = A^T v (used by the KKT measure).
template <typename T, typename V>
__global__ void __launch_bounds__(256)
k_backproject(int64_t J, const int64_t *__restrict__ colptr, const int32_t *__restrict__ row,
              const V *__restrict__ val, const T *__restrict__ v, T *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; j < J; j += nwarps) {
        T acc = warp_sum(seg_dot<8, T, V>(colptr[j], colptr[j + 1], row, val, v, lane));
        if (lane == 0) out[j] = acc;
    }
}

// s_j = sum_i a_ij.
template <typename T, typename V>
__global__ void __launch_bounds__(256)
k_colsum(int64_t J, const int64_t *__restrict__ colptr, const V *__restrict__ val, T *__restrict__ s)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; j < J; j += nwarps) {
        T acc = warp_sum(seg_sum<T, V>(colptr[j], colptr[j + 1], val, lane));
        if (lane == 0) s[j] = acc;
    }
}

// ---------------------------------------------------------------------------------------
// a5 + a6: group shrink (Eq. 6) and dual update (Eq. 7), one warp per spatial bin.

template <typename T>
__device__ __forceinline__ double wgrad_at_f64(const Geom &g, const Loc &L, const T *__restrict__ f, int64_t j,
                                               int p)
{
    const bool in = inside(L, L.x + g.dx[p], L.z + g.dz[p]);
    return g.w[p] * (double(f[j]) - (in ? double(f[j + step_of(g, L, p)]) : 0.0));
}

template <typename T>
__device__ __forceinline__ T wgrad_at(const Geom &g, const Loc &L, const T *__restrict__ f, int64_t j, int p)
{
    const bool in = inside(L, L.x + g.dx[p], L.z + g.dz[p]);
    return wgt<T>(g, p) * (f[j] - (in ? f[j + step_of(g, L, p)] : T(0)));
}

// Site `site` (global) of its scan: geometry plus its first hyper-voxel.
__device__ __forceinline__ Loc locate_site(const Geom &g, int64_t site, int64_t &vox)
{
    const Scan &sc = g.scans[scan_of(g.site_off, g.nscans, site)];
    const int64_t ls = site - sc.site0;
    Loc L;
    L.Nx = sc.Nx;
    L.Nz = sc.Nz;
    L.Nq = sc.Nq;
    L.x = int32_t(uint32_t(ls) / uint32_t(sc.Nz));  // S < 2^31: exact in 32 bits
    L.z = int32_t(uint32_t(ls) - uint32_t(L.x) * uint32_t(sc.Nz));
    L.rho = sc.rho;
    L.tau = sc.tau;
    L.beta = sc.beta;
    L.rhof = sc.rhof;
    L.tauf = sc.tauf;
    vox = sc.vox0 + ls * sc.Nq;
    return L;
}

// Eqs. 6-7 for one spatial site, by one warp. QPL > 0: a site of at most
// 32 QPL q-bins keeps v = w.G f + c in registers between the group norm and
// the writes of d and c (the same arithmetic in the same order as the
// two-sweep form that recomputes v).
template <typename T, int QPL = 0>
__device__ __forceinline__ void shrink_site(const Geom &g, const T *__restrict__ f, T *__restrict__ d,
                                            T *__restrict__ c, int64_t site, int lane, int *__restrict__ flag,
                                            T *__restrict__ u = nullptr)
{
    int64_t v0;
    const Loc L = locate_site(g, site, v0);
    const T tau = ltau<T>(L);
    if (g.per_bin) {  // standard TV: each lane shrinks its own (site, q) groups over p
        for (int q = lane; q < L.Nq; q += 32) {
            const int64_t j = v0 + q;
            T v[4];
            T m2 = T(0);
#pragma unroll
            for (int p = 0; p < 4; p++) {
                v[p] = T(0);
                if (p < g.n_dirs) {
                    v[p] = wgrad_at(g, L, f, j, p) + c[int64_t(p) * g.J + j];
                    m2 = fma(v[p], v[p], m2);
                }
            }
            const T m = sqrt(m2);
            if (!isfinite(m)) atomicOr(flag, 1);
            T sc = (m > T(0)) ? T(1) - tau / m : T(0);
            sc = sc > T(0) ? sc : T(0);
#pragma unroll
            for (int p = 0; p < 4; p++) {
                if (p >= g.n_dirs) break;
                const int64_t pj = int64_t(p) * g.J + j;
                const T dv = sc * v[p];
                const T cv = v[p] - dv;
                d[pj] = dv;
                c[pj] = cv;
                if (u) u[pj] = dv - cv;
            }
        }
        return;
    }
    if (QPL > 0 && L.Nq <= 32 * QPL) {  // v stays in registers between the norm and the writes
        constexpr int QR = QPL > 0 ? QPL : 1;
        T v[QR][4];
        T n2 = T(0);
#pragma unroll
        for (int qq = 0; qq < QR; qq++) {
            const int q = lane + 32 * qq;
#pragma unroll
            for (int p = 0; p < 4; p++) {
                v[qq][p] = T(0);
                if (q < L.Nq && p < g.n_dirs) {
                    const int64_t j = v0 + q;
                    v[qq][p] = wgrad_at(g, L, f, j, p) + c[int64_t(p) * g.J + j];
                    n2 = fma(v[qq][p], v[qq][p], n2);
                }
            }
        }
        n2 = warp_sum(n2);
        const T n = sqrt(n2);
        if (!isfinite(n)) {
            if (lane == 0) atomicOr(flag, 1);
        }
        T scale = (n > T(0)) ? T(1) - tau / n : T(0);
        scale = scale > T(0) ? scale : T(0);
#pragma unroll
        for (int qq = 0; qq < QR; qq++) {
            const int q = lane + 32 * qq;
#pragma unroll
            for (int p = 0; p < 4; p++) {
                if (q < L.Nq && p < g.n_dirs) {
                    const int64_t pj = int64_t(p) * g.J + v0 + q;
                    const T dv = scale * v[qq][p];
                    const T cv = v[qq][p] - dv;
                    d[pj] = dv;
                    c[pj] = cv;
                    if (u) u[pj] = dv - cv;
                }
            }
        }
        return;
    }
    T n2 = T(0);
    for (int q = lane; q < L.Nq; q += 32) {
        const int64_t j = v0 + q;
#pragma unroll
        for (int p = 0; p < 4; p++) {
            if (p >= g.n_dirs) break;
            T v = wgrad_at(g, L, f, j, p) + c[int64_t(p) * g.J + j];
            n2 = fma(v, v, n2);
        }
    }
    n2 = warp_sum(n2);
    const T n = sqrt(n2);
    if (!isfinite(n)) {
        if (lane == 0) atomicOr(flag, 1);
    }
    T scale = (n > T(0)) ? T(1) - tau / n : T(0);
    scale = scale > T(0) ? scale : T(0);
    for (int q = lane; q < L.Nq; q += 32) {
        const int64_t j = v0 + q;
#pragma unroll
        for (int p = 0; p < 4; p++) {
            if (p >= g.n_dirs) break;
            const int64_t pj = int64_t(p) * g.J + j;
            T v = wgrad_at(g, L, f, j, p) + c[pj];
            T dv = scale * v;
            const T cv = v - dv;
            d[pj] = dv;
            c[pj] = cv;
            if (u) u[pj] = dv - cv;
        }
    }
}

// d is double-buffered: the shrink writes d^{k+1} into d_out (the buffer that
// held d^{k-1}) and leaves d^k in place for the dual residual.
template <typename T, int QPL>
__global__ void __launch_bounds__(256)
k_shrink(Geom g, const T *__restrict__ f, T *__restrict__ d_out, T *__restrict__ c, int *__restrict__ flag,
         T *__restrict__ u)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t site = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; site < g.S; site += nwarps)
        shrink_site<T, QPL>(g, f, d_out, c, site, lane, flag, u);
}

// Eqs. 6-7 under the group TV (Nq <= 32 QPL): the arithmetic of
// shrink_site's register form in the same order, hence the same bits, with
// less around it. ONE (a one-scan problem): the scan's shape, the direction
// offsets and the threshold are read once per thread, with no scan-table
// lookup. Otherwise (a batch) each site looks up its scan once. Either way a
// site's neighbour tests are made once per site, not per q-bin, and every
// operand of the site (f, its in-scan neighbours, c) is loaded before the
// first product, so each warp has all of them in flight together.
template <typename T, int QPL, bool ONE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (QPL >= 4 ? 3 : 4) : 1)  // FP32: 80 / 64 registers
k_shrink_lean(Geom g, const T *__restrict__ f, T *__restrict__ d_out, T *__restrict__ c, int *__restrict__ flag,
              T *__restrict__ u)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int64_t J = g.J;
    struct Shape {
        int32_t Nx, Nz, Nq;
        int64_t vox0, site0;
        T tau;
        int32_t step[4];
    };
    auto shape_of = [&](int sidx) {
        const Scan &sc = g.scans[sidx];
        Shape sh;
        sh.Nx = sc.Nx;
        sh.Nz = sc.Nz;
        sh.Nq = sc.Nq;
        sh.vox0 = sc.vox0;
        sh.site0 = sc.site0;
        Loc L0;
        L0.tau = sc.tau;
        L0.tauf = sc.tauf;
        sh.tau = ltau<T>(L0);
#pragma unroll
        for (int p = 0; p < 4; p++) sh.step[p] = (g.dx[p] * sh.Nz + g.dz[p]) * sh.Nq;  // |step| < J < 2^31
        return sh;
    };
    Shape one;
    if (ONE) one = shape_of(0);
    for (int64_t site = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; site < g.S; site += nwarps) {
        const Shape sh = ONE ? one : shape_of(scan_of(g.site_off, g.nscans, site));
        // S < 2^31 (checked at set-up): 32-bit unsigned divisions are exact
        const uint32_t ls = uint32_t(site - sh.site0);
        const int32_t x = int32_t(ls / uint32_t(sh.Nz));
        const int32_t z = int32_t(ls - uint32_t(x) * uint32_t(sh.Nz));
        const int64_t v0 = sh.vox0 + int64_t(ls) * sh.Nq;
        bool in[4];
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const int32_t xn = x + g.dx[p], zn = z + g.dz[p];
            in[p] = p < g.n_dirs && xn >= 0 && xn < sh.Nx && zn >= 0 && zn < sh.Nz;
        }
        T fj[QPL], fn[QPL][4], cj[QPL][4];
#pragma unroll
        for (int qq = 0; qq < QPL; qq++) {
            const int q = lane + 32 * qq;
            const int64_t j = v0 + q;
            if (q < sh.Nq) {
                fj[qq] = f[j];
#pragma unroll
                for (int p = 0; p < 4; p++) {
                    if (p < g.n_dirs) {
                        fn[qq][p] = in[p] ? f[j + sh.step[p]] : T(0);
                        cj[qq][p] = c[int64_t(p) * J + j];
                    }
                }
            }
        }
        T v[QPL][4];
        T n2 = T(0);
#pragma unroll
        for (int qq = 0; qq < QPL; qq++) {
            const int q = lane + 32 * qq;
#pragma unroll
            for (int p = 0; p < 4; p++) {
                v[qq][p] = T(0);
                if (q < sh.Nq && p < g.n_dirs) {
                    v[qq][p] = wgt<T>(g, p) * (fj[qq] - fn[qq][p]) + cj[qq][p];
                    n2 = fma(v[qq][p], v[qq][p], n2);
                }
            }
        }
        n2 = warp_sum(n2);
        const T n = sqrt(n2);
        if (!isfinite(n)) {
            if (lane == 0) atomicOr(flag, 1);
        }
        T scale = (n > T(0)) ? T(1) - sh.tau / n : T(0);
        scale = scale > T(0) ? scale : T(0);
#pragma unroll
        for (int qq = 0; qq < QPL; qq++) {
            const int q = lane + 32 * qq;
#pragma unroll
            for (int p = 0; p < 4; p++) {
                if (q < sh.Nq && p < g.n_dirs) {
                    const int64_t pj = int64_t(p) * J + v0 + q;
                    const T dv = scale * v[qq][p];
                    const T cv = v[qq][p] - dv;
                    d_out[pj] = dv;
                    c[pj] = cv;
                    if (u) u[pj] = dv - cv;
                }
            }
        }
    }
}

// out = a - b elementwise (u = d - c after a state set from outside).
template <typename T>
__global__ void k_sub(int64_t n, const T *__restrict__ a, const T *__restrict__ b, T *__restrict__ out)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        out[k] = a[k] - b[k];
}

// Scaled dual consistent with the group shrink (Eq. 6) at a fixed point of
// Eqs. 6-7: there d = w.G f, and v = d + c must shrink back to d, which for a
// group with d_s != 0 forces c_s = tau * d_s / |d_s|; a group with d_s = 0 only
// needs |c_s| <= tau and gets 0. `theta` in [0, 1] scales the rule (0: c = 0).
template <typename T>
__global__ void __launch_bounds__(256)
k_dual_rule(Geom g, const T *__restrict__ d, T *__restrict__ c, double theta)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t site = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; site < g.S; site += nwarps) {
        int64_t v0;
        const Loc L = locate_site(g, site, v0);
        if (g.per_bin) {  // standard TV: groups (site, q)
            for (int q = lane; q < L.Nq; q += 32) {
                double m2 = 0.0;
                for (int p = 0; p < g.n_dirs; p++) {
                    const double v = double(d[int64_t(p) * g.J + v0 + q]);
                    m2 = fma(v, v, m2);
                }
                const double m = sqrt(m2);
                const double k = m > 0.0 ? theta * L.tau / m : 0.0;
                for (int p = 0; p < g.n_dirs; p++) {
                    const int64_t pj = int64_t(p) * g.J + v0 + q;
                    c[pj] = T(k * double(d[pj]));
                }
            }
            continue;
        }
        double n2 = 0.0;
        for (int q = lane; q < L.Nq; q += 32)
            for (int p = 0; p < g.n_dirs; p++) {
                const double v = double(d[int64_t(p) * g.J + v0 + q]);
                n2 = fma(v, v, n2);
            }
        n2 = warp_sum(n2);
        const double n = sqrt(n2);
        const double k = n > 0.0 ? theta * L.tau / n : 0.0;
        for (int q = lane; q < L.Nq; q += 32)
            for (int p = 0; p < g.n_dirs; p++) {
                const int64_t pj = int64_t(p) * g.J + v0 + q;
                c[pj] = T(k * double(d[pj]));
            }
    }
}

// d = w.G f (initial split variable).
template <typename T>
__global__ void k_wgrad(Geom g, const T *__restrict__ f, T *__restrict__ out)
{
    const int64_t n = g.J * g.n_dirs;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int p = int(k / g.J);
        const int64_t j = k - int64_t(p) * g.J;
        const Loc L = locate_voxel(g, j);
        out[k] = wgrad_at(g, L, f, j, p);
    }
}

// out = num / den elementwise (0 where den = 0), as FP32: the normalised
// backprojection A^T y / A^T 1.
template <typename T>
__global__ void k_ratio_out(int64_t n, const T *__restrict__ num, const T *__restrict__ den, float *__restrict__ out)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const T dv = den[k];
        out[k] = dv > T(0) ? float(num[k] / dv) : 0.0f;
    }
}

// f = max(src, 0) from an FP32 image; flags a non-finite value (bit 0).
template <typename T>
__global__ void k_load_image(int64_t n, const float *__restrict__ src, T *__restrict__ f, int *__restrict__ flag)
{
    bool bad = false;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float v = src[k];
        bad |= !isfinite(v);
        f[k] = T(v > 0.0f ? v : 0.0f);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// a = src converted to T; a non-finite value sets flag bit 0.
template <typename T>
__global__ void k_load_vec(int64_t n, const float *__restrict__ src, T *__restrict__ a, int *__restrict__ flag)
{
    bool bad = false;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float v = src[k];
        bad |= !isfinite(v);
        a[k] = T(v);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

template <typename T>
__global__ void k_fill(int64_t n, T *__restrict__ a, double val)
{
    const T v = T(val);
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        a[k] = v;
}

// ---------------------------------------------------------------------------------------
// Tiled local-index (TLI) forms of the two sparse products.
//
// At set-up every tile of 64 consecutive rows (columns) gets 16-bit local
// indices into a per-tile staging buffer (see sgtv_tli.cu), in one of two
// forms chosen per tile:
//   window (wlen[t] > 0): the tile's index window [wbase[t], wbase[t] + wlen[t]),
//                  16-byte aligned; staged by one TMA bulk copy
//                  (cp.async.bulk, completion on an mbarrier)
//   list (wlen[t] == 0): the tile's sorted unique global indices
//                  uidx[uoff[t] .. uoff[t+1]); staged by a gather,
//                  x_s[k] = x[uidx[uoff[t] + k]]
// The stream then carries 2-byte indices instead of 4, and the gathers hit
// shared memory instead of the L1 data pipe.

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return uint32_t(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bulk prefetch into L2 of the bytes [a, b) of an array, widened to 16-byte
// bounds (the arrays are padded past their last element, so the widened
// range stays inside them). A hint only: no register or shared memory holds
// the data, and the later loads of the range hit L2 instead of waiting on
// HBM. One thread issues it for the whole block's tile at the block's start.
__device__ __forceinline__ void prefetch_l2(const void *base, int64_t a, int64_t b)
{
    a &= ~int64_t(15);
    b = (b + 15) & ~int64_t(15);
    if (b <= a) return;
    const char *p = static_cast<const char *>(base) + a;
    // evict-first: the stream is read once, and should not push the
    // iteration's resident vectors (f, d, c, s, e) out of L2
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    while (b > a) {  // one bulk prefetch moves at most 2^31 bytes here
        const int64_t n = (b - a) < (int64_t(1) << 31) ? (b - a) : (int64_t(1) << 31);
        asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(p), "r"(uint32_t(n)),
                     "l"(pol)
                     : "memory");
        p += n;
        a += n;
    }
}

// The index and value streams of segments [s0, s1) (positions ptr[s0] ..
// ptr[s1]) into L2.
template <typename IdxT, typename V>
__device__ __forceinline__ void prefetch_segments_l2(const int64_t *__restrict__ ptr, int64_t s0, int64_t s1,
                                                     const IdxT *idx, const V *val)
{
    const int64_t p0 = ptr[s0], p1 = ptr[s1];
    prefetch_l2(idx, p0 * int64_t(sizeof(IdxT)), p1 * int64_t(sizeof(IdxT)));
    prefetch_l2(val, p0 * int64_t(sizeof(V)), p1 * int64_t(sizeof(V)));
}

// Stage x[base .. base + n) into xs with one bulk copy; every thread returns
// true once the bytes have landed, false if the wait gave up (about 1 s),
// after a second bounded wait for the copy still in flight.
template <typename T>
__device__ __forceinline__ bool stage_window(T *xs, const T *x, int64_t base, int n, uint64_t *mbar)
{
    const uint32_t bar = smem_u32(mbar);
    const uint32_t bytes = uint32_t(n) * uint32_t(sizeof(T));
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (bytes == 0) return true;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(xs)), "l"(x + base), "r"(bytes), "r"(bar) : "memory");
    }
    const uint64_t t0 = global_ns();
    for (int pass = 0; pass < 2; pass++) {
        for (;;) {
            uint32_t done;
            asm volatile("{\n\t.reg .pred p;\n\t"
                         "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done) : "r"(bar) : "memory");
            if (done) return pass == 0;
            if (global_ns() - t0 > (pass == 0 ? 1000000000ull : 2000000000ull)) break;
        }
    }
    return false;
}

template <typename T>
__device__ __forceinline__ bool stage_tile(T *xs, const T *x, int64_t t, const int64_t *__restrict__ uoff,
                                           const int32_t *__restrict__ uidx, const int32_t *__restrict__ wbase,
                                           const int32_t *__restrict__ wlen, uint64_t *mbar)
{
    const int n = wlen[t];
    if (n == 0) {  // list form (block-uniform branch)
        const int64_t u0 = uoff[t];
        const int nu = int(uoff[t + 1] - u0);
        for (int k = threadIdx.x; k < nu; k += blockDim.x) xs[k] = __ldg(x + uidx[u0 + k]);
        __syncthreads();
        return true;
    }
    return stage_window<T>(xs, x, wbase[t], n, mbar);
}

struct TliTiles {
    const uint16_t *lidx;
    const int64_t *uoff;
    const int32_t *uidx;
    const int32_t *wbase;
    const int32_t *wlen;
};

template <typename T, typename V, int RPW, int U, bool PIPE, int UV = 0, int MINB = 1, bool L2PF = false>
__global__ void __launch_bounds__(256, MINB)
k_forward_tli(int64_t I, const int64_t *__restrict__ rowptr, TliTiles tl, const V *__restrict__ val,
              const T *__restrict__ f, const T *__restrict__ r, int r_scalar, const T *__restrict__ y,
              T *__restrict__ ratio, int *__restrict__ flag)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    T *xs = reinterpret_cast<T *>(smem_raw);
    const int64_t t = blockIdx.x;
    if (L2PF && threadIdx.x == 0)
        prefetch_segments_l2(rowptr, t * (8 * RPW), (t + 1) * (8 * RPW) < I ? (t + 1) * (8 * RPW) : I, tl.lidx, val);
    if (!stage_tile<T>(xs, f, t, tl.uoff, tl.uidx, tl.wbase, tl.wlen, &mbar)) {
        if (threadIdx.x == 0) atomicOr(flag, 2);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = t * (8 * RPW) + int64_t(warp) * RPW;
    if (i0 >= I) return;
    const int n = int(I - i0 < RPW ? I - i0 : RPW);
    const T acc = UV > 0 ? warp_segments_v4<(UV > 0 ? UV : 1), T, V>(rowptr, i0, n, tl.lidx, val, xs, lane)
                         : warp_segments<U, T, V, PIPE, uint16_t, true>(rowptr, i0, n, tl.lidx, val, xs, lane);
    const int64_t i = i0 + lane;
    if (lane < n) {
        const T yb = acc + (r_scalar ? r[0] : r[i]);
        const T yi = y[i];
        ratio[i] = (yi == T(0)) ? T(0) : yi / yb;
    }
}

template <typename T, typename V, int CPW, int U, bool PIPE, int UV = 0, int MINB = 1, bool L2PF = false>
__global__ void __launch_bounds__(256, MINB)
k_back_update_tli(Geom g, const int64_t *__restrict__ colptr, TliTiles tl, const V *__restrict__ val,
                  const T *__restrict__ ratio, const T *__restrict__ s, const T *__restrict__ f,
                  const T *__restrict__ d, const T *__restrict__ c, T *__restrict__ f_new,
                  int *__restrict__ flag)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    T *xs = reinterpret_cast<T *>(smem_raw);
    const int64_t t = blockIdx.x;
    if (L2PF && threadIdx.x == 0)
        prefetch_segments_l2(colptr, t * (8 * CPW), (t + 1) * (8 * CPW) < g.J ? (t + 1) * (8 * CPW) : g.J, tl.lidx,
                             val);
    if (!stage_tile<T>(xs, ratio, t, tl.uoff, tl.uidx, tl.wbase, tl.wlen, &mbar)) {
        if (threadIdx.x == 0) atomicOr(flag, 2);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j0 = t * (8 * CPW) + int64_t(warp) * CPW;
    if (j0 >= g.J) return;
    const int n = int(g.J - j0 < CPW ? g.J - j0 : CPW);
    const T my_e = UV > 0 ? warp_segments_v4<(UV > 0 ? UV : 1), T, V>(colptr, j0, n, tl.lidx, val, xs, lane)
                          : warp_segments<U, T, V, PIPE, uint16_t, true>(colptr, j0, n, tl.lidx, val, xs, lane);
    const int64_t j = j0 + lane;
    if (lane < n) f_new[j] = voxel_update<T>(g, j, my_e, s, f, d, c);
}

// ---------------------------------------------------------------------------------------
// Single-pass form of a1 + a2: A is streamed once per surrogate step, by rows.
//
// e = A^T ratio needs ratio_i = y_i / (A f + r)_i, which is complete as soon as
// row i has been reduced; the row's nonzeros are then still in the warp's
// registers, so the warp scatters a_ij * ratio_i at once. The scatter goes to a
// shared-memory accumulator over the tile's staged columns (indexed by the
// same 16-bit local indices as the gather), and the block adds each touched
// column's partial to e with one global atomic add. The f-update then runs as
// an elementwise pass over e. Each lane adds its elements of a row in
// increasing position, as the lane-strided two-pass forward does, so ratio
// is bit-identical to it; e's sums are formed in an order set by the atomics,
// so this form is deterministic only up to rounding.

template <bool PRIV, typename T>
__device__ __forceinline__ void scatter_add(T *acc, int32_t c, T v)
{
    if (PRIV) acc[c] += v;
    else atomicAdd(acc + c, v);
}

// PRIV = false: one accumulator per block, shared-memory atomic adds.
// PRIV = true: one accumulator per warp (8 x the staging buffer), plain
// read-add-write (a row's columns are distinct, and a __syncwarp orders one
// row's updates before the next row's), summed over the warps in a fixed
// order before the global add; only the order of the global adds varies.
// KEEP = true: the first 32 U elements of a row stay in registers between the
// product and the scatter (longer rows are read again); KEEP = false: the
// scatter reads the row again (from L2, where the product's read left it),
// which keeps far fewer registers live and more warps resident.
template <typename T, typename V, int RPW, int U, bool PRIV, bool KEEP, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_project_scatter_tli(int64_t I, int64_t J, const int64_t *__restrict__ rowptr, TliTiles tl,
                      const V *__restrict__ val, const T *__restrict__ f, const T *__restrict__ r, int r_scalar,
                      const T *__restrict__ y, int cap, T *__restrict__ e, int *__restrict__ flag)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *acc = xs + cap;
    const int64_t t = blockIdx.x;
    const int wl = tl.wlen[t];
    const int nstage = wl > 0 ? wl : int(tl.uoff[t + 1] - tl.uoff[t]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *accw = PRIV ? acc + warp * cap : acc;
    if (PRIV) {
        for (int k = lane; k < nstage; k += 32) accw[k] = T(0);
    } else {
        for (int k = threadIdx.x; k < nstage; k += blockDim.x) acc[k] = T(0);
    }
    const bool staged = stage_tile<T>(xs, f, t, tl.uoff, tl.uidx, tl.wbase, tl.wlen, &mbar);
    if (!__syncthreads_and(staged)) {  // block-uniform exit
        if (threadIdx.x == 0) atomicOr(flag, 2);
        return;
    }
    const int64_t i0 = t * (8 * RPW) + int64_t(warp) * RPW;
    if (i0 < I) {
        const int n = int(I - i0 < RPW ? I - i0 : RPW);
        // the warp's rows: positions relative to their first nonzero (set-up
        // checks that RPW consecutive rows hold fewer than 2^31), counts and
        // backgrounds loaded lane-parallel up front so that no row waits on a
        // dependent global load
        const int64_t base = rowptr[i0];
        const uint16_t *__restrict__ li = tl.lidx + base;
        const V *__restrict__ va = val + base;
        const int bound = (lane <= n) ? int(rowptr[i0 + lane] - base) : 0;
        const T ylane = (lane < n) ? y[i0 + lane] : T(0);
        const T rlane = (lane < n) ? (r_scalar ? r[0] : r[i0 + lane]) : T(0);
#pragma unroll 1
        for (int k = 0; k < n; k++) {
            const int s0 = __shfl_sync(0xffffffffu, bound, k);
            const int s1 = __shfl_sync(0xffffffffu, bound, k + 1);
            const T yi = __shfl_sync(0xffffffffu, ylane, k);
            const T ri = __shfl_sync(0xffffffffu, rlane, k);
            if (KEEP) {
                int32_t c[U];
                T v[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int q = s0 + lane + 32 * u;
                    c[u] = 0;
                    v[u] = T(0);
                    if (q < s1) {
                        c[u] = ld_idx(li + q);
                        v[u] = T(ld_val(va + q));
                    }
                }
                T dot = T(0);
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (s0 + lane + 32 * u < s1) dot = fma(v[u], xs[c[u]], dot);
                for (int p = s0 + lane + 32 * U; p < s1; p += 32)  // rows longer than 32 U
                    dot = fma(T(ld_val(va + p)), xs[ld_idx(li + p)], dot);
                dot = warp_sum(dot);
                if (yi != T(0)) {  // warp-uniform; a zero count scatters nothing
                    const T qr = yi / (dot + ri);
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (s0 + lane + 32 * u < s1) scatter_add<PRIV>(accw, c[u], v[u] * qr);
                    for (int p = s0 + lane + 32 * U; p < s1; p += 32)
                        scatter_add<PRIV>(accw, ld_idx(li + p), T(ld_val(va + p)) * qr);
                }
            } else {
                T dot = T(0);
                for (int p0 = s0 + lane; p0 < s1; p0 += 32 * U) {
                    int32_t c[U];
                    T v[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int q = p0 + 32 * u;
                        c[u] = 0;
                        v[u] = T(0);
                        if (q < s1) {
                            c[u] = ld_idx(li + q);
                            v[u] = T(ld_val(va + q));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (p0 + 32 * u < s1) dot = fma(v[u], xs[c[u]], dot);
                }
                dot = warp_sum(dot);
                if (yi != T(0)) {
                    const T qr = yi / (dot + ri);
                    for (int p0 = s0 + lane; p0 < s1; p0 += 32 * U) {
                        int32_t c[U];
                        T v[U];
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            const int q = p0 + 32 * u;
                            c[u] = 0;
                            v[u] = T(0);
                            if (q < s1) {
                                c[u] = int32_t(li[q]);
                                v[u] = T(va[q]);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; u++)
                            if (p0 + 32 * u < s1) scatter_add<PRIV>(accw, c[u], v[u] * qr);
                    }
                }
            }
            if (PRIV) __syncwarp();
        }
    }
    __syncthreads();
    const int64_t u0 = wl > 0 ? 0 : tl.uoff[t];
    const int64_t wb = wl > 0 ? tl.wbase[t] : 0;
    for (int k = threadIdx.x; k < nstage; k += blockDim.x) {
        T a = acc[k];
        if (PRIV) {
#pragma unroll
            for (int w = 1; w < 8; w++) a += acc[w * cap + k];
        }
        if (a != T(0)) {
            const int64_t col = wl > 0 ? wb + k : int64_t(tl.uidx[u0 + k]);
            if (col < J) atomicAdd(e + col, a);
        }
    }
}

// 4-wide form of the single-pass scatter: each lane loads 4 consecutive
// (16-bit index, value) pairs of a row from a 4-aligned position (8-byte and
// 16-byte loads, masked at the row's ends), UV such chunks (128 elements per
// warp each) in flight; the first UV chunks of a row stay in registers for
// the scatter, longer rows read the rest again. The product's element order
// is that of the 4-wide two-pass forward with the same UV, so ratio matches it
// bit for bit. PRIV as in k_project_scatter_tli.
template <typename T, typename V, int RPW, int UV, bool PRIV, int MINB, bool L2PF = false>
__global__ void __launch_bounds__(256, MINB)
k_project_scatter_tli_v4(int64_t I, int64_t J, const int64_t *__restrict__ rowptr, TliTiles tl,
                         const V *__restrict__ val, const T *__restrict__ f, const T *__restrict__ r,
                         int r_scalar, const T *__restrict__ y, int cap, T *__restrict__ e, int *__restrict__ flag)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *acc = xs + cap;
    const int64_t t = blockIdx.x;
    if (L2PF && threadIdx.x == 0)
        prefetch_segments_l2(rowptr, t * (8 * RPW), (t + 1) * (8 * RPW) < I ? (t + 1) * (8 * RPW) : I, tl.lidx, val);
    const int wl = tl.wlen[t];
    const int nstage = wl > 0 ? wl : int(tl.uoff[t + 1] - tl.uoff[t]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *accw = PRIV ? acc + warp * cap : acc;
    if (PRIV) {
        for (int k = lane; k < nstage; k += 32) accw[k] = T(0);
    } else {
        for (int k = threadIdx.x; k < nstage; k += blockDim.x) acc[k] = T(0);
    }
    const bool staged = stage_tile<T>(xs, f, t, tl.uoff, tl.uidx, tl.wbase, tl.wlen, &mbar);
    if (!__syncthreads_and(staged)) {  // block-uniform exit
        if (threadIdx.x == 0) atomicOr(flag, 2);
        return;
    }
    const int64_t i0 = t * (8 * RPW) + int64_t(warp) * RPW;
    if (i0 < I) {
        const int n = int(I - i0 < RPW ? I - i0 : RPW);
        // positions relative to a 4-aligned base, so that aligned relative
        // positions are aligned addresses (set-up checks that RPW consecutive
        // rows hold fewer than 2^31 nonzeros)
        const int64_t base = rowptr[i0] & ~int64_t(3);
        const uint16_t *__restrict__ li = tl.lidx + base;
        const V *__restrict__ va = val + base;
        const int bound = (lane <= n) ? int(rowptr[i0 + lane] - base) : 0;
        const T ylane = (lane < n) ? y[i0 + lane] : T(0);
        const T rlane = (lane < n) ? (r_scalar ? r[0] : r[i0 + lane]) : T(0);
#pragma unroll 1
        for (int k = 0; k < n; k++) {
            const int s0 = __shfl_sync(0xffffffffu, bound, k);
            const int s1 = __shfl_sync(0xffffffffu, bound, k + 1);
            const T yi = __shfl_sync(0xffffffffu, ylane, k);
            const T ri = __shfl_sync(0xffffffffu, rlane, k);
            const int p0 = (s0 & ~3) + 4 * lane;
            int32_t c[UV][4];
            T v[UV][4];
#pragma unroll
            for (int u = 0; u < UV; u++) {
                const int q = p0 + 128 * u;
                if (q < s1) {
                    ld_idx4(li + q, c[u]);
                    ld_val4(va + q, v[u]);
                } else {
#pragma unroll
                    for (int m = 0; m < 4; m++) { c[u][m] = 0; v[u][m] = T(0); }
                }
            }
            T dot = T(0);
#pragma unroll
            for (int u = 0; u < UV; u++)
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    const int q = p0 + 128 * u + m;
                    if (q >= s0 && q < s1) dot = fma(v[u][m], xs[c[u][m]], dot);
                }
            for (int p = p0 + 128 * UV; p < s1; p += 128 * UV) {  // rows longer than the kept chunks
#pragma unroll
                for (int u = 0; u < UV; u++) {
                    const int q = p + 128 * u;
                    if (q < s1) {
                        int32_t c2[4];
                        T v2[4];
                        ld_idx4(li + q, c2);
                        ld_val4(va + q, v2);
#pragma unroll
                        for (int m = 0; m < 4; m++)
                            if (q + m < s1) dot = fma(v2[m], xs[c2[m]], dot);
                    }
                }
            }
            dot = warp_sum(dot);
            if (yi != T(0)) {  // warp-uniform; a zero count scatters nothing
                const T qr = yi / (dot + ri);
#pragma unroll
                for (int u = 0; u < UV; u++)
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const int q = p0 + 128 * u + m;
                        if (q >= s0 && q < s1) scatter_add<PRIV>(accw, c[u][m], v[u][m] * qr);
                    }
                for (int p = p0 + 128 * UV; p < s1; p += 128 * UV) {
#pragma unroll
                    for (int u = 0; u < UV; u++) {
                        const int q = p + 128 * u;
                        if (q < s1) {
                            int32_t c2[4];
                            T v2[4];
                            ld_idx4(li + q, c2);
                            ld_val4(va + q, v2);
#pragma unroll
                            for (int m = 0; m < 4; m++)
                                if (q + m < s1) scatter_add<PRIV>(accw, c2[m], v2[m] * qr);
                        }
                    }
                }
            }
            if (PRIV) __syncwarp();
        }
    }
    __syncthreads();
    const int64_t u0 = wl > 0 ? 0 : tl.uoff[t];
    const int64_t wb = wl > 0 ? tl.wbase[t] : 0;
    for (int k = threadIdx.x; k < nstage; k += blockDim.x) {
        T a = acc[k];
        if (PRIV) {
#pragma unroll
            for (int w = 1; w < 8; w++) a += acc[w * cap + k];
        }
        if (a != T(0)) {
            const int64_t col = wl > 0 ? wb + k : int64_t(tl.uidx[u0 + k]);
            if (col < J) atomicAdd(e + col, a);
        }
    }
}

// Single-pass scatter over the bank-dealt row stream (SpStream, built at
// set-up in sgtv_sp.cu): rows padded to multiples of 4 and 4-aligned, each
// lane holding whole 4-element chunks (position rp[i] + 128 u + 4 lane), so
// no element needs a position mask, and the elements of one access
// instruction spread over the shared-memory banks. The UV chunks of the next
// row are loaded into registers before the current row's gathers (PF), so a
// warp always has a row of the stream in flight while it reduces, divides and
// scatters the previous one. Rows longer than 128 UV elements read their
// further chunks in place. One accumulator per warp, as in the PRIV forms
// above; the padding slots gather the zeroed dummy entry xs[nstage] and add 0
// to the unflushed accumulator slot acc[nstage].
template <int UV, typename T>
struct SpRow {
    uint2 c[UV];    // 4 16-bit local indices per chunk
    T v[UV][4];
};

// ZERO = false leaves the chunks past the row's end unset: every use of a
// chunk is guarded by the same position test, so they are never read.
template <int UV, typename T, typename V, bool ZERO = true>
__device__ __forceinline__ void sp_load(SpRow<UV, T> &b, const uint16_t *__restrict__ li, const V *__restrict__ va,
                                        int s0, int n4, int lane)
{
    const uint16_t *__restrict__ lr = li + s0 + 4 * lane;
    const V *__restrict__ vr = va + s0 + 4 * lane;
#pragma unroll
    for (int u = 0; u < UV; u++) {
        if (128 * u + 4 * lane < n4) {
            b.c[u] = __ldcs(reinterpret_cast<const uint2 *>(lr + 128 * u));
            ld_val4(vr + 128 * u, b.v[u]);
        } else if (ZERO) {
            b.c[u] = make_uint2(0u, 0u);
#pragma unroll
            for (int m = 0; m < 4; m++) b.v[u][m] = T(0);
        }
    }
}

__device__ __forceinline__ int sp_idx(const uint2 &c, int m)
{
    const uint32_t w = (m < 2) ? c.x : c.y;
    return int((m & 1) ? (w >> 16) : (w & 0xFFFFu));
}

// Options of the row-stream scatter without register prefetch (bit flags):
// kSpBatch4: each 4-element chunk's accumulator entries are read before any
//   of them is written back (acc + a * ratio as one fused multiply-add).
//   Valid because a row's columns are distinct (only padding shares the
//   dummy slot, and adds 0); it keeps the compiler from ordering each
//   read-add-write behind the previous write, which it must assume may alias.
// kSpLean: the row's chunks past its end are not zero-filled.
constexpr int kSpBatch4 = 1, kSpLean = 2;

// One row: the dot product with the staged f (warp-reduced), then the ratio
// and the scatter into the warp's accumulator (PRIV) or the block's
// (shared-memory atomic adds).
template <int UV, typename T, typename V>
__device__ __forceinline__ T sp_dot(const SpRow<UV, T> &b, const uint16_t *__restrict__ li,
                                    const V *__restrict__ va, int s0, int n4, const T *xs, int lane)
{
    T dot = T(0);
#pragma unroll
    for (int u = 0; u < UV; u++)
        if (128 * u + 4 * lane < n4) {
#pragma unroll
            for (int m = 0; m < 4; m++) dot = fma(b.v[u][m], xs[sp_idx(b.c[u], m)], dot);
        }
    for (int p = 128 * UV + 4 * lane; p < n4; p += 128) {  // rows longer than the kept chunks
        int32_t c2[4];
        T v2[4];
        ld_idx4(li + s0 + p, c2);
        ld_val4(va + s0 + p, v2);
#pragma unroll
        for (int m = 0; m < 4; m++) dot = fma(v2[m], xs[c2[m]], dot);
    }
    return warp_sum(dot);
}

template <int UV, typename T, typename V, bool PRIV, int OPT = 0>
__device__ __forceinline__ void sp_scatter(const SpRow<UV, T> &b, const uint16_t *__restrict__ li,
                                           const V *__restrict__ va, int s0, int n4, T yi, T ri, T dot, T *accw,
                                           int lane)
{
    if (yi != T(0)) {  // warp-uniform; a zero count scatters nothing
        const T qr = yi / (dot + ri);
#pragma unroll
        for (int u = 0; u < UV; u++)
            if (128 * u + 4 * lane < n4) {
                if constexpr (PRIV && (OPT & kSpBatch4)) {
                    T a[4];
#pragma unroll
                    for (int m = 0; m < 4; m++) a[m] = accw[sp_idx(b.c[u], m)];
#pragma unroll
                    for (int m = 0; m < 4; m++) accw[sp_idx(b.c[u], m)] = fma(b.v[u][m], qr, a[m]);
                } else {
#pragma unroll
                    for (int m = 0; m < 4; m++) scatter_add<PRIV>(accw, sp_idx(b.c[u], m), b.v[u][m] * qr);
                }
            }
        for (int p = 128 * UV + 4 * lane; p < n4; p += 128) {
            int32_t c2[4];
            T v2[4];
            ld_idx4(li + s0 + p, c2);
            ld_val4(va + s0 + p, v2);
#pragma unroll
            for (int m = 0; m < 4; m++) scatter_add<PRIV>(accw, c2[m], v2[m] * qr);
        }
    }
    if (PRIV) __syncwarp();
}

template <int UV, typename T, typename V, bool PRIV>
__device__ __forceinline__ void sp_row(const SpRow<UV, T> &b, const uint16_t *__restrict__ li,
                                       const V *__restrict__ va, int s0, int n4, T yi, T ri, const T *xs, T *accw,
                                       int lane)
{
    const T dot = sp_dot<UV, T, V>(b, li, va, s0, n4, xs, lane);
    sp_scatter<UV, T, V, PRIV>(b, li, va, s0, n4, yi, ri, dot, accw, lane);
}

template <typename T, typename V, int UV, int MINB, bool L2PF = false, bool PRIV = true, bool PF = true,
          int OPT = 0>
__global__ void __launch_bounds__(256, MINB)
k_scatter_sp(int64_t I, int64_t J, const int64_t *__restrict__ rp, const uint16_t *__restrict__ li,
             const V *__restrict__ va, TliTiles tl, const T *__restrict__ f, const T *__restrict__ r, int r_scalar,
             const T *__restrict__ y, int cap, T *__restrict__ e, int *__restrict__ flag)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *acc = xs + cap;
    const int64_t t = blockIdx.x;
    if (L2PF && threadIdx.x == 0)
        prefetch_segments_l2(rp, t * kTliTile, (t + 1) * kTliTile < I ? (t + 1) * kTliTile : I, li, va);
    const int wl = tl.wlen[t];
    const int nstage = wl > 0 ? wl : int(tl.uoff[t + 1] - tl.uoff[t]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T *accw = PRIV ? acc + warp * cap : acc;
    // this thread's entries of a list tile's unique list (k = threadIdx.x + 256 m):
    // loaded once, for the staging gather and for the flush of the sums into e
    constexpr int kU = 3;
    const int64_t u0 = wl > 0 ? 0 : tl.uoff[t];
    int32_t ucol[kU];
#pragma unroll
    for (int m = 0; m < kU; m++) {
        const int k = threadIdx.x + 256 * m;
        ucol[m] = (wl == 0 && k < nstage) ? tl.uidx[u0 + k] : 0;
    }
    // the warp's rows, relative to their first slot (set-up checks that
    // kTliTile / 8 consecutive padded rows hold fewer than 2^31 slots); the
    // first row's chunks are loaded before the staging so that they overlap it
    const int64_t i0 = t * kTliTile + int64_t(warp) * (kTliTile / 8);
    const int n = i0 < I ? int(I - i0 < kTliTile / 8 ? I - i0 : kTliTile / 8) : 0;
    const int64_t base = n > 0 ? rp[i0] : 0;
    const uint16_t *__restrict__ lw = li + base;
    const V *__restrict__ vw = va + base;
    const int bound = (lane <= n && n > 0) ? int(rp[i0 + lane] - base) : 0;
    const T ylane = (lane < n) ? y[i0 + lane] : T(0);
    const T rlane = (lane < n) ? (r_scalar ? r[0] : r[i0 + lane]) : T(0);
    SpRow<UV, T> A, B;
    int a0 = __shfl_sync(0xffffffffu, bound, 0), a1 = __shfl_sync(0xffffffffu, bound, 1);
    if (n > 0) sp_load<UV, T, V, !(OPT & kSpLean)>(A, lw, vw, a0, a1 - a0, lane);
    if (PRIV) {
        for (int k = lane; k <= nstage; k += 32) accw[k] = T(0);  // with the dummy slot
    } else {
        for (int k = threadIdx.x; k <= nstage; k += blockDim.x) acc[k] = T(0);
    }
    bool staged = true;
    if (wl > 0) {  // window tile: one bulk copy (block-uniform branch)
        staged = stage_window<T>(xs, f, tl.wbase[t], wl, &mbar);
    } else {
#pragma unroll
        for (int m = 0; m < kU; m++) {
            const int k = threadIdx.x + 256 * m;
            if (k < nstage) xs[k] = __ldg(f + ucol[m]);
        }
        for (int k = threadIdx.x + 256 * kU; k < nstage; k += blockDim.x) xs[k] = __ldg(f + tl.uidx[u0 + k]);
    }
    if (threadIdx.x == 0) xs[nstage] = T(0);  // the padding slots' operand (outside the staged range)
    if (!__syncthreads_and(staged)) {  // block-uniform exit
        if (threadIdx.x == 0) atomicOr(flag, 2);
        return;
    }
    if (n > 0) {
        if (!PF) {  // one row at a time: the row's chunks loaded, then reduced and scattered
#pragma unroll 1
            for (int k = 0; k < n; k++) {
                const int s0 = __shfl_sync(0xffffffffu, bound, k), s1 = __shfl_sync(0xffffffffu, bound, k + 1);
                if (k > 0) sp_load<UV, T, V, !(OPT & kSpLean)>(A, lw, vw, s0, s1 - s0, lane);
                const T dot = sp_dot<UV, T, V>(A, lw, vw, s0, s1 - s0, xs, lane);
                sp_scatter<UV, T, V, PRIV, OPT>(A, lw, vw, s0, s1 - s0, __shfl_sync(0xffffffffu, ylane, k),
                                                __shfl_sync(0xffffffffu, rlane, k), dot, accw, lane);
            }
        }
#pragma unroll 1
        for (int k = 0; PF && k < n; k += 2) {
            // row k from A while row k + 1 streams into B
            const int b0 = a1, b1 = __shfl_sync(0xffffffffu, bound, (k + 2 <= n) ? k + 2 : n);
            if (k + 1 < n) sp_load<UV, T, V>(B, lw, vw, b0, b1 - b0, lane);
            sp_row<UV, T, V, PRIV>(A, lw, vw, a0, a1 - a0, __shfl_sync(0xffffffffu, ylane, k),
                                   __shfl_sync(0xffffffffu, rlane, k), xs, accw, lane);
            if (k + 1 >= n) break;
            // row k + 1 from B while row k + 2 streams into A
            a0 = b1;
            a1 = __shfl_sync(0xffffffffu, bound, (k + 3 <= n) ? k + 3 : n);
            if (k + 2 < n) sp_load<UV, T, V>(A, lw, vw, a0, a1 - a0, lane);
            sp_row<UV, T, V, PRIV>(B, lw, vw, b0, b1 - b0, __shfl_sync(0xffffffffu, ylane, k + 1),
                                   __shfl_sync(0xffffffffu, rlane, k + 1), xs, accw, lane);
        }
    }
    __syncthreads();
    const int64_t wb = wl > 0 ? tl.wbase[t] : 0;
    auto flush = [&](int k, int32_t ucolk) {
        T a = acc[k];
        if (PRIV) {
#pragma unroll
            for (int w = 1; w < 8; w++) a += acc[w * cap + k];
        }
        if (a != T(0)) {
            const int64_t col = wl > 0 ? wb + k : int64_t(ucolk);
            if (col < J) atomicAdd(e + col, a);
        }
    };
#pragma unroll
    for (int m = 0; m < kU; m++) {
        const int k = threadIdx.x + 256 * m;
        if (k < nstage) flush(k, ucol[m]);
    }
    for (int k = threadIdx.x + 256 * kU; k < nstage; k += blockDim.x) flush(k, wl > 0 ? 0 : tl.uidx[u0 + k]);
}

// The f-update (Eq. 5 closed form) from the accumulated e, which it clears
// for the next scatter: one warp per spatial site, lanes over q. It reads
// u = d - c as the shrink left it (one load per direction and position
// instead of two), the site's stencil (which neighbours exist, their
// offsets) is found once per warp, and QB q-steps of every lane issue all
// their loads before any arithmetic, which is that of voxel_update_at in the
// same order.
template <typename T, int QB>
__global__ void __launch_bounds__(256, QB == 1 ? 4 : 3)
k_fupdate_site(Geom g, T *__restrict__ e, const T *__restrict__ s, const T *__restrict__ f,
               const T *__restrict__ u, T *__restrict__ f_new)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
#pragma unroll 1
    for (int64_t site = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; site < g.S; site += nwarps) {
        int64_t v0;
        const Loc L = locate_site(g, site, v0);
        int32_t stF[4], stB[4];  // offsets of the existing neighbours (0 for a ghost: the voxel itself, unused)
        bool inF[4], inB[4];
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const int32_t step = p < g.n_dirs ? int32_t(step_of(g, L, p)) : 0;
            inF[p] = p < g.n_dirs && inside(L, L.x + g.dx[p], L.z + g.dz[p]);
            inB[p] = p < g.n_dirs && inside(L, L.x - g.dx[p], L.z - g.dz[p]);
            stF[p] = inF[p] ? step : 0;
            stB[p] = inB[p] ? step : 0;
        }
        const T rho = lrho<T>(L);
        const int nd = g.n_dirs;
#pragma unroll 1
        for (int q0 = 0; q0 < L.Nq; q0 += 32 * QB) {
            T ej[QB], fj[QB], sj[QB], fF[QB][4], fB[QB][4], uF[QB][4], uB[QB][4];
#pragma unroll
            for (int b = 0; b < QB; b++) {
                const int q = q0 + 32 * b + lane;
                const bool act = q < L.Nq;
                const int64_t j = v0 + (act ? q : 0);
                ej[b] = e[j];
                fj[b] = f[j];
                sj[b] = s[j];
#pragma unroll
                for (int p = 0; p < 4; p++) {
                    const int64_t pj = int64_t(p < nd ? p : 0) * g.J + j;
                    fF[b][p] = f[j + stF[p]];
                    fB[b][p] = f[j - stB[p]];
                    uF[b][p] = u[pj];
                    uB[b][p] = u[pj - stB[p]];
                }
            }
#pragma unroll
            for (int b = 0; b < QB; b++) {
                const int q = q0 + 32 * b + lane;
                if (q >= L.Nq) continue;
                const int64_t j = v0 + q;
                e[j] = T(0);
                T alpha = T(0), gamma = T(0);
#pragma unroll
                for (int p = 0; p < 4; p++) {
                    if (p >= nd) break;
                    const T w = wgt<T>(g, p);
                    const T w2 = w * w;
                    if (inF[p]) {
                        alpha += w2;
                        gamma += w * (w * (fj[b] + fF[b][p]) + uF[b][p]);
                    } else {
                        alpha += T(0.5) * w2;
                        gamma += w * uF[b][p];
                    }
                    if (inB[p]) {
                        alpha += w2;
                        gamma += w * (w * (fB[b][p] + fj[b]) - uB[b][p]);
                    }
                }
                alpha *= rho;
                gamma *= rho;
                f_new[j] = sgtv_root<T>(alpha, sj[b] - gamma, fj[b] * ej[b], sj[b]);
            }
        }
    }
}

// Same update, one thread per hyper-voxel.
template <typename T>
__global__ void __launch_bounds__(256)
k_fupdate(Geom g, T *__restrict__ e, const T *__restrict__ s, const T *__restrict__ f, const T *__restrict__ d,
          const T *__restrict__ c, T *__restrict__ f_new)
{
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < g.J; j += int64_t(gridDim.x) * blockDim.x) {
        const T ej = e[j];
        e[j] = T(0);
        f_new[j] = voxel_update<T, true>(g, j, ej, s, f, d, c);
    }
}

// ---------------------------------------------------------------------------------------
// TMA-streamed persistent forms of the two sparse products.
//
// One CTA per SM walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// through an NS-deep ring of shared-memory stages, with one producer warp and
// NW consumer warps. Filling a stage is one mbarrier phase of bulk copies
// (cp.async.bulk) issued by the producer: the tile's kTliTile + 2 segment
// pointers, its 16-bit local indices, its values, and either its index window
// of the dense operand or its unique-index list. A list tile then needs a
// gather of the dense operand into the stage, which the producer issues one
// tile behind its bulk copies as 4/8-byte cp.async copies completing on the
// stage's full barrier. Consumers compute from shared memory only and release
// the stage on its empty barrier; no block-wide barrier is taken in the loop,
// so warps drift freely and the HBM stream never waits on a computing warp.

struct TmaMat {
    const int64_t *ptr;      // segment pointers, padded to ntiles * kTliTile + 2 entries
    const uint16_t *lidx;    // local indices (padded past nnz)
    const int32_t *wbase, *wlen;
    const int64_t *uoff;
    const int32_t *uidx;     // padded past the last entry
    int64_t nseg, ntiles;
};

// Byte offsets of the regions of one stage (each 128-byte aligned).
struct TmaLayout {
    int off_lidx, off_val, off_uidx, off_xs, stage_bytes;
};

struct TileDesc {
    int64_t p0, p1, u0, u1;
    int32_t wb, wl;
};

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b)) : "memory");
}

// Bounded wait for the phase with the given parity: false once timeout_ns
// have passed since the first unsuccessful try.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, uint64_t timeout_ns)
{
    uint64_t t0 = 0;
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(b)), "r"(parity) : "memory");
        if (done) return true;
        const uint64_t now = global_ns();
        if (t0 == 0) t0 = now;
        else if (now - t0 > timeout_ns) return false;
    }
}

template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *dst, const void *src)
{
    if (BYTES == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t *b)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t round16(int64_t bytes) { return uint32_t((bytes + 15) & ~int64_t(15)); }

template <typename T, typename V, int TS, int NS, int NW>
struct TmaPipe {
    static_assert(NS >= 3, "a tile's bulk copies need an iteration to land before its gathers");
    static_assert(TS % NW == 0, "whole segments per warp");
    static constexpr int VA = 16 / int(sizeof(V));   // value elements per 16 bytes
    static constexpr int SPW = TS / NW;              // segments per warp

    __device__ static TileDesc desc(const TmaMat &m, int64_t t)
    {
        TileDesc D;
        D.p0 = m.ptr[t * TS];
        D.p1 = m.ptr[t * TS + TS];
        D.u0 = m.uoff[t];
        D.u1 = m.uoff[t + 1];
        D.wb = m.wbase[t];
        D.wl = m.wlen[t];
        return D;
    }

    // Thread 0: one mbarrier phase of bulk copies filling stage sb with tile t.
    __device__ static void fill(const TmaMat &m, const TmaLayout &L, const V *val, const T *x, int64_t t,
                                const TileDesc &D, unsigned char *sb, uint64_t *tmab)
    {
        const uint32_t b_ptr = (TS + 2) * 8;
        const int64_t a0 = D.p0 & ~int64_t(7);
        const int64_t v0 = D.p0 & ~int64_t(VA - 1);
        const uint32_t b_lidx = D.p1 > D.p0 ? round16((D.p1 - a0) * 2) : 0u;
        const uint32_t b_val = D.p1 > D.p0 ? round16((D.p1 - v0) * int64_t(sizeof(V))) : 0u;
        const int64_t c0 = D.u0 & ~int64_t(3);
        const uint32_t b_u = (D.wl == 0 && D.u1 > D.u0) ? round16((D.u1 - c0) * 4) : 0u;
        const uint32_t b_w = D.wl > 0 ? uint32_t(D.wl) * uint32_t(sizeof(T)) : 0u;
        mbar_arrive_expect_tx(tmab, b_ptr + b_lidx + b_val + b_u + b_w);
        bulk_g2s(sb, m.ptr + t * TS, b_ptr, tmab);
        if (b_lidx) bulk_g2s(sb + L.off_lidx, m.lidx + a0, b_lidx, tmab);
        if (b_val) bulk_g2s(sb + L.off_val, val + v0, b_val, tmab);
        if (b_u) bulk_g2s(sb + L.off_uidx, m.uidx + c0, b_u, tmab);
        if (b_w) bulk_g2s(sb + L.off_xs, x + D.wb, b_w, tmab);
    }

    // Producer warp, after the stage's bulk copies landed: gather a list
    // tile's dense values with async copies, then every lane arrives on fullb
    // once its own copies complete.
    __device__ static void gather(const TileDesc &D, const T *x, unsigned char *sb, const TmaLayout &L,
                                  uint64_t *fullb, int lane)
    {
        if (D.wl == 0 && D.u1 > D.u0) {
            const int32_t *us = reinterpret_cast<const int32_t *>(sb + L.off_uidx) + (D.u0 & 3);
            T *xs = reinterpret_cast<T *>(sb + L.off_xs);
            const int n = int(D.u1 - D.u0);
            for (int k = lane; k < n; k += 32) cp_async_small<sizeof(T)>(xs + k, x + us[k]);
        }
        cp_async_arrive_noinc(fullb);
    }

    // Consumer warp: its SPW segments of the tile from shared memory; lane k
    // returns segment warp * SPW + k's dot product.
    __device__ static T compute(const TileDesc &D, const unsigned char *sb, const TmaLayout &L, int warp, int lane)
    {
        const int64_t *ps = reinterpret_cast<const int64_t *>(sb);
        const uint16_t *ls = reinterpret_cast<const uint16_t *>(sb + L.off_lidx);
        const V *vs = reinterpret_cast<const V *>(sb + L.off_val);
        const T *xs = reinterpret_cast<const T *>(sb + L.off_xs);
        const int64_t a0 = D.p0 & ~int64_t(7);
        const int64_t v0 = D.p0 & ~int64_t(VA - 1);
        T mine = T(0);
#pragma unroll
        for (int k = 0; k < SPW; k++) {
            const int sidx = warp * SPW + k;
            const int64_t st = ps[sidx], en = ps[sidx + 1];
            T acc = T(0);
            int64_t q = st + lane;
            for (; q + 96 < en; q += 128) {
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int64_t qq = q + 32 * u;
                    acc = fma(T(vs[qq - v0]), xs[ls[qq - a0]], acc);
                }
            }
            for (; q < en; q += 32) acc = fma(T(vs[q - v0]), xs[ls[q - a0]], acc);
            acc = warp_sum(acc);
            if (lane == k) mine = acc;
        }
        return mine;
    }

    // Warp-specialised persistent loop: warp NW is the producer (bulk copies of
    // tile k into stage k % NS once the consumers released it, then the list
    // gathers of tile k - 1), warps 0 .. NW-1 consume tiles in order and
    // release each stage on its empty barrier. epi(seg, value) runs on lane
    // k < SPW of each consumer warp for segment tile * TS + warp * SPW + k.
    template <typename Epi>
    __device__ static void run(const TmaMat &m, const TmaLayout &L, const V *val, const T *x, int *flag, Epi epi)
    {
        extern __shared__ __align__(128) unsigned char smem_raw[];
        __shared__ uint64_t tmab[NS], fullb[NS], emptyb[NS];
        __shared__ TileDesc sdesc[NS];
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        if (tid == 0) {
            for (int k = 0; k < NS; k++) {
                mbar_init(&tmab[k], 1);
                mbar_init(&fullb[k], 32);
                mbar_init(&emptyb[k], NW);
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        const int64_t t0 = blockIdx.x, step = gridDim.x;
        const int64_t n = m.ntiles > t0 ? (m.ntiles - t0 + step - 1) / step : 0;  // tiles of this CTA
        auto stage = [&](int64_t k) { return smem_raw + size_t(k % NS) * L.stage_bytes; };
        const uint64_t limit = 1000000000ull;  // 1 s per wait: far beyond any healthy copy
        bool bad = false;
        if (warp == NW) {
            TileDesc Dn{};
            if (lane == 0 && n > 0) Dn = desc(m, t0);
            int64_t filled = -1;
            for (int64_t k = 0; k <= n && !bad; k++) {
                if (k < n) {
                    const int s = int(k % NS);
                    if (k >= NS) bad |= !mbar_wait(&emptyb[s], uint32_t((k / NS - 1) & 1), limit);
                    if (!bad && lane == 0) {
                        sdesc[s] = Dn;
                        fill(m, L, val, x, t0 + k * step, Dn, stage(k), &tmab[s]);
                        if (k + 1 < n) Dn = desc(m, t0 + (k + 1) * step);
                    }
                    if (!bad) filled = k;
                    __syncwarp();
                }
                if (k >= 1 && !bad) {
                    const int s1 = int((k - 1) % NS);
                    bad |= !mbar_wait(&tmab[s1], uint32_t(((k - 1) / NS) & 1), limit);
                    if (!bad) gather(sdesc[s1], x, stage(k - 1), L, &fullb[s1], lane);
                }
                bad = __any_sync(0xffffffffu, bad);
            }
            cp_async_wait_all();
            if (bad) {
                if (lane == 0) {
                    atomicOr(flag, 2);
                    // the last fill may still be landing: one more bounded wait
                    if (filled >= 0) mbar_wait(&tmab[filled % NS], uint32_t((filled / NS) & 1), limit);
                }
            }
        } else {
            for (int64_t i = 0; i < n; i++) {
                const int s = int(i % NS);
                if (!mbar_wait(&fullb[s], uint32_t((i / NS) & 1), limit)) {
                    if (lane == 0) atomicOr(flag, 2);
                    break;
                }
                const TileDesc D = sdesc[s];
                const T v = compute(D, stage(i), L, warp, lane);
                const int64_t seg = (t0 + i * step) * TS + int64_t(warp) * SPW + lane;
                if (lane < SPW && seg < m.nseg) epi(seg, v);
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&emptyb[s])) : "memory");
            }
        }
    }
};

template <typename T, typename V, int NS, int NW>
__global__ void __launch_bounds__(32 * (NW + 1), 1)
k_forward_tma(TmaMat m, TmaLayout L, const V *__restrict__ val, const T *__restrict__ f,
              const T *__restrict__ r, int r_scalar, const T *__restrict__ y, T *__restrict__ ratio,
              int *__restrict__ flag)
{
    TmaPipe<T, V, kTliTile, NS, NW>::run(m, L, val, f, flag, [&](int64_t i, T acc) {
        const T yb = acc + (r_scalar ? r[0] : r[i]);
        const T yi = y[i];
        ratio[i] = (yi == T(0)) ? T(0) : yi / yb;
    });
}

template <typename T, typename V, int NS, int NW>
__global__ void __launch_bounds__(32 * (NW + 1), 1)
k_back_update_tma(TmaMat m, TmaLayout L, Geom g, const V *__restrict__ val, const T *__restrict__ ratio,
                  const T *__restrict__ s, const T *__restrict__ f, const T *__restrict__ d,
                  const T *__restrict__ c, T *__restrict__ f_new, int *__restrict__ flag)
{
    TmaPipe<T, V, kTliTile, NS, NW>::run(m, L, val, ratio, flag, [&](int64_t j, T e) {
        f_new[j] = voxel_update<T>(g, j, e, s, f, d, c);
    });
}

// ---------------------------------------------------------------------------------------
// One persistent (cooperative) launch per ADMM iteration: the three phases
// of sgtv_iterate -- tiled forward projection, tiled backprojection with the
// f-update, group shrink with the dual update -- separated by grid-wide
// barriers. Every block walks the tiles (then the sites) of each phase with a
// grid stride. Per segment the arithmetic is that of the tiled kernels, so
// results are identical to the three-launch path with the same tile forms.

// Grid-wide barrier (all blocks co-resident: cooperative launch). The last
// block to arrive resets the count and advances the generation; the others
// spin on the generation for at most bar->limit_ns (1 s unless the host set
// another bound; 0 gives up at the first unsuccessful look), then record a
// timeout and report false (the whole block learns it). No bulk copy of the
// block is in flight at a barrier, so a block that gives up may exit.
__device__ __forceinline__ bool grid_sync(GridBar *bar, int *flag)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = &bar->gen;
        const unsigned int gen = *vgen;
        const uint64_t limit = bar->limit_ns;
        __threadfence();
        if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*vgen == gen) {
                if (global_ns() - t0 >= limit) {
                    ok = 0;
                    atomicOr(flag, 2);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <typename T, typename V, int UVF, int UVB, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_iteration(int64_t I, const int64_t *__restrict__ rowptr, TliTiles tr, int64_t ntr, const V *__restrict__ rval,
            const T *__restrict__ r, int r_scalar, const T *__restrict__ y, T *__restrict__ ratio, Geom g,
            const int64_t *__restrict__ colptr, TliTiles tc, int64_t ntc, const V *__restrict__ cval,
            const T *__restrict__ s, const T *__restrict__ f, T *__restrict__ f_new, const T *__restrict__ d,
            T *__restrict__ d_out, T *__restrict__ c, int do_shrink, GridBar *bar, int *__restrict__ flag)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t mbar;
    T *xs = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // phase 1: ybar, ratio (Eq. 1)
    for (int64_t t = blockIdx.x; t < ntr; t += gridDim.x) {
        __syncthreads();  // the previous tile's staging is no longer read
        if (!stage_tile<T>(xs, f, t, tr.uoff, tr.uidx, tr.wbase, tr.wlen, &mbar)) {
            if (threadIdx.x == 0) atomicOr(flag, 2);
            continue;
        }
        const int64_t i0 = t * kTliTile + int64_t(warp) * (kTliTile / 8);
        if (i0 < I) {
            const int n = int(I - i0 < kTliTile / 8 ? I - i0 : kTliTile / 8);
            const T acc = UVF > 0 ? warp_segments_v4<(UVF > 0 ? UVF : 1), T, V>(rowptr, i0, n, tr.lidx, rval, xs, lane)
                                  : warp_segments<8, T, V, false, uint16_t, true>(rowptr, i0, n, tr.lidx, rval, xs, lane);
            const int64_t i = i0 + lane;
            if (lane < n) {
                const T yb = acc + (r_scalar ? r[0] : r[i]);
                const T yi = y[i];
                ratio[i] = (yi == T(0)) ? T(0) : yi / yb;
            }
        }
    }
    if (!grid_sync(bar, flag)) return;
    // phase 2: e = A^T ratio and the closed-form f-update (Eq. 5)
    for (int64_t t = blockIdx.x; t < ntc; t += gridDim.x) {
        __syncthreads();
        if (!stage_tile<T>(xs, ratio, t, tc.uoff, tc.uidx, tc.wbase, tc.wlen, &mbar)) {
            if (threadIdx.x == 0) atomicOr(flag, 2);
            continue;
        }
        const int64_t j0 = t * kTliTile + int64_t(warp) * (kTliTile / 8);
        if (j0 < g.J) {
            const int n = int(g.J - j0 < kTliTile / 8 ? g.J - j0 : kTliTile / 8);
            const T e = UVB > 0 ? warp_segments_v4<(UVB > 0 ? UVB : 1), T, V>(colptr, j0, n, tc.lidx, cval, xs, lane)
                                : warp_segments<8, T, V, false, uint16_t, true>(colptr, j0, n, tc.lidx, cval, xs, lane);
            const int64_t j = j0 + lane;
            if (lane < n) f_new[j] = voxel_update<T>(g, j, e, s, f, d, c);
        }
    }
    if (!do_shrink) return;
    if (!grid_sync(bar, flag)) return;
    // phase 3: group shrink and dual update (Eqs. 6-7)
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t site = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; site < g.S; site += nwarps)
        shrink_site(g, f_new, d_out, c, site, lane, flag);
}

// ---------------------------------------------------------------------------------------
// FP64 reductions. Each block writes one partial per field to `part`
// (field-major: part[field * nblocks + block]); k_finalize then reduces the
// partials of every field in a fixed order, so results do not depend on timing.

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum (or max) over the block of one value per thread; result valid in thread 0.
template <bool MAX>
__device__ __forceinline__ double block_reduce(double v, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = MAX ? warp_max_d(v) : warp_sum_d(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (lane < nw) ? sh[lane] : (MAX ? -1.0 : 0.0);
        v = MAX ? warp_max_d(v) : warp_sum_d(v);
    }
    return v;
}

// Deviance partials: ybar accumulated in FP64 from the stored A values and f.
template <typename T, typename V>
__global__ void __launch_bounds__(256)
k_dev_partials(int64_t I, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
               const V *__restrict__ val, const T *__restrict__ f, const T *__restrict__ r,
               int r_scalar, const T *__restrict__ y, double *__restrict__ part)
{
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    double mine = 0.0;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < I; i += nwarps) {
        double acc = 0.0;
        const int64_t start = rowptr[i], end = rowptr[i + 1];
        for (int64_t p = start + lane; p < end; p += 32)
            acc = fma(to_f64(val[p]), double(f[col[p]]), acc);
        acc = warp_sum_d(acc);
        if (lane == 0) {
            const double yb = acc + double(r_scalar ? r[0] : r[i]);
            const double yi = double(y[i]);
            double t = yb - yi;
            if (yi > 0.0) t += yi * log(yi / yb);
            mine += t;
        }
    }
    double tot = block_reduce<false>(mine, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Group-TV partials over sites [s0, s1) of a direction-major field. Without
// `d`: field 0 = sum_s ||(w.G f)_s||, field 1 = sum_s beta_scan ||(w.G f)_s||.
// With `d`: field 0 = ||w.G f - d||^2 and field 1 = ||d||^2 (primal residual).
template <typename T>
__global__ void __launch_bounds__(256)
k_tv_partials(Geom g, const T *__restrict__ f, const T *__restrict__ d, int64_t s0, int64_t s1,
              double *__restrict__ part)
{
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    double a0 = 0.0, a1 = 0.0;
    for (int64_t site = s0 + ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); site < s1; site += nwarps) {
        int64_t v0;
        const Loc L = locate_site(g, site, v0);
        double n2 = 0.0, dd = 0.0, rb = 0.0;  // rb: sum of the (site, q) norms (standard TV)
        for (int q = lane; q < L.Nq; q += 32) {
            const int64_t j = v0 + q;
            double m2 = 0.0;
            for (int p = 0; p < g.n_dirs; p++) {
                double v = wgrad_at_f64(g, L, f, j, p);
                if (d) {
                    const double dv = double(d[int64_t(p) * g.J + j]);
                    v -= dv;
                    dd += dv * dv;
                }
                n2 += v * v;
                m2 += v * v;
            }
            rb += sqrt(m2);
        }
        n2 = warp_sum_d(n2);
        dd = warp_sum_d(dd);
        rb = warp_sum_d(rb);
        if (lane == 0) {
            if (d) {
                a0 += n2;
                a1 += dd;
            } else {
                const double r = g.per_bin ? rb : sqrt(n2);
                a0 += r;
                a1 += L.beta * r;
            }
        }
    }
    double t0 = block_reduce<false>(a0, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t0;
    double t1 = block_reduce<false>(a1, sh);
    if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t1;
}

// KKT partials: g_j = s_j - e_j + rho_scan ((w.G)^T c)_j, max_j |min(f_j, g_j)|, and max s.
template <typename T>
__global__ void __launch_bounds__(256)
k_kkt_partials(Geom g, const T *__restrict__ f, const T *__restrict__ e, const T *__restrict__ s,
               const T *__restrict__ c, double *__restrict__ part)
{
    __shared__ double sh[32];
    double m = 0.0, smax = 0.0;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < g.J; j += int64_t(gridDim.x) * blockDim.x) {
        const Loc L = locate_voxel(g, j);
        double adj = 0.0;
        for (int p = 0; p < g.n_dirs; p++) {
            const int64_t pj = int64_t(p) * g.J + j;
            adj += g.w[p] * double(c[pj]);
            if (inside(L, L.x - g.dx[p], L.z - g.dz[p])) adj -= g.w[p] * double(c[pj - step_of(g, L, p)]);
        }
        const double gj = double(s[j]) - double(e[j]) + L.rho * adj;
        m = fmax(m, fabs(fmin(double(f[j]), gj)));
        smax = fmax(smax, double(s[j]));
    }
    double t0 = block_reduce<true>(m, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t0;
    double t1 = block_reduce<true>(smax, sh);
    if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t1;
}

// Dual-residual partials: with a_j = rho_scan ((w.G)^T (d - d_prev))_j and
// b_j = rho_scan ((w.G)^T c)_j, field 0 = sum_j a_j^2, field 1 = sum_j b_j^2.
template <typename T>
__global__ void __launch_bounds__(256)
k_dual_partials(Geom g, const T *__restrict__ d, const T *__restrict__ d_prev, const T *__restrict__ c,
                double *__restrict__ part)
{
    __shared__ double sh[32];
    double sa = 0.0, sb = 0.0;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < g.J; j += int64_t(gridDim.x) * blockDim.x) {
        const Loc L = locate_voxel(g, j);
        double a = 0.0, b = 0.0;
        for (int p = 0; p < g.n_dirs; p++) {
            const int64_t pj = int64_t(p) * g.J + j;
            a += g.w[p] * (double(d[pj]) - double(d_prev[pj]));
            b += g.w[p] * double(c[pj]);
            if (inside(L, L.x - g.dx[p], L.z - g.dz[p])) {
                const int64_t pa = pj - step_of(g, L, p);
                a -= g.w[p] * (double(d[pa]) - double(d_prev[pa]));
                b -= g.w[p] * double(c[pa]);
            }
        }
        a *= L.rho;
        b *= L.rho;
        sa += a * a;
        sb += b * b;
    }
    double t0 = block_reduce<false>(sa, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t0;
    double t1 = block_reduce<false>(sb, sh);
    if (threadIdx.x == 0) part[gridDim.x + blockIdx.x] = t1;
}

// Sum of a T vector in FP64 (kappa of the initialisation).
template <typename T>
__global__ void __launch_bounds__(256)
k_sum_partials(int64_t n, const T *__restrict__ a, double *__restrict__ part)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        acc += double(a[k]);
    double t = block_reduce<false>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

}  // namespace sgtv
