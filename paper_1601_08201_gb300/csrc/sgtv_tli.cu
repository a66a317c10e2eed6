// sgtv_tli.cu -- set-up of the tiled local-index (TLI) form of a compressed
// matrix: per tile of kTliTile consecutive rows (columns), 16-bit local
// indices into a per-tile staging buffer of the dense operand.
//
//   window form : the tile's index window [wbase, wbase + wlen), aligned to
//                 16 bytes so one bulk copy stages it; lidx = idx - wbase
//   list form   : the tile's sorted unique indices; lidx = rank in that list,
//                 found through a shared-memory bitmap over [tmin, tmax] (in
//                 chunks of kMaxWords words when the range is wider) and
//                 prefix popcounts (no sort needed)
#include <limits.h>

#include "sgtv_internal.h"

namespace sgtv {

namespace {

constexpr int kT = 256;
constexpr int kMaxWords = 48 * 1024;   // 192 KB bitmap: tile ranges up to 1.5M indices

__global__ void k_tile_range(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx, int64_t nseg,
                             int64_t ntiles, int32_t *__restrict__ tmin, int32_t *__restrict__ tmax)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t t = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; t < ntiles; t += nwarps) {
        int32_t mn = INT_MAX, mx = -1;
        for (int k = lane; k < kTliTile; k += 32) {
            const int64_t s = t * kTliTile + k;
            if (s < nseg) {
                const int64_t a = ptr[s], b = ptr[s + 1];
                if (b > a) {
                    mn = min(mn, idx[a]);
                    mx = max(mx, idx[b - 1]);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            tmin[t] = mn;
            tmax[t] = mx;
        }
    }
}

__global__ void k_window_lidx(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx, int64_t nseg,
                              const int32_t *__restrict__ wbase, const int32_t *__restrict__ wlen,
                              uint16_t *__restrict__ lidx)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t s = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < nseg; s += nwarps) {
        if (wlen[s / kTliTile] == 0) continue;  // a list tile
        const int32_t base = wbase[s / kTliTile];
        for (int64_t p = ptr[s] + lane; p < ptr[s + 1]; p += 32) lidx[p] = uint16_t(idx[p] - base);
    }
}

// Bitmap of the tile's indices in the chunk [lo, lo + 32 * words) of its
// index range (a tile whose range exceeds the bitmap is processed chunk by
// chunk). p0, p1 bound the tile's nonzeros.
__device__ void chunk_bitmap(const int32_t *__restrict__ idx, int64_t p0, int64_t p1, int64_t lo, int words,
                             uint32_t *bits)
{
    for (int w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
    __syncthreads();
    const int64_t hi = lo + int64_t(words) * 32;
    for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const int64_t v = int64_t(idx[p]) - lo;
        if (v >= 0 && v < hi - lo) atomicOr(&bits[v >> 5], 1u << (v & 31));
    }
    __syncthreads();
}

// The tile's nonzeros, and its chunks: number of words in the chunk starting
// at lo (0 once past tmax).
__device__ __forceinline__ void tile_span(const int64_t *__restrict__ ptr, int64_t nseg, int64_t t, int64_t &p0,
                                          int64_t &p1)
{
    const int64_t s0 = t * kTliTile;
    const int64_t s1 = (s0 + kTliTile < nseg) ? s0 + kTliTile : nseg;
    p0 = ptr[s0];
    p1 = ptr[s1];
}

__device__ __forceinline__ int chunk_words(int64_t lo, int32_t tmax, int max_words)
{
    if (lo > tmax) return 0;
    const int64_t w = (int64_t(tmax) - lo) / 32 + 1;
    return int(w < max_words ? w : max_words);
}

__global__ void k_list_count(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx, int64_t nseg,
                             const int32_t *__restrict__ tmin, const int32_t *__restrict__ tmax, int max_words,
                             int32_t *__restrict__ ucnt)
{
    extern __shared__ uint32_t bits[];
    __shared__ int total;
    const int64_t t = blockIdx.x;
    const int32_t mn = tmin[t], mx = tmax[t];
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    if (mx >= mn) {  // block-uniform: an empty tile or a window tile has mx < mn
        int64_t p0, p1;
        tile_span(ptr, nseg, t, p0, p1);
        for (int64_t lo = mn;; lo += int64_t(max_words) * 32) {
            const int words = chunk_words(lo, mx, max_words);
            if (words == 0) break;
            chunk_bitmap(idx, p0, p1, lo, words, bits);
            int c = 0;
            for (int w = threadIdx.x; w < words; w += blockDim.x) c += __popc(bits[w]);
            atomicAdd(&total, c);
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) ucnt[t] = total;
}

__global__ void k_list_build(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx, int64_t nseg,
                             const int32_t *__restrict__ tmin, const int32_t *__restrict__ tmax,
                             const int32_t *__restrict__ wlen, int max_words, const int64_t *__restrict__ uoff,
                             int32_t *__restrict__ uidx, uint16_t *__restrict__ lidx)
{
    extern __shared__ uint32_t bits[];
    int32_t *chunk_pre = reinterpret_cast<int32_t *>(bits + max_words);  // one per 32 words
    __shared__ int base;   // rank of the first index of the current chunk
    __shared__ int run;
    const int64_t t = blockIdx.x;
    const int32_t mn = tmin[t], mx = tmax[t];
    if (wlen[t] != 0 || mx < mn) return;  // a window tile or an empty one (block-uniform)
    int64_t p0, p1;
    tile_span(ptr, nseg, t, p0, p1);
    const int64_t u0 = uoff[t];
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int64_t lo = mn;; lo += int64_t(max_words) * 32) {
        const int words = chunk_words(lo, mx, max_words);
        if (words == 0) break;
        chunk_bitmap(idx, p0, p1, lo, words, bits);
        const int nchunks = (words + 31) / 32;
        for (int ch = threadIdx.x; ch < nchunks; ch += blockDim.x) {
            int c = 0;
            for (int w = ch * 32; w < words && w < ch * 32 + 32; w++) c += __popc(bits[w]);
            chunk_pre[ch] = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) {  // exclusive scan over the chunk's 32-word groups
            int r = base;
            for (int ch = 0; ch < nchunks; ch++) {
                const int c = chunk_pre[ch];
                chunk_pre[ch] = r;
                r += c;
            }
            run = r;
        }
        __syncthreads();
        for (int w = threadIdx.x; w < words; w += blockDim.x) {
            int rank = chunk_pre[w >> 5];
            for (int w2 = w & ~31; w2 < w; w2++) rank += __popc(bits[w2]);
            uint32_t m = bits[w];
            while (m) {
                const int b = __ffs(m) - 1;
                uidx[u0 + rank++] = int32_t(lo + 32 * w + b);
                m &= m - 1;
            }
        }
        const int64_t hi = lo + int64_t(words) * 32;
        for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int64_t v = int64_t(idx[p]) - lo;
            if (v < 0 || v >= hi - lo) continue;
            const int w = int(v >> 5);
            int rank = chunk_pre[w >> 5];
            for (int w2 = w & ~31; w2 < w; w2++) rank += __popc(bits[w2]);
            rank += __popc(bits[w] & ((1u << (v & 31)) - 1u));
            lidx[p] = uint16_t(rank);
        }
        __syncthreads();
        if (threadIdx.x == 0) base = run;
        __syncthreads();
    }
}

// Every local index must fall inside its tile's staging buffer and every
// list entry inside the dense vector: checked once at set-up so the hot
// kernels can index shared memory without bounds checks.
__global__ void k_check_lidx(const int64_t *__restrict__ ptr, int64_t nseg, const uint16_t *__restrict__ lidx,
                             const int32_t *__restrict__ wlen, const int64_t *__restrict__ uoff,
                             const int32_t *__restrict__ uidx, int64_t n_dense, int *__restrict__ flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    bool bad = false;
    for (int64_t s = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; s < nseg; s += nwarps) {
        const int64_t t = s / kTliTile;
        const int64_t lim = wlen[t] > 0 ? int64_t(wlen[t]) : uoff[t + 1] - uoff[t];
        for (int64_t p = ptr[s] + lane; p < ptr[s + 1]; p += 32) bad |= int64_t(lidx[p]) >= lim;
        if (wlen[t] == 0 && (s % kTliTile) == 0)
            for (int64_t k = uoff[t] + lane; k < uoff[t + 1]; k += 32) bad |= uidx[k] < 0 || uidx[k] >= n_dense;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 16);
}

int blocks_for(int64_t warps, int cap)
{
    int64_t b = (warps + 7) / 8;
    if (b < 1) b = 1;
    return int(b < cap ? b : cap);
}

}  // namespace

int tli_list_max_words() { return kMaxWords; }

void tli_check(const int64_t *ptr, int64_t nseg, const uint16_t *lidx, const int32_t *wlen, const int64_t *uoff,
               const int32_t *uidx, int64_t n_dense, int *flag, int sm_count, cudaStream_t st)
{
    k_check_lidx<<<blocks_for(nseg, sm_count * 8), kT, 0, st>>>(ptr, nseg, lidx, wlen, uoff, uidx, n_dense, flag);
}

void tli_tile_range(const int64_t *ptr, const int32_t *idx, int64_t nseg, int64_t ntiles, int32_t *tmin,
                    int32_t *tmax, cudaStream_t st)
{
    k_tile_range<<<blocks_for(ntiles, 65535), kT, 0, st>>>(ptr, idx, nseg, ntiles, tmin, tmax);
}

void tli_window_lidx(const int64_t *ptr, const int32_t *idx, int64_t nseg, const int32_t *wbase,
                     const int32_t *wlen, uint16_t *lidx, int sm_count, cudaStream_t st)
{
    k_window_lidx<<<blocks_for(nseg, sm_count * 8), kT, 0, st>>>(ptr, idx, nseg, wbase, wlen, lidx);
}

cudaError_t tli_list_count(const int64_t *ptr, const int32_t *idx, int64_t nseg, int64_t ntiles,
                           const int32_t *tmin, const int32_t *tmax, int max_words, int32_t *ucnt,
                           cudaStream_t st)
{
    const size_t smem = size_t(max_words) * 4;
    cudaError_t e = cudaFuncSetAttribute(k_list_count, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_list_count<<<unsigned(ntiles), kT, smem, st>>>(ptr, idx, nseg, tmin, tmax, max_words, ucnt);
    return cudaGetLastError();
}

cudaError_t tli_list_build(const int64_t *ptr, const int32_t *idx, int64_t nseg, int64_t ntiles,
                           const int32_t *tmin, const int32_t *tmax, const int32_t *wlen, int max_words,
                           const int64_t *uoff, int32_t *uidx, uint16_t *lidx, cudaStream_t st)
{
    const size_t smem = size_t(max_words) * 4 + size_t(max_words / 32 + 1) * 4;
    cudaError_t e = cudaFuncSetAttribute(k_list_build, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_list_build<<<unsigned(ntiles), kT, smem, st>>>(ptr, idx, nseg, tmin, tmax, wlen, max_words, uoff, uidx,
                                                    lidx);
    return cudaGetLastError();
}

}  // namespace sgtv
