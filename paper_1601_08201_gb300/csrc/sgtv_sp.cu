// sgtv_sp.cu -- set-up of the single-pass row stream.
//
// The single-pass iteration streams A once per surrogate step, by rows: each
// warp reduces a row against the tile's staged f, forms the row's ratio and
// adds a_ij * ratio_i into its shared-memory accumulator at the same local
// indices. Every element thus costs three shared-memory accesses (gather,
// accumulator read, accumulator write), and the 32 lanes of one access
// instruction collide whenever their local indices share a bank (index mod
// 32). In the stored order about three such collisions stack up per
// instruction. This stream stores the tiled CSR form again so that they
// mostly do not:
//   * each row is padded to a multiple of 4 elements, so rows start
//     4-aligned and a lane's 4-element chunk (one 8-byte index load, one
//     16-byte FP32 value load) never straddles two rows; padding slots carry
//     value 0 and a dummy local index (the tile's staging size, one past its
//     last staged value, held at 0 in shared memory);
//   * within each row the elements are dealt out to the access instructions
//     by bank: sorted by bank (stable), element t of that order goes to
//     instruction (chunk u, element m) = group t mod G of the row's G = 4 *
//     chunks groups, lane t div G -- a bank holding h elements of the row then
//     appears at most ceil(h / G) times in any one instruction.
// Only the order of a row's terms changes (the product rounds differently,
// the iteration is the same). Layout of row i: elements at rp[i] + 128 u +
// 4 k + m (lane k, chunk u, element m), rp[i] a multiple of 4.
#include <stdint.h>

#include "sgtv_internal.h"

namespace sgtv {

namespace {

constexpr int kT = 256;

// Position inside a padded row of n4 elements (a multiple of 4) of the
// element with rank t in the row's bank order (the dealing described above).
__device__ __forceinline__ int dealt_slot(int t, int n4)
{
    const int nch = (n4 + 127) >> 7;
    const int G = 4 * nch;                       // access groups (chunk, element)
    const int R4 = (n4 - 128 * (nch - 1)) >> 2;  // lanes holding the last chunk
    int k, g;
    if (t < R4 * G) {
        k = t / G;
        g = t - k * G;
    } else {  // lanes R4..31 hold only the full chunks
        const int tp = t - R4 * G;
        k = R4 + tp / (G - 4);
        g = tp - (k - R4) * (G - 4);
    }
    return 128 * (g >> 2) + 4 * k + (g & 3);
}

template <typename VB>
__global__ void __launch_bounds__(kT)
k_sp_build(int64_t I, const int64_t *__restrict__ rowptr, const uint16_t *__restrict__ lidx,
           const VB *__restrict__ val, const int64_t *__restrict__ sp_rp, const int32_t *__restrict__ wlen,
           const int64_t *__restrict__ uoff, uint16_t *__restrict__ sp_lidx, VB *__restrict__ sp_val)
{
    __shared__ int hist[kT / 32][32], used[kT / 32][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < I; i += nwarps) {
        const int64_t src = rowptr[i], dst = sp_rp[i];
        const int n = int(rowptr[i + 1] - src), n4 = int(sp_rp[i + 1] - dst);
        const int64_t t = i / kTliTile;
        const uint16_t dummy = uint16_t(wlen[t] > 0 ? wlen[t] : int(uoff[t + 1] - uoff[t]));
        hist[w][lane] = 0;
        used[w][lane] = 0;
        __syncwarp();
        for (int k = lane; k < n; k += 32) atomicAdd(&hist[w][lidx[src + k] & 31], 1);
        __syncwarp();
        // exclusive scan of the bank counts: lane b holds the first rank of bank b
        int off = hist[w][lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, off, o);
            if (lane >= o) off += v;
        }
        off -= hist[w][lane];
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const bool act = k < n;
            const uint16_t li = act ? lidx[src + k] : uint16_t(0);
            const int b = li & 31;
            const int first = __shfl_sync(0xffffffffu, off, b);
            const unsigned peers = __match_any_sync(0xffffffffu, act ? b : 32 + lane);
            const int before = used[w][b];
            __syncwarp();
            if (act) {
                const int rank = first + before + __popc(peers & lt);
                const int pos = dealt_slot(rank, n4);
                sp_lidx[dst + pos] = li;
                sp_val[dst + pos] = val[src + k];
                if ((peers & lt) == 0u) used[w][b] = before + __popc(peers);  // the group's first lane
            }
            __syncwarp();
        }
        for (int k = n + lane; k < n4; k += 32) {  // padding: ranks n .. n4 - 1
            const int pos = dealt_slot(k, n4);
            sp_lidx[dst + pos] = dummy;
            sp_val[dst + pos] = VB(0);
        }
        __syncwarp();
    }
}

// The stream must be a padded permutation of each row: per row, the sums of
// the local indices and of the values' bit patterns (as integers) match the
// tiled CSR form's, every padding slot counted as the dummy index and zero
// bits, and no index exceeds the dummy. Sets flag bit 32 otherwise.
template <typename VB>
__global__ void __launch_bounds__(kT)
k_sp_check(int64_t I, const int64_t *__restrict__ rowptr, const uint16_t *__restrict__ lidx,
           const VB *__restrict__ val, const int64_t *__restrict__ sp_rp, const int32_t *__restrict__ wlen,
           const int64_t *__restrict__ uoff, const uint16_t *__restrict__ sp_lidx, const VB *__restrict__ sp_val,
           int *__restrict__ flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    bool bad = false;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < I; i += nwarps) {
        const int64_t src = rowptr[i], dst = sp_rp[i];
        const int n = int(rowptr[i + 1] - src), n4 = int(sp_rp[i + 1] - dst);
        const int64_t t = i / kTliTile;
        const int dummy = wlen[t] > 0 ? wlen[t] : int(uoff[t + 1] - uoff[t]);
        unsigned long long a = 0, b = 0, va = 0, vb = 0;
        for (int k = lane; k < n; k += 32) {
            a += lidx[src + k];
            va += (unsigned long long)val[src + k];
        }
        for (int k = lane; k < n4; k += 32) {
            const int li = sp_lidx[dst + k];
            bad |= li > dummy;
            b += (unsigned long long)li;
            vb += (unsigned long long)sp_val[dst + k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            va += __shfl_xor_sync(0xffffffffu, va, o);
            vb += __shfl_xor_sync(0xffffffffu, vb, o);
        }
        bad |= (n4 != ((n + 3) & ~3)) || (b != a + (unsigned long long)(n4 - n) * dummy) || (va != vb);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 32);
}

int grid_rows(int64_t rows, int sm_count)
{
    int64_t b = (rows + kT / 32 - 1) / (kT / 32);
    const int64_t cap = int64_t(sm_count) * 16;
    if (b < 1) b = 1;
    return int(b < cap ? b : cap);
}

template <typename VB>
void build_typed(int64_t I, const int64_t *rowptr, const uint16_t *lidx, const void *val, const int64_t *sp_rp,
                 const int32_t *wlen, const int64_t *uoff, uint16_t *sp_lidx, void *sp_val, int *flag,
                 int sm_count, cudaStream_t st)
{
    const int grid = grid_rows(I, sm_count);
    k_sp_build<VB><<<grid, kT, 0, st>>>(I, rowptr, lidx, static_cast<const VB *>(val), sp_rp, wlen, uoff, sp_lidx,
                                        static_cast<VB *>(sp_val));
    k_sp_check<VB><<<grid, kT, 0, st>>>(I, rowptr, lidx, static_cast<const VB *>(val), sp_rp, wlen, uoff, sp_lidx,
                                        static_cast<const VB *>(sp_val), flag);
}

}  // namespace

cudaError_t sp_build(int64_t I, const int64_t *rowptr, const uint16_t *lidx, const void *val, int val_bytes,
                     const int64_t *sp_rp, const int32_t *wlen, const int64_t *uoff, uint16_t *sp_lidx, void *sp_val,
                     int *flag, int sm_count, cudaStream_t st)
{
    if (I < 1) return cudaSuccess;
    if (val_bytes == 2)
        build_typed<uint16_t>(I, rowptr, lidx, val, sp_rp, wlen, uoff, sp_lidx, sp_val, flag, sm_count, st);
    else if (val_bytes == 4)
        build_typed<uint32_t>(I, rowptr, lidx, val, sp_rp, wlen, uoff, sp_lidx, sp_val, flag, sm_count, st);
    else
        build_typed<unsigned long long>(I, rowptr, lidx, val, sp_rp, wlen, uoff, sp_lidx, sp_val, flag, sm_count,
                                        st);
    return cudaGetLastError();
}

}  // namespace sgtv
