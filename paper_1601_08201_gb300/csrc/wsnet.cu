// wsnet.cu -- the learned warm start: a small encoder-decoder (include/wsnet.h)
// trained and run with hand-written kernels. BF16 weights, FP32 activations,
// FP32 accumulation; FP32 master weights updated by Adam.
//
// Convolutions are 3x3, stride 1, zero padding, computed as implicit GEMMs on
// the CUDA cores: a block owns 32 output channels x an 8 x 16 pixel tile of
// one sample, stages 16 input channels (with halo) and their weights in shared
// memory per step, and each thread accumulates 4 channels x 4 pixels. The
// data gradient is the same kernel on the flipped, channel-transposed weights;
// the weight gradient accumulates 16 x 16 (output, input) channel pairs over
// pixel tiles and adds its partial into the gradient buffer atomically.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <random>
#include <string>
#include <vector>

#include "../../include/sgtv.h"
#include "../../include/wsnet.h"

namespace {

constexpr int kT = 256;
constexpr int TC = 32, TH = 8, TW = 16, CK = 16;  // forward tile: channels, rows, columns, input chunk
constexpr int WC = 16, WI = 16;                    // weight-gradient tile: output x input channels

int blocks_for(int64_t n)
{
    int64_t b = (n + kT - 1) / kT;
    if (b > 8192) b = 8192;
    return int(b < 1 ? 1 : b);
}

template <bool RELU>
__global__ void __launch_bounds__(256)
k_conv_fwd(const float *__restrict__ x, const __nv_bfloat16 *__restrict__ w, const float *__restrict__ b,
           float *__restrict__ y, int Ci, int Co, int H, int W)
{
    __shared__ float xs[CK][TH + 2][TW + 3];
    __shared__ float ws[TC][CK * 9 + 1];
    const int tiles_w = (W + TW - 1) / TW;
    const int th0 = (blockIdx.x / tiles_w) * TH, tw0 = (blockIdx.x % tiles_w) * TW;
    const int co0 = blockIdx.y * TC;
    const int n = blockIdx.z;
    const int t = threadIdx.x;
    const int cg = t >> 5;  // warp: 4 output channels
    const int pg = t & 31;  // lane: 4 consecutive pixels of one row
    const int py = (pg * 4) / TW, px = (pg * 4) % TW;
    float acc[4][4];
#pragma unroll
    for (int o = 0; o < 4; o++)
#pragma unroll
        for (int p = 0; p < 4; p++) acc[o][p] = 0.f;
    const float *xn = x + size_t(n) * Ci * H * W;
    for (int ci0 = 0; ci0 < Ci; ci0 += CK) {
        for (int k = t; k < CK * (TH + 2) * (TW + 2); k += blockDim.x) {
            const int c = k / ((TH + 2) * (TW + 2)), r = k % ((TH + 2) * (TW + 2));
            const int yy = r / (TW + 2), xx = r % (TW + 2);
            const int gy = th0 + yy - 1, gx = tw0 + xx - 1, gc = ci0 + c;
            float v = 0.f;
            if (gc < Ci && gy >= 0 && gy < H && gx >= 0 && gx < W) v = xn[(size_t(gc) * H + gy) * W + gx];
            xs[c][yy][xx] = v;
        }
        for (int k = t; k < TC * CK * 9; k += blockDim.x) {
            const int co = k / (CK * 9), r = k % (CK * 9);
            const int c = r / 9, kk = r % 9;
            const int gco = co0 + co, gc = ci0 + c;
            float v = 0.f;
            if (gco < Co && gc < Ci) v = __bfloat162float(w[(size_t(gco) * Ci + gc) * 9 + kk]);
            ws[co][r] = v;
        }
        __syncthreads();
        const int cmax = Ci - ci0 < CK ? Ci - ci0 : CK;
        for (int c = 0; c < cmax; c++) {
#pragma unroll
            for (int kh = 0; kh < 3; kh++) {
                float xv[6];
#pragma unroll
                for (int q = 0; q < 6; q++) xv[q] = xs[c][py + kh][px + q];
#pragma unroll
                for (int kw = 0; kw < 3; kw++)
#pragma unroll
                    for (int o = 0; o < 4; o++) {
                        const float wv = ws[cg * 4 + o][c * 9 + kh * 3 + kw];
#pragma unroll
                        for (int p = 0; p < 4; p++) acc[o][p] = fmaf(wv, xv[p + kw], acc[o][p]);
                    }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 0; o < 4; o++) {
        const int co = co0 + cg * 4 + o;
        const int hh = th0 + py;
        if (co >= Co || hh >= H) continue;
        const float bias = b ? b[co] : 0.f;
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const int ww = tw0 + px + p;
            if (ww >= W) continue;
            float v = acc[o][p] + bias;
            if (RELU) v = v > 0.f ? v : 0.f;
            y[((size_t(n) * Co + co) * H + hh) * W + ww] = v;
        }
    }
}

// dw[co][ci][k] += sum over the block's pixels of dy[n][co][h][w] x[n][ci][h+kh-1][w+kw-1];
// db[co] += sum of dy (blocks of the first input-channel tile only).
__global__ void __launch_bounds__(256)
k_conv_bwd_w(const float *__restrict__ x, const float *__restrict__ dy, float *__restrict__ dw,
             float *__restrict__ db, int Ci, int Co, int H, int W)
{
    __shared__ float dys[WC][TH * TW + 1];
    __shared__ float xs[WI][(TH + 2) * (TW + 2) + 1];
    const int co0 = blockIdx.x * WC, ci0 = blockIdx.y * WI;
    const int tiles_h = (H + TH - 1) / TH;
    const int n = blockIdx.z / tiles_h;
    const int th0 = (blockIdx.z % tiles_h) * TH;
    const int t = threadIdx.x;
    const int col = t / WI, cil = t % WI;
    float acc[9];
#pragma unroll
    for (int k = 0; k < 9; k++) acc[k] = 0.f;
    float dbacc = 0.f;
    for (int tw0 = 0; tw0 < W; tw0 += TW) {
        for (int k = t; k < WC * TH * TW; k += blockDim.x) {
            const int c = k / (TH * TW), r = k % (TH * TW);
            const int hh = th0 + r / TW, ww = tw0 + r % TW, gc = co0 + c;
            float v = 0.f;
            if (gc < Co && hh < H && ww < W) v = dy[((size_t(n) * Co + gc) * H + hh) * W + ww];
            dys[c][r] = v;
        }
        for (int k = t; k < WI * (TH + 2) * (TW + 2); k += blockDim.x) {
            const int c = k / ((TH + 2) * (TW + 2)), r = k % ((TH + 2) * (TW + 2));
            const int gy = th0 + r / (TW + 2) - 1, gx = tw0 + r % (TW + 2) - 1, gc = ci0 + c;
            float v = 0.f;
            if (gc < Ci && gy >= 0 && gy < H && gx >= 0 && gx < W) v = x[((size_t(n) * Ci + gc) * H + gy) * W + gx];
            xs[c][r] = v;
        }
        __syncthreads();
        for (int p = 0; p < TH * TW; p++) {
            const float d = dys[col][p];
            const int py = p / TW, px = p % TW;
            dbacc += d;
#pragma unroll
            for (int kh = 0; kh < 3; kh++)
#pragma unroll
                for (int kw = 0; kw < 3; kw++) acc[kh * 3 + kw] = fmaf(d, xs[cil][(py + kh) * (TW + 2) + px + kw], acc[kh * 3 + kw]);
        }
        __syncthreads();
    }
    const int co = co0 + col, ci = ci0 + cil;
    if (co < Co && ci < Ci)
#pragma unroll
        for (int k = 0; k < 9; k++) atomicAdd(&dw[(size_t(co) * Ci + ci) * 9 + k], acc[k]);
    if (cil == 0 && blockIdx.y == 0 && co < Co) atomicAdd(&db[co], dbacc);
}

// wt[ci][co][kh][kw] = w[co][ci][2-kh][2-kw]: the data gradient as a forward convolution.
__global__ void k_flip_weights(const __nv_bfloat16 *__restrict__ w, __nv_bfloat16 *__restrict__ wt, int Ci, int Co)
{
    const int64_t n = int64_t(Ci) * Co * 9;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int kk = int(k % 9);
        const int64_t r = k / 9;
        const int co = int(r % Co), ci = int(r / Co);
        wt[k] = w[(int64_t(co) * Ci + ci) * 9 + (8 - kk)];
    }
}

__global__ void k_relu_bwd(float *__restrict__ g, const float *__restrict__ a, int64_t n)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        if (!(a[k] > 0.f)) g[k] = 0.f;
}

// y [NC][H/2][W/2] = 2x2 average of x [NC][H][W]; with accumulate, the backward adds into dx.
__global__ void k_pool_fwd(const float *__restrict__ x, float *__restrict__ y, int64_t NC, int H, int W)
{
    const int h2 = H / 2, w2 = W / 2;
    const int64_t n = NC * h2 * w2;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int ww = int(k % w2), hh = int((k / w2) % h2);
        const int64_t c = k / (int64_t(w2) * h2);
        const float *p = x + (c * H + 2 * hh) * W + 2 * ww;
        y[k] = 0.25f * (p[0] + p[1] + p[W] + p[W + 1]);
    }
}

__global__ void k_pool_bwd_add(const float *__restrict__ dy, float *__restrict__ dx, int64_t NC, int H, int W)
{
    const int64_t n = NC * H * W;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int ww = int(k % W), hh = int((k / W) % H);
        const int64_t c = k / (int64_t(W) * H);
        dx[k] += 0.25f * dy[(c * (H / 2) + hh / 2) * (W / 2) + ww / 2];
    }
}

// s [NC][2h][2w] = nearest upsample of a [NC][h][w] + skip.
__global__ void k_up_add(const float *__restrict__ a, const float *__restrict__ skip, float *__restrict__ s, int64_t NC,
                         int h, int w)
{
    const int H = 2 * h, W = 2 * w;
    const int64_t n = NC * H * W;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int ww = int(k % W), hh = int((k / W) % H);
        const int64_t c = k / (int64_t(W) * H);
        s[k] = a[(c * h + hh / 2) * w + ww / 2] + skip[k];
    }
}

// da [NC][h][w] = sum of the 4 gradients of its upsampled copies.
__global__ void k_up_bwd(const float *__restrict__ ds, float *__restrict__ da, int64_t NC, int h, int w)
{
    const int W = 2 * w;
    const int64_t n = NC * h * w;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int ww = int(k % w), hh = int((k / w) % h);
        const int64_t c = k / (int64_t(w) * h);
        const float *p = ds + (c * (2 * h) + 2 * hh) * W + 2 * ww;
        da[k] = p[0] + p[1] + p[W] + p[W + 1];
    }
}

__device__ __forceinline__ float softplus(float z) { return z > 20.f ? z : log1pf(expf(z)); }

// Output head: channel ch of a sample (ch = (k / HW) % Co) is the image's
// softplus(z) for ch < Q and z itself for the dual channels ch >= Q.
__global__ void k_head(const float *__restrict__ z, float *__restrict__ o, int64_t n, int64_t HW, int Co, int Q)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int ch = int((k / HW) % Co);
        o[k] = ch < Q ? softplus(z[k]) : z[k];
    }
}

// loss += sum (head(z) - t)^2 / n (FP64); dz = 2 (head(z) - t) head'(z) / n with
// head' = sigmoid on the image channels and 1 on the dual channels.
__global__ void k_mse_head(const float *__restrict__ z, const float *__restrict__ tgt, float *__restrict__ dz,
                           int64_t n, int64_t HW, int Co, int Q, double *__restrict__ loss)
{
    __shared__ double sh[32];
    double acc = 0.0;
    const float inv = 1.0f / float(n);
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float zz = z[k];
        const bool img = int((k / HW) % Co) < Q;
        const float diff = (img ? softplus(zz) : zz) - tgt[k];
        acc += double(diff) * double(diff);
        dz[k] = img ? 2.f * diff * inv / (1.f + expf(-zz)) : 2.f * diff * inv;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < int(blockDim.x >> 5); k++) s += sh[k];
        atomicAdd(loss, s / double(n));
    }
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       __nv_bfloat16 *__restrict__ wb, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        w[k] = wk;
        wb[k] = __float2bfloat16_rn(wk);
    }
}

__global__ void k_to_bf16(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, int64_t n)
{
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        wb[k] = __float2bfloat16_rn(w[k]);
}

__global__ void k_pack_input(const float *__restrict__ bp, int Nx, int Nz, int Nq, float inv_scale, float level,
                             float *__restrict__ x)
{
    const int64_t n = int64_t(Nq + 1) * Nx * Nz;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int zz = int(k % Nz), xx = int((k / Nz) % Nx), q = int(k / (int64_t(Nz) * Nx));
        x[k] = q < Nq ? bp[(int64_t(xx) * Nz + zz) * Nq + q] * inv_scale : level;
    }
}

__global__ void k_unpack_output(const float *__restrict__ o, int Nx, int Nz, int Nq, float scale, float *__restrict__ f)
{
    const int64_t n = int64_t(Nq) * Nx * Nz;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int q = int(k % Nq);
        const int64_t s = k / Nq;
        const int zz = int(s % Nz), xx = int(s / Nz);
        f[k] = scale * o[(int64_t(q) * Nx + xx) * Nz + zz];
    }
}

// c [p][J] = tau * out[Q + p * Q + q][x][z] (sample 0), p < n_dual.
__global__ void k_unpack_dual(const float *__restrict__ o, int Nx, int Nz, int Nq, int n_dual, float tau,
                              float *__restrict__ c)
{
    const int64_t J = int64_t(Nx) * Nz * Nq;
    const int64_t n = J * n_dual;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        const int p = int(k / J);
        const int64_t j = k - int64_t(p) * J;
        const int q = int(j % Nq);
        const int64_t s = j / Nq;
        const int zz = int(s % Nz), xx = int(s / Nz);
        c[k] = tau * o[((int64_t(Nq) * (1 + p) + q) * Nx + xx) * Nz + zz];
    }
}

struct Layer {
    int ci, co;
    int64_t woff, boff;  // offsets in the packed parameter vector
};

}  // namespace

struct wsnet_ctx {
    int H, W, C, maxN;
    int n_dual = 0, Co = 0;  // dual blocks of Q channels after the image's; output channels Q (1 + n_dual)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void *> blocks;
    Layer L[9];
    int64_t P = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr, *wt = nullptr;  // BF16 weights, flipped scratch
    // activations and gradients
    float *a1, *a2, *p1, *a3, *a4, *p2, *a5, *a6, *s1, *a7, *s2, *a8, *z;
    float *gz, *g8, *gs2, *g7, *gs1, *g6, *g5, *gp2, *g4, *g3, *gp1, *g2, *g1;
    double *loss = nullptr;
    int64_t step = 0;
    std::string err;
};

namespace {

int wfail(wsnet_t h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    return code;
}

#define WK(h, call)                                                                       \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return wfail(h, SGTV_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

void *walloc(wsnet_t h, size_t bytes)
{
    void *p = nullptr;
    if (cudaMalloc(&p, bytes < 16 ? 16 : bytes) != cudaSuccess) return nullptr;
    h->blocks.push_back(p);
    return p;
}

void conv_fwd(wsnet_t h, const float *x, int l, float *y, int N, int Hh, int Ww, bool relu)
{
    const Layer &L = h->L[l];
    dim3 grid(unsigned(((Hh + TH - 1) / TH) * ((Ww + TW - 1) / TW)), unsigned((L.co + TC - 1) / TC), unsigned(N));
    if (relu)
        k_conv_fwd<true><<<grid, kT, 0, h->stream>>>(x, h->wb + L.woff, h->w + L.boff, y, L.ci, L.co, Hh, Ww);
    else
        k_conv_fwd<false><<<grid, kT, 0, h->stream>>>(x, h->wb + L.woff, h->w + L.boff, y, L.ci, L.co, Hh, Ww);
}

// dy -> weight and bias gradients, and (if dx) the data gradient.
void conv_bwd(wsnet_t h, const float *x, const float *dy, int l, float *dx, int N, int Hh, int Ww)
{
    const Layer &L = h->L[l];
    dim3 gw(unsigned((L.co + WC - 1) / WC), unsigned((L.ci + WI - 1) / WI), unsigned(N * ((Hh + TH - 1) / TH)));
    k_conv_bwd_w<<<gw, kT, 0, h->stream>>>(x, dy, h->g + L.woff, h->g + L.boff, L.ci, L.co, Hh, Ww);
    if (dx) {
        k_flip_weights<<<blocks_for(int64_t(L.ci) * L.co * 9), kT, 0, h->stream>>>(h->wb + L.woff, h->wt, L.ci, L.co);
        dim3 grid(unsigned(((Hh + TH - 1) / TH) * ((Ww + TW - 1) / TW)), unsigned((L.ci + TC - 1) / TC), unsigned(N));
        k_conv_fwd<false><<<grid, kT, 0, h->stream>>>(dy, h->wt, nullptr, dx, L.co, L.ci, Hh, Ww);
    }
}

void relu_bwd(wsnet_t h, float *g, const float *a, int64_t n)
{
    k_relu_bwd<<<blocks_for(n), kT, 0, h->stream>>>(g, a, n);
}

// The forward pass up to z (pre-softplus output).
void forward_to_z(wsnet_t h, const float *x, int N)
{
    const int H = h->H, W = h->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    cudaStream_t st = h->stream;
    conv_fwd(h, x, 0, h->a1, N, H, W, true);
    conv_fwd(h, h->a1, 1, h->a2, N, H, W, true);
    k_pool_fwd<<<blocks_for(int64_t(N) * 64 * H2 * W2), kT, 0, st>>>(h->a2, h->p1, int64_t(N) * 64, H, W);
    conv_fwd(h, h->p1, 2, h->a3, N, H2, W2, true);
    conv_fwd(h, h->a3, 3, h->a4, N, H2, W2, true);
    k_pool_fwd<<<blocks_for(int64_t(N) * 128 * H4 * W4), kT, 0, st>>>(h->a4, h->p2, int64_t(N) * 128, H2, W2);
    conv_fwd(h, h->p2, 4, h->a5, N, H4, W4, true);
    conv_fwd(h, h->a5, 5, h->a6, N, H4, W4, true);
    k_up_add<<<blocks_for(int64_t(N) * 128 * H2 * W2), kT, 0, st>>>(h->a6, h->a4, h->s1, int64_t(N) * 128, H4, W4);
    conv_fwd(h, h->s1, 6, h->a7, N, H2, W2, true);
    k_up_add<<<blocks_for(int64_t(N) * 64 * H * W), kT, 0, st>>>(h->a7, h->a2, h->s2, int64_t(N) * 64, H2, W2);
    conv_fwd(h, h->s2, 7, h->a8, N, H, W, true);
    conv_fwd(h, h->a8, 8, h->z, N, H, W, false);
}

}  // namespace

extern "C" {

int wsnet_create(wsnet_t *out, int32_t H, int32_t W, int32_t Q, int32_t n_dual, int32_t max_batch, uint64_t seed,
                 void *stream)
{
    if (!out) return SGTV_ERR_ARG;
    *out = nullptr;
    if (H < 4 || W < 4 || H % 4 || W % 4 || Q < 1 || max_batch < 1 || n_dual < 0 || n_dual > 4 ||
        int64_t(Q) * (1 + n_dual) > 1024)
        return SGTV_ERR_ARG;
    wsnet_t h = new wsnet_ctx();
    h->H = H;
    h->W = W;
    h->C = Q;
    h->n_dual = n_dual;
    h->Co = Q * (1 + n_dual);
    h->maxN = max_batch;
    const int ch[9][2] = {{Q + 1, 64}, {64, 64}, {64, 128}, {128, 128}, {128, 256},
                          {256, 128}, {128, 64}, {64, 64}, {64, h->Co}};
    int64_t off = 0;
    for (int l = 0; l < 9; l++) {
        h->L[l].ci = ch[l][0];
        h->L[l].co = ch[l][1];
        h->L[l].woff = off;
        off += int64_t(ch[l][0]) * ch[l][1] * 9;
        h->L[l].boff = off;
        off += ch[l][1];
    }
    h->P = off;
    auto fail_create = [&](int code) {
        for (void *p : h->blocks) cudaFree(p);
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        delete h;
        return code;
    };
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return fail_create(SGTV_ERR_CUDA);
        h->own_stream = true;
    }
    const size_t P = size_t(h->P);
    h->w = static_cast<float *>(walloc(h, 4 * P));
    h->g = static_cast<float *>(walloc(h, 4 * P));
    h->m = static_cast<float *>(walloc(h, 4 * P));
    h->v = static_cast<float *>(walloc(h, 4 * P));
    h->wb = static_cast<__nv_bfloat16 *>(walloc(h, 2 * P));
    h->wt = static_cast<__nv_bfloat16 *>(walloc(h, 2 * size_t(256) * (h->Co > 256 ? h->Co : 256) * 9));
    h->loss = static_cast<double *>(walloc(h, sizeof(double)));
    const size_t N = size_t(max_batch);
    const size_t f1 = N * H * W, f2 = N * (H / 2) * (W / 2), f4 = N * (H / 4) * (W / 4);
    const int Cz = h->Co > 64 ? h->Co : 64;
    float **bufs[] = {&h->a1, &h->a2, &h->s2, &h->a8, &h->g8, &h->gs2, &h->g2, &h->g1};
    for (float **b : bufs) *b = static_cast<float *>(walloc(h, 4 * f1 * 64));
    h->z = static_cast<float *>(walloc(h, 4 * f1 * Cz));
    h->gz = static_cast<float *>(walloc(h, 4 * f1 * Cz));
    float **b2[] = {&h->p1, &h->a7, &h->g7, &h->gp1};
    for (float **b : b2) *b = static_cast<float *>(walloc(h, 4 * f2 * 64));
    float **b3[] = {&h->a3, &h->a4, &h->s1, &h->gs1, &h->g4, &h->g3};
    for (float **b : b3) *b = static_cast<float *>(walloc(h, 4 * f2 * 128));
    float **b4[] = {&h->p2, &h->a6, &h->g6, &h->gp2};
    for (float **b : b4) *b = static_cast<float *>(walloc(h, 4 * f4 * 128));
    h->a5 = static_cast<float *>(walloc(h, 4 * f4 * 256));
    h->g5 = static_cast<float *>(walloc(h, 4 * f4 * 256));
    for (void *p : h->blocks)
        if (!p) return fail_create(SGTV_ERR_OOM);
    if (h->blocks.size() != 7 + 8 + 2 + 4 + 6 + 4 + 2) return fail_create(SGTV_ERR_OOM);
    // He initialisation (normal, std sqrt(2 / fan_in)), deterministic from seed; biases 0
    std::vector<float> hw(P, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 9; l++) {
        std::normal_distribution<float> nd(0.f, sqrtf(2.f / float(h->L[l].ci * 9)) * (l == 8 ? 0.1f : 1.f));
        for (int64_t k = 0; k < int64_t(h->L[l].ci) * h->L[l].co * 9; k++) hw[h->L[l].woff + k] = nd(rng);
    }
    if (wsnet_set_params(h, hw.data()) != SGTV_OK) return fail_create(SGTV_ERR_CUDA);
    *out = h;
    return SGTV_OK;
}

int wsnet_destroy(wsnet_t h)
{
    if (!h) return SGTV_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void *p : h->blocks) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return SGTV_OK;
}

int64_t wsnet_num_params(wsnet_t h) { return h ? h->P : 0; }

int wsnet_set_params(wsnet_t h, const float *host)
{
    if (!h || !host) return SGTV_ERR_ARG;
    const size_t P = size_t(h->P);
    WK(h, cudaMemcpyAsync(h->w, host, 4 * P, cudaMemcpyHostToDevice, h->stream));
    WK(h, cudaMemsetAsync(h->m, 0, 4 * P, h->stream));
    WK(h, cudaMemsetAsync(h->v, 0, 4 * P, h->stream));
    WK(h, cudaMemsetAsync(h->g, 0, 4 * P, h->stream));
    k_to_bf16<<<blocks_for(h->P), kT, 0, h->stream>>>(h->w, h->wb, h->P);
    WK(h, cudaGetLastError());
    WK(h, cudaStreamSynchronize(h->stream));
    h->step = 0;
    return SGTV_OK;
}

int wsnet_get_params(wsnet_t h, float *host)
{
    if (!h || !host) return SGTV_ERR_ARG;
    WK(h, cudaMemcpyAsync(host, h->w, 4 * size_t(h->P), cudaMemcpyDeviceToHost, h->stream));
    WK(h, cudaStreamSynchronize(h->stream));
    return SGTV_OK;
}

int wsnet_get_grads(wsnet_t h, float *host)
{
    if (!h || !host) return SGTV_ERR_ARG;
    WK(h, cudaMemcpyAsync(host, h->g, 4 * size_t(h->P), cudaMemcpyDeviceToHost, h->stream));
    WK(h, cudaStreamSynchronize(h->stream));
    return SGTV_OK;
}

int wsnet_forward(wsnet_t h, const float *x, int32_t N, float *out)
{
    if (!h || !x || !out) return SGTV_ERR_ARG;
    if (N < 1 || N > h->maxN) return wfail(h, SGTV_ERR_ARG, "N must be in [1, max_batch]");
    forward_to_z(h, x, N);
    const int64_t HW = int64_t(h->H) * h->W;
    const int64_t n = int64_t(N) * h->Co * HW;
    k_head<<<blocks_for(n), kT, 0, h->stream>>>(h->z, out, n, HW, h->Co, h->C);
    WK(h, cudaGetLastError());
    return SGTV_OK;
}

int wsnet_loss_grad(wsnet_t h, const float *x, const float *target, int32_t N, double *loss)
{
    if (!h || !x || !target) return SGTV_ERR_ARG;
    if (N < 1 || N > h->maxN) return wfail(h, SGTV_ERR_ARG, "N must be in [1, max_batch]");
    const int H = h->H, W = h->W, H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4;
    cudaStream_t st = h->stream;
    forward_to_z(h, x, N);
    WK(h, cudaMemsetAsync(h->g, 0, 4 * size_t(h->P), st));
    WK(h, cudaMemsetAsync(h->loss, 0, sizeof(double), st));
    const int64_t nz = int64_t(N) * h->Co * H * W;
    k_mse_head<<<blocks_for(nz), kT, 0, st>>>(h->z, target, h->gz, nz, int64_t(H) * W, h->Co, h->C, h->loss);
    const int64_t n64 = int64_t(N) * 64 * H * W, n64h = int64_t(N) * 64 * H2 * W2, n128h = int64_t(N) * 128 * H2 * W2;
    const int64_t n128q = int64_t(N) * 128 * H4 * W4, n256q = int64_t(N) * 256 * H4 * W4;
    conv_bwd(h, h->a8, h->gz, 8, h->g8, N, H, W);
    relu_bwd(h, h->g8, h->a8, n64);
    conv_bwd(h, h->s2, h->g8, 7, h->gs2, N, H, W);
    // s2 = up(a7) + a2
    WK(h, cudaMemcpyAsync(h->g2, h->gs2, 4 * size_t(n64), cudaMemcpyDeviceToDevice, st));
    k_up_bwd<<<blocks_for(n64h), kT, 0, st>>>(h->gs2, h->g7, int64_t(N) * 64, H2, W2);
    relu_bwd(h, h->g7, h->a7, n64h);
    conv_bwd(h, h->s1, h->g7, 6, h->gs1, N, H2, W2);
    // s1 = up(a6) + a4
    WK(h, cudaMemcpyAsync(h->g4, h->gs1, 4 * size_t(n128h), cudaMemcpyDeviceToDevice, st));
    k_up_bwd<<<blocks_for(n128q), kT, 0, st>>>(h->gs1, h->g6, int64_t(N) * 128, H4, W4);
    relu_bwd(h, h->g6, h->a6, n128q);
    conv_bwd(h, h->a5, h->g6, 5, h->g5, N, H4, W4);
    relu_bwd(h, h->g5, h->a5, n256q);
    conv_bwd(h, h->p2, h->g5, 4, h->gp2, N, H4, W4);
    k_pool_bwd_add<<<blocks_for(n128h), kT, 0, st>>>(h->gp2, h->g4, int64_t(N) * 128, H2, W2);
    relu_bwd(h, h->g4, h->a4, n128h);
    conv_bwd(h, h->a3, h->g4, 3, h->g3, N, H2, W2);
    relu_bwd(h, h->g3, h->a3, n128h);
    conv_bwd(h, h->p1, h->g3, 2, h->gp1, N, H2, W2);
    k_pool_bwd_add<<<blocks_for(n64), kT, 0, st>>>(h->gp1, h->g2, int64_t(N) * 64, H, W);
    relu_bwd(h, h->g2, h->a2, n64);
    conv_bwd(h, h->a1, h->g2, 1, h->g1, N, H, W);
    relu_bwd(h, h->g1, h->a1, n64);
    conv_bwd(h, x, h->g1, 0, nullptr, N, H, W);
    WK(h, cudaGetLastError());
    if (loss) {
        WK(h, cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        WK(h, cudaStreamSynchronize(st));
    }
    return SGTV_OK;
}

int wsnet_adam_step(wsnet_t h, float lr, float beta1, float beta2, float eps)
{
    if (!h) return SGTV_ERR_ARG;
    h->step += 1;
    const float c1 = 1.f - powf(beta1, float(h->step)), c2 = 1.f - powf(beta2, float(h->step));
    k_adam<<<blocks_for(h->P), kT, 0, h->stream>>>(h->w, h->g, h->m, h->v, h->wb, h->P, lr, beta1, beta2, eps, c1, c2);
    WK(h, cudaGetLastError());
    return SGTV_OK;
}

int wsnet_pack_input(const float *bp, int32_t Nx, int32_t Nz, int32_t Nq, float scale, float level, float *x_in,
                     void *stream)
{
    if (!bp || !x_in || Nx < 1 || Nz < 1 || Nq < 1 || !(scale > 0.f)) return SGTV_ERR_ARG;
    k_pack_input<<<blocks_for(int64_t(Nq + 1) * Nx * Nz), kT, 0, static_cast<cudaStream_t>(stream)>>>(
        bp, Nx, Nz, Nq, 1.f / scale, level, x_in);
    return cudaGetLastError() == cudaSuccess ? SGTV_OK : SGTV_ERR_CUDA;
}

int wsnet_unpack_output(const float *out, int32_t Nx, int32_t Nz, int32_t Nq, float scale, float *f, void *stream)
{
    if (!out || !f || Nx < 1 || Nz < 1 || Nq < 1) return SGTV_ERR_ARG;
    k_unpack_output<<<blocks_for(int64_t(Nq) * Nx * Nz), kT, 0, static_cast<cudaStream_t>(stream)>>>(out, Nx, Nz, Nq,
                                                                                                     scale, f);
    return cudaGetLastError() == cudaSuccess ? SGTV_OK : SGTV_ERR_CUDA;
}

int wsnet_unpack_dual(const float *out, int32_t Nx, int32_t Nz, int32_t Nq, int32_t n_dual, float tau, float *c,
                      void *stream)
{
    if (!out || !c || Nx < 1 || Nz < 1 || Nq < 1 || n_dual < 1 || n_dual > 4 || !(tau >= 0.f)) return SGTV_ERR_ARG;
    k_unpack_dual<<<blocks_for(int64_t(Nq) * Nx * Nz * n_dual), kT, 0, static_cast<cudaStream_t>(stream)>>>(
        out, Nx, Nz, Nq, n_dual, tau, c);
    return cudaGetLastError() == cudaSuccess ? SGTV_OK : SGTV_ERR_CUDA;
}

int32_t wsnet_num_outputs(wsnet_t h) { return h ? h->Co : 0; }

const char *wsnet_last_error(wsnet_t h) { return h ? h->err.c_str() : ""; }

}  // extern "C"
