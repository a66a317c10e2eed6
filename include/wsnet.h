/*
 * wsnet.h -- C ABI of the learned warm start for SGTV reconstruction
 * (part of libsgtv.so).
 *
 * The paper has no counterpart: its ADMM (Sec. III) starts from a flat image.
 * This network only proposes the starting image f0 of that iteration; plain
 * ADMM always finishes the solve and its objective judges the result. It maps
 * the normalised backprojection A^T y / A^T 1 (the q-bins as channels) plus
 * one channel holding the count level to an initial image with the same
 * shape.
 *
 * Architecture (3x3 convolutions, stride 1, zero padding; ReLU after every
 * convolution but the last; C = Q input/output channels):
 *   in  [C+1, H, W] -> conv1 C+1->64 -> conv2 64->64 (= s1)
 *   -> 2x2 average pool -> conv3 64->128 -> conv4 128->128 (= s2)
 *   -> 2x2 average pool -> conv5 128->256 -> conv6 256->128
 *   -> nearest 2x upsample, + s2 -> conv7 128->64
 *   -> nearest 2x upsample, + s1 -> conv8 64->64 -> conv9 64->C (1 + n_dual)
 *   (no ReLU) -> out: softplus(.) on the C image channels, the n_dual * C
 *   dual channels as they are.
 * About 1.03M parameters for C = 64 and n_dual = 0 (1.18M with n_dual = 4).
 * H and W must be multiples of 4.
 *
 * The optional dual channels predict the ADMM scaled dual c of the same scan
 * in units of the shrink threshold tau = beta / rho (one block of C channels
 * per neighbour direction, in the solver's direction order): an image alone
 * does not shorten the solve, because the dual restarts from zero and sets
 * the pace of convergence; a start that carries both does.
 *
 * Precision: FP32 master weights (Adam), BF16 copies used by every kernel,
 * FP32 activations and FP32 accumulation. Training loss: mean squared error
 * between `out` and a target, over all outputs of the batch.
 *
 * All device pointers are on the handle's device; NCHW layout
 * ([batch][channel][H][W], W fastest). Errors: SGTV_* codes of sgtv.h.
 */
#ifndef WSNET_H
#define WSNET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wsnet_ctx *wsnet_t;

/* Create a network for C = Q channels on H x W images, 0 <= n_dual <= 4 dual
 * blocks (Q * (1 + n_dual) <= 1024 outputs) and batches of up to max_batch
 * samples; weights He-initialised from `seed` (deterministic), biases 0;
 * stream: cudaStream_t (NULL = a stream the handle owns). */
int wsnet_create(wsnet_t *out, int32_t H, int32_t W, int32_t Q, int32_t n_dual, int32_t max_batch, uint64_t seed,
                 void *stream);
/* Output channels per sample, Q * (1 + n_dual). */
int32_t wsnet_num_outputs(wsnet_t h);
int wsnet_destroy(wsnet_t h);

/* Parameter count and the FP32 master parameters, packed layer by layer
 * (conv1 weights [64][C+1][3][3], conv1 bias [64], conv2 ..., conv9 bias). */
int64_t wsnet_num_params(wsnet_t h);
int wsnet_get_params(wsnet_t h, float *host);
int wsnet_set_params(wsnet_t h, const float *host);
/* Gradients of the last wsnet_loss_grad, same packing. */
int wsnet_get_grads(wsnet_t h, float *host);

/* out [N, Co, H, W] = network(x [N, C+1, H, W]), Co = wsnet_num_outputs;
 * 1 <= N <= max_batch. */
int wsnet_forward(wsnet_t h, const float *x, int32_t N, float *out);

/* Forward and backward pass on (x, target [N, Co, H, W]); writes the loss
 * (mean squared error, FP64 reduction) and leaves the gradients in the handle. */
int wsnet_loss_grad(wsnet_t h, const float *x, const float *target, int32_t N, double *loss);

/* One Adam step on the FP32 master weights from the current gradients
 * (bias-corrected, step count kept by the handle), then refresh the BF16 copies. */
int wsnet_adam_step(wsnet_t h, float lr, float beta1, float beta2, float eps);

/* Layout helpers between the reconstruction's hyper-voxel order
 * j = (x * Nz + z) * Nq + q and the network's [channel = q][H = x][W = z]:
 *   x_in [Nq + 1][Nx][Nz] = (bp / scale, then a constant channel `level`)
 *   f    [J] = scale * out[q][x][z]
 * Device pointers; run on `stream` (a cudaStream_t, NULL = legacy default). */
int wsnet_pack_input(const float *bp, int32_t Nx, int32_t Nz, int32_t Nq, float scale, float level, float *x_in,
                     void *stream);
int wsnet_unpack_output(const float *out, int32_t Nx, int32_t Nz, int32_t Nq, float scale, float *f, void *stream);
/* The dual channels of sample 0 in the solver's layout:
 *   c [p][J] = tau * out[Nq + p * Nq + q][x][z],  0 <= p < n_dual, j = (x * Nz + z) * Nq + q. */
int wsnet_unpack_dual(const float *out, int32_t Nx, int32_t Nz, int32_t Nq, int32_t n_dual, float tau, float *c,
                      void *stream);

const char *wsnet_last_error(wsnet_t h);

#ifdef __cplusplus
}
#endif

#endif /* WSNET_H */
