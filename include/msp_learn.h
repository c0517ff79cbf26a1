/*
 * msp_learn.h -- C ABI of the learned-proposal form of libmsp: an extension of the method of
 * arXiv 2205.03902, which itself has no learned component.
 *
 * A small convolutional network proposes an update of every slice potential from the current
 * potentials and their gradients; the proposal is kept only if the true multislice loss of
 * Sec. 3.2 drops (evaluated with msp_loss_grad), otherwise the plain method's step is taken.
 *
 * The network: six 3 x 3 convolutions (stride 1, zero padding 1), c_in = 2L -> 64 -> 64 -> 64
 * -> 64 -> 64 -> L, GELU (0.5 x (1 + erf(x / sqrt 2))) after all but the last, a bias per output
 * channel.  Input channels: [s_V V_1 .. s_V V_L, s_G dL/dV_1 .. s_G dL/dV_L]; output: the
 * proposed change of the potentials divided by s_D.  Weights and activations are BF16, every
 * convolution accumulates in FP32 on the tensor cores (tcgen05, kind::f16, implicit GEMM: the
 * 3 x 3 x c_in patch of each pixel is gathered on chip, never materialised), the master
 * weights and the Adam moments are FP32.
 *
 * Parameters: one FP32 array of msp_net_param_count entries, layer after layer, each layer's
 * weights [c_out][9][c_in] (tap t = 3 (dy + 1) + (dx + 1)) followed by its biases [c_out].
 * Images: the object frame of the slices, row-major planes [L][height][width], FP32.
 * Conventions, ownership and errors as in msp.h: device pointers owned by the caller, a caller
 * workspace (256-byte aligned, one call at a time), asynchronous calls on `stream`, status codes,
 * no allocation.  The tensor-core waits are bounded (msp_set_wait_limit); a wait that runs out is
 * reported by msp_check_workspace on the same workspace (MSP_ETIMEOUT, or MSP_EDEVICE), as for
 * the calls of msp.h.
 */
#ifndef MSP_LEARN_H
#define MSP_LEARN_H

#include <stddef.h>
#include <stdint.h>

#include "msp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n_slices;   /* L, 1 .. 8 (2L input channels, padded to 16)                 */
  int32_t height;     /* object rows, >= 1                                            */
  int32_t width;      /* object columns, a multiple of 128                            */
  double scale_v;     /* s_V: input scale of the potentials                           */
  double scale_g;     /* s_G: input scale of the gradients                            */
  double scale_d;     /* s_D: output scale (proposed change = s_D x network output)   */
} msp_net_shape;

/* Checks a shape on the host: MSP_OK, MSP_EINVAL or MSP_EUNSUPPORTED. */
msp_status msp_net_validate(const msp_net_shape* s);

/* FP32 parameters of the network (weights and biases of the six layers). */
size_t msp_net_param_count(const msp_net_shape* s);

/* Workspace bytes of msp_net_forward / msp_net_train_step (0 if the shape is invalid). */
size_t msp_net_workspace_bytes(const msp_net_shape* s);

/* Deterministic initialisation: weights uniform in +-sqrt(6 / (9 c_in + 9 c_out)) (last layer
 * scaled by 0.1) from a counter-based hash of (seed, index), biases 0; Adam moments must be
 * zeroed by the caller. */
msp_status msp_net_init(const msp_net_shape* s, float* params, uint64_t seed, void* stream);

/* Proposal: dV_prop [L][height][width] = s_D x net(s_V V, s_G G). */
msp_status msp_net_forward(const msp_net_shape* s, const float* params, const float* V, const float* G,
                           float* dV_prop, void* ws, size_t ws_bytes, void* stream);

/* Loss of the proposal against `target` [L][height][width] (FP32),
 *   loss = mean over the L x height x width values of (dV_prop - target)^2 / s_D^2,
 * and its gradient with respect to the parameters: grad (FP32, msp_net_param_count entries, the
 * parameter layout); loss_out (device double, may be NULL).  The BF16 storage points of the
 * forward pass stay, and the gradient of every pre-activation is stored in BF16 as well; the
 * rounding of the activations counts as the identity in the chain rule. */
msp_status msp_net_loss_grad(const msp_net_shape* s, const float* params, const float* V, const float* G,
                             const float* target, float* grad, double* loss_out, void* ws, size_t ws_bytes,
                             void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, `step` >= 1 counts the steps taken) on the
 * gradient of msp_net_loss_grad:
 *   m = 0.9 m + 0.1 g,  v = 0.999 v + 0.001 g^2,  p -= lr (m / (1 - 0.9^step)) / (sqrt(v / (1 - 0.999^step)) + 1e-8).
 * params, adam_m, adam_v (FP32, msp_net_param_count entries) are updated in place; loss_out
 * (device double, may be NULL) receives the loss before the step. */
msp_status msp_net_train_step(const msp_net_shape* s, float* params, float* adam_m, float* adam_v, int32_t step,
                              double lr, const float* V, const float* G, const float* target, double* loss_out,
                              void* ws, size_t ws_bytes, void* stream);

/* Scratch of msp_learned_propose: the network's workspace and three [L][Ny][Nx] planes (the
 * gradient, the proposal, the candidate).  0 if g and s are invalid or disagree. */
size_t msp_learned_workspace_bytes(const msp_geometry* g, const msp_net_shape* s);

/* One proposal under the acceptance rule, all on `stream` without a host synchronisation:
 *   loss[0] = L(V), G = dL/dV                         (msp_loss_grad, Sec. 3.2)
 *   Vc = V + msp_net_forward(V, G)
 *   loss[1] = L(Vc)                                   (msp_loss_grad, loss only)
 *   if loss[1] < loss[0]: V <- Vc, *accepted = 1; else V unchanged, *accepted = 0.
 * The caller takes the plain method's step (msp_layer_step / msp_reconstruct) when the proposal
 * is rejected.  s must match g (n_slices = L, height = obj_ny, width = obj_nx), potential mode.
 *   loss      device double [2];  accepted device int32 [1] (may be NULL)
 *   ws        the msp_loss_grad workspace of g (msp_workspace_bytes)
 *   learn_ws  msp_learned_workspace_bytes bytes, 256-byte aligned; msp_check_workspace on it
 *             reports the network's tensor-core waits, on ws those of the multislice calls. */
msp_status msp_learned_propose(const msp_geometry* g, const msp_net_shape* s, const float* params,
                               const float* probe, float* V, const int32_t* pos, const float* I_meas,
                               int32_t* accepted, double* loss, void* ws, size_t ws_bytes, void* learn_ws,
                               size_t learn_ws_bytes, void* stream);

/* Test hooks of the building blocks, on NHWC BF16 images of `height` x `width` pixels:
 * the 3 x 3 convolution out = conv(in) + bias (pre-activation, FP32 NHWC [h][w][c_out]) for
 * c_in, c_out in {16, 64}, and the gradient of the weights and biases of that convolution from
 * the gradient of its pre-activation (grad_pre, BF16 NHWC): dW [c_out][9][c_in], db [c_out] (FP32).
 * `w` is FP32 [c_out][9][c_in]; both run the kernels msp_net_train_step uses. */
msp_status msp_conv3x3_test(int32_t height, int32_t width, int32_t c_in, int32_t c_out, const void* in_bf16,
                            const float* w, const float* bias, float* pre_out, void* ws, size_t ws_bytes,
                            void* stream);
msp_status msp_conv3x3_wgrad_test(int32_t height, int32_t width, int32_t c_in, int32_t c_out, const void* in_bf16,
                                  const void* grad_pre_bf16, float* dW, float* db, void* ws, size_t ws_bytes,
                                  void* stream);
size_t msp_conv3x3_test_workspace_bytes(int32_t height, int32_t width, int32_t c_in, int32_t c_out);

#ifdef __cplusplus
}
#endif

#endif /* MSP_LEARN_H */
