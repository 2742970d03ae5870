/*
 * nrmg_net.h -- the learned initial guess: a small convolutional network, its training, and
 * the field-level glue between the network and the solver of nrmg.h.
 *
 * The paper has no counterpart: the paper's solver starts from the global Maxwellian
 * (Sec. 4).  This library adds a start that a network predicts from a solution on the grid
 * twice as coarse, and keeps the plain FAS cycle of Algorithm 2 as the solver: it takes the
 * predicted state to the same discrete fixed point, and the caller keeps the unaided start
 * when the network's start has the larger residual after the same number of FAS cycles.  The field layout is that of
 * nrmg_fields (the Grad fields of eq. moments-relation).
 *
 * Network: four 3x3 "same" convolutions (zero padding), channels cin -> hidden -> hidden ->
 * hidden -> cout, ReLU after the first three.  Activations are stored NHWC in BF16 with the
 * channel count padded to a multiple of 16; weights are BF16 copies of FP32 master weights;
 * every product accumulates in FP32 on the tensor cores (mma.sync m16n8k16, BF16).  The
 * backward pass rounds each layer's output gradient to BF16 before it meets the tensor
 * cores; bias gradients sum those BF16 values in FP32.
 *
 * Arrays are device memory unless stated.  Images are [B][H][W][channels] row-major:
 * inputs x with cin FP32 channels, targets and outputs with cout FP32 channels.  Parameters
 * are one flat FP32 array: for each layer l = 0..3 the weights [9][co_l][ci_l] (tap
 * t = 3 (dy + 1) + (dx + 1) multiplies the input pixel (h + dy, w + dx)) followed by the biases
 * [co_l], where ci_0 = 16, 32 or 64 (the smallest that holds cin), co_3 = 16 and every
 * other count is `hidden`;
 * entries of padded channels are zero and stay zero.  All work runs on the stream given at
 * creation; calls that return host scalars synchronize it.  The caller owns the workspace
 * (256-byte aligned, at least nrmg_net_workspace_bytes).  Status codes are those of nrmg.h:
 * NRMG_ERR_ARG for bad sizes or pointers, NRMG_ERR_CUDA for a failed launch.
 */
#ifndef NRMG_NET_H
#define NRMG_NET_H

#include <stddef.h>

#include "nrmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nrmg_net nrmg_net;

/* cin in [1, 64]; hidden 32 or 64; cout in [1, 16]; max_pixels = the largest B*H*W a
 * call may use.  0 when the sizes are invalid. */
size_t nrmg_net_workspace_bytes(int cin, int hidden, int cout, long long max_pixels);
/* Weights drawn uniformly in +-sqrt(6 / fan_in) (+-sqrt(3 / fan_in) for the last layer) from a
 * counter-based generator keyed by seed; biases zero; AdamW moments zero. */
nrmg_status nrmg_net_create(int cin, int hidden, int cout, long long max_pixels, unsigned long long seed,
                            void *dev_workspace, size_t ws_bytes, void *cuda_stream, nrmg_net **out);
nrmg_status nrmg_net_destroy(nrmg_net *net);

/* Number of FP32 parameters in the flat layout above; copy them out or in (device arrays).
 * set_params also clears the AdamW moments and step count. */
long long nrmg_net_param_count(const nrmg_net *net);
nrmg_status nrmg_net_get_params(nrmg_net *net, float *dev_params);
nrmg_status nrmg_net_set_params(nrmg_net *net, const float *dev_params);

/* y = net(x) for B images of H x W (B*H*W <= max_pixels).  Asynchronous. */
nrmg_status nrmg_net_forward(nrmg_net *net, const float *dev_x, int B, int H, int W, float *dev_y);

/* Loss = mean over the B*H*W*cout outputs of (y - target)^2, and its gradient with respect to
 * every parameter (flat layout, FP32) into dev_grad.  Deterministic (no atomics).  *loss_out
 * (host, may be NULL; synchronizes when given) receives the loss. */
nrmg_status nrmg_net_gradients(nrmg_net *net, const float *dev_x, const float *dev_target, int B, int H, int W,
                               float *dev_grad, double *loss_out);

/* One AdamW step on that loss: beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected moments,
 * decoupled weight decay wd on the weights (not the biases).  *loss_out as above: the loss
 * before the step. */
nrmg_status nrmg_net_train_step(nrmg_net *net, const float *dev_x, const float *dev_target, int B, int H, int W,
                                float lr, float wd, double *loss_out);

/* ---- field-level glue of the lid-driven cavity family (walls at rest except the top one,
 * which moves along x with speed U > 0).  Fields are [cells][14] FP64 in the order of
 * nrmg_fields, cells row-major from the bottom-left corner (cell = row * nx + column).
 * The ten learned fields are rho, u1, u2, theta, s11, s12, s22, s33, q1, q2. */
#define NRMG_LEARN_CIN 19
#define NRMG_LEARN_COUT 10
#define NRMG_LEARN_FEATURE_SCALE 10.0  /* field features: 10 (f - rest) / U */
#define NRMG_LEARN_TARGET_SCALE 100.0  /* targets: 100 (fine - interpolated) / U */

/* Network input on the grid twice as fine as the coarse one (H = 2 Hc, W = 2 Wc): the coarse
 * fields interpolated bilinearly between cell centres (constant beyond the outermost centres)
 * into dev_prolonged [H*W][14], and the features dev_x [H*W][19] FP32: the ten learned fields
 * minus their rest values (1 for rho and theta), times NRMG_LEARN_FEATURE_SCALE / U; log10 Kn;
 * log10 (Kn W / lx); U; the cell-centre coordinates x / lx and y / ly; and four indicators of the cells next to
 * the bottom, right, top and left walls. */
nrmg_status nrmg_learned_features(const double *dev_coarse_fields, int Hc, int Wc, double lx, double ly, double Kn,
                                  double U, double *dev_prolonged, float *dev_x, void *cuda_stream);
/* Training target dev_t [H*W][10] FP32: NRMG_LEARN_TARGET_SCALE (fine - prolonged) / U of the
 * ten learned fields (the two scalings make features and targets of order one). */
nrmg_status nrmg_learned_targets(const double *dev_prolonged, const double *dev_fine_fields, int cells, double U,
                                 float *dev_t, void *cuda_stream);
/* dev_fields = dev_prolonged + (U / NRMG_LEARN_TARGET_SCALE) dev_y on the ten learned fields
 * (dev_y [cells][10] is the network's output); u3, s13, s23 and q3 are set to zero (the
 * planar flow). */
nrmg_status nrmg_learned_combine(const double *dev_prolonged, const float *dev_y, int cells, double U,
                                 double *dev_fields, void *cuda_stream);

/* Set the finest level of a solver context to the 13-moment Grad state of given fields
 * (dev_fields [cells][14] FP64): expansion centre (u1, u2, 0, theta); f_0 = rho;
 * f_{e_i+e_j} = s_ij / (1 + delta_ij) with the trace of s removed; f_{3e_i} = f_{e_i+2e_d}
 * (d != i) = q_i / 5, which reproduces q_i exactly under eq. moments-relation; every other
 * coefficient zero.  Then checks the state as nrmg_set_state does (NRMG_ERR_NONPHYSICAL for
 * rho <= 0, theta <= 0 or a non-finite value) and, like it, resets the reference mass and
 * residual of the context.  Synchronizes. */
nrmg_status nrmg_set_state_from_fields(nrmg_ctx *ctx, const double *dev_fields);

#ifdef __cplusplus
}
#endif

#endif
