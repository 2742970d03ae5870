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

/* ---- learned coarse-level correction of the lid-driven cavity family.
 * The paper's cycle updates the fine grid with the coarse change carried over piecewise
 * constant (eq. rewritten-update: f^ = f-_h - f-_H + f~_H in each fine cell of a coarse cell).
 * This library adds, on the finest level only, a network's correction of that update: the
 * network sees the coarse change of the ten learned fields (f~_H - f-_H) interpolated to the
 * fine grid and the fine fields after the plain update, and predicts the remaining error of
 * those ten fields.  Its correction is kept only when the residual norm of eq.
 * (relative-residual) right after the update is smaller with it than without it; otherwise
 * the plain update stands.  The converged solution is still R(f) = 0 of the paper's operator.
 *
 * Scaling: with s the largest |change| of the ten coarse fields times
 * NRMG_CORR_FIELD_SCALE / U (over all coarse cells and fields), the network input is
 * x [H*W][NRMG_CORR_CIN] FP32:
 *   0..9   the interpolated coarse change (bilinear between cell centres, constant beyond
 *          the outermost ones) times NRMG_CORR_FIELD_SCALE / (U s);
 *   10..19 the fine fields after the plain update minus their rest values (1 for rho and
 *          theta), times NRMG_CORR_FIELD_SCALE / U;
 *   20..28 log10 Kn, log10 (Kn W / lx), U, x / lx, y / ly and the four wall indicators, as
 *          channels 10..18 of nrmg_learned_features;
 * and its output y [H*W][10] is the correction of the ten fields in units of U s /
 * NRMG_CORR_FIELD_SCALE.  The correction enters each cell's Grad expansion as a linear
 * increment (rho += d_rho; f_{e_i} += rho' d_u_i; every f_{2e_d} += rho' (3 d_theta + |d_u|^2) / 6
 * with rho' = rho + d_rho; f_{e_i+e_j} += d_s_ij / (1 + delta_ij) with the trace of d_s removed;
 * f_{3e_i} and f_{e_i+2e_d} += d_q_i / 5), after which the cell is projected back to Grad form
 * as after a sweep update. */
#define NRMG_CORR_CIN 29
#define NRMG_CORR_FIELD_SCALE 10.0

/* Device workspace of nrmg_fas_cycle_learned for this context (0 for a one-level context or
 * an odd finest grid). */
size_t nrmg_learned_cycle_workspace_bytes(const nrmg_ctx *ctx);

/* Acceptance rule of the correction, i.e. which residual decides whether it is kept: right
 * after the update (both candidates before the post-smoothing), after the post-smoothing (each
 * candidate smoothed s2 times; the cheaper rule also counts high-frequency defects of a
 * correction that the smoother would remove), or none (the correction is always kept). */
#define NRMG_ACCEPT_UPDATE 0
#define NRMG_ACCEPT_SMOOTHED 1
#define NRMG_ACCEPT_ALWAYS 2

/* One cycle as nrmg_fas_cycle (Algorithm 2 on the finest level with gamma coarse cycles, then
 * the mass correction), with a learned correction of the finest level's update:
 *   net        the network (cin NRMG_CORR_CIN, cout 10, created on the context's stream, at
 *              least H*W pixels), or NULL;
 *   dev_y      used when net is NULL: a given correction [H*W][10] in the network's output
 *              units (tests and bounds on what a correction can gain); NULL with net NULL =
 *              the plain update (the cycle is then nrmg_fas_cycle's, bit for bit);
 *   accept_rule  NRMG_ACCEPT_UPDATE, NRMG_ACCEPT_SMOOTHED or NRMG_ACCEPT_ALWAYS;
 *   Kn, U      the problem's Knudsen number and lid speed (the input scaling);
 *   dev_ws     caller-owned device workspace, 256-byte aligned, ws_bytes >=
 *              nrmg_learned_cycle_workspace_bytes;
 *   dev_x_out, dev_fine_out  (may be NULL) receive the network input of this cycle and the
 *              fine fields [H*W][14] after the plain update (training data);
 *   scale_out  (host, may be NULL) receives s;
 *   accepted_out (host, may be NULL) receives 1 when the network's correction was kept;
 *   rel_res_out as for nrmg_fas_cycle.
 * Synchronizes.  NRMG_ERR_ARG for a one-level context, a bad workspace or acceptance rule, or a network
 * of the wrong shape or stream. */
nrmg_status nrmg_fas_cycle_learned(nrmg_ctx *ctx, nrmg_net *net, const float *dev_y, int accept_rule, double Kn, double U,
                                   void *dev_ws, size_t ws_bytes, float *dev_x_out, double *dev_fine_out,
                                   double *scale_out, int *accepted_out, double *rel_res_out);

/* The correction step alone, for tests and custom cycles: the finest level's state f becomes
 * Grad(f + increment) with the increment above for the fields U scale y / NRMG_CORR_FIELD_SCALE
 * (dev_y [cells][10] FP32 in the order rho, u1, u2, theta, s11, s12, s22, s33, q1, q2).  No
 * acceptance test.  NRMG_ERR_NONPHYSICAL when a cell leaves rho > 0, theta > 0 (the level is
 * then undefined).  Synchronizes. */
nrmg_status nrmg_learned_correct(nrmg_ctx *ctx, const float *dev_y, double scale, double U);

/* Training target of the correction: dev_t [cells][10] = (converged - fine) of the ten learned
 * fields times NRMG_CORR_FIELD_SCALE / (U scale) (fields [cells][14] FP64 as nrmg_fields). */
nrmg_status nrmg_learned_correction_targets(const double *dev_fine, const double *dev_converged, int cells, double U,
                                            double scale, float *dev_t, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif
