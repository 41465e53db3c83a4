/* Learned warm start for the LBM iteration.
 *
 * The LBM of arXiv:1809.01600 is iterated from an initial state to the
 * steady state (Section 4.1 starts it from a 1-D profile; lbms.h offers that
 * profile as LBMS_INIT_PROFILE_1D).  The steady state does not depend on the
 * start, so a better start only shortens the iteration.  This network
 * predicts that steady state from the anode's geometry and boundary data;
 * the LBM then iterates from the prediction to the same residual as from any
 * other start, and its result is the one that counts.  The paper has no network:
 * this is an addition on top of its method.
 *
 * Two models.  lbms_unet_* (at the end of this file) is a 3-D U-Net whose
 * convolutions are implicit GEMMs on the tcgen05 tensor cores; it sees the
 * pore structure and is the better start at the grid it was trained on.
 * lbms_net_* is a pointwise multilayer perceptron, described here, which
 * carries over to longer anodes than it was trained on.
 *
 * Pointwise model.  Every fluid cell gets a feature
 * row built on the GPU from the solid mask and the boundary data: the
 * Section 4.1 profile at its x, x / L, the fluid fraction of cubes of
 * half-width 1, 3 and 7 cells around it, the cross-section porosity at x and
 * the cumulative resistance int_0^x dx / porosity(x) (normalised), the
 * current density and the inlet composition.  The network maps the row to
 * 100 (X_steady - X_profile) for the three species.  Hidden layers use ReLU;
 * weights are stored in BF16 for the tensor-core matrix products (tcgen05,
 * FP32 accumulation in tensor memory) with FP32 master copies updated by
 * Adam.
 *
 * All functions return an lbms_status and never abort; buffers are host
 * memory owned by the caller unless stated otherwise.  A net (either model)
 * is not thread safe; its device work runs on the legacy default stream. */
#ifndef LBMS_NET_H
#define LBMS_NET_H

#include <stdint.h>

#include "lbms.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbms_net lbms_net;

enum { LBMS_NET_FEATURES = 64 };   /* feature row width (16 used, zero padded) */

/* width: hidden units per layer (multiple of 64, 64..2048); depth: hidden
 * layers (1..8).  Weights are drawn from a counter-based generator
 * (SplitMix64) keyed by seed; the output layer starts at zero. */
lbms_status lbms_net_create(int width, int depth, uint64_t seed, lbms_net **out);

/* Adds one case of a handle as training data: the feature rows of its fluid
 * cells and, as the target, the handle's current mole fractions of that case
 * (call it on a steady state).  The case must have boundary data. */
lbms_status lbms_net_add_sample(lbms_net *net, lbms_ctx *ctx, int case_index);

/* The feature rows the network sees for one case of a handle (the rows
 * lbms_net_add_sample and lbms_net_warm_start build on the GPU), for
 * inspection and tests: rows [n_rows][LBMS_NET_FEATURES] BF16 bit patterns,
 * one per fluid cell in x-fastest order; n_rows must equal the case's fluid
 * cell count.  Columns: 0-2 the Section 4.1 profile X at the cell's x, 3
 * x / (nx - 1), 4-6 the fluid fraction of the (2h+1)^dim boxes with h = 1, 3,
 * 7 around the cell (clamped at the ends of x, periodic in y and z), 7 the
 * current density / 2 (A/cm^2), 8-10 the inlet X, 11 column 3 times column
 * 7, 12 the fluid fraction phi(x) of the cell's x-plane (at least one cell),
 * 13 the trapezoidal integral of 1 / phi from 0 to x over its value at
 * nx - 1, 14 1 / (4 phi(x)), 15 one, 16-63 zero. */
lbms_status lbms_net_features(lbms_net *net, lbms_ctx *ctx, int case_index, uint16_t *rows, int64_t n_rows);

/* iters steps of Adam (beta 0.9 / 0.999, eps 1e-8) on mean-square error over
 * batches of `batch` rows (a multiple of 64) drawn uniformly with replacement
 * from the training rows by a counter-based generator; the learning rate
 * decays from lr by a cosine to lr / 20 over the iterations of this call.
 * last_loss (may be NULL) receives the mean loss of the last 10 steps. */
lbms_status lbms_net_train(lbms_net *net, int iters, int batch, double lr, double *last_loss);

/* Predicts the steady mole fractions of one case of a handle and restarts
 * that case from them (f = w X, as lbms_batch_set_fields).  The prediction
 * is clamped to X >= 1e-6 and renormalised to sum 1 per cell.  X (may be
 * NULL) receives the predicted dense field [3][N] (0 in solid cells). */
lbms_status lbms_net_warm_start(lbms_net *net, lbms_ctx *ctx, int case_index, double *X);

/* Inference and one training step on caller-given rows, for tests:
 * features [rows][LBMS_NET_FEATURES] as BF16 bit patterns, targets
 * [rows][3]; rows a multiple of 64.  out [rows][3] receives the network
 * output (before the step).  With lr = 0 the parameters do not change;
 * the gradients are kept for lbms_net_get. */
lbms_status lbms_net_forward(lbms_net *net, const uint16_t *features, int rows, float *out);
lbms_status lbms_net_train_batch(lbms_net *net, const uint16_t *features, const float *targets, int rows,
                                 double lr, double *loss);

/* Parameters and gradients, layer by layer: for layer l (0 = input layer,
 * depth = output layer) W_l [out_l][in_l] row-major then b_l [out_l], with
 * in_0 = LBMS_NET_FEATURES, out_depth = 3 and every other size = width.
 * what: 0 = FP32 master parameters, 1 = gradients of the last step.
 * n = number of floats the buffer holds (lbms_net_info's n_params). */
lbms_status lbms_net_get(const lbms_net *net, int what, float *buf, int64_t n);
lbms_status lbms_net_set(lbms_net *net, const float *params, int64_t n);

lbms_status lbms_net_info(const lbms_net *net, int64_t *n_params, int64_t *n_samples);

/* Which kernel computes the network's matrix products.  AUTO: the tcgen05
 * tensor-core kernel (operands staged by TMA, FP32 accumulators in tensor
 * memory) for every product whose sizes it takes (N and each K chunk
 * multiples of 64), the mma.sync kernel for the others; TCGEN05: the
 * tcgen05 kernel only (a product it cannot take is LBMS_EINVAL); MMA_SYNC:
 * the mma.sync kernel only.  lbms_net_gemm_calls counts the products each
 * kernel has computed since the net was created.  A timed-out wait inside
 * the tcgen05 kernel is reported as LBMS_ECUDA by the call that ran it. */
enum { LBMS_NET_GEMM_AUTO = 0, LBMS_NET_GEMM_TCGEN05 = 1, LBMS_NET_GEMM_MMA_SYNC = 2 };
lbms_status lbms_net_set_gemm(lbms_net *net, int kind);
lbms_status lbms_net_gemm_calls(const lbms_net *net, int64_t *tcgen05_calls, int64_t *mma_sync_calls);
const char *lbms_net_last_error(const lbms_net *net);
void lbms_net_destroy(lbms_net *net);

/* ------------------------------------------------------------------------
 * Convolutional warm start: a three-level 3-D U-Net over the anode's voxels
 * (two 3x3x3 convolutions with zero padding and ReLU per level, 2x2x2 max
 * pooling down, 2x2x2 stride-2 transposed convolutions up, skip
 * concatenation, a 1x1 convolution to 3 outputs), with `width`, 2 width and
 * 4 width channels on its levels.  Input channels: the 16 used feature
 * columns of lbms_net_features on fluid voxels (zero on solid ones) and the
 * fluid mask; output: 100 (X - X_profile), as the pointwise network.  Every
 * convolution is an implicit GEMM on the tcgen05 tensor cores (BF16
 * operands staged by TMA, FP32 accumulation): activations are stored BF16
 * with a zero halo around each volume, so each tap reads the activation
 * matrix at a shifted row; weights are BF16 with FP32 master copies (Adam,
 * beta 0.9 / 0.999, eps 1e-8).
 *
 * A volume's extents must be multiples of 4 (the two poolings): a case is
 * placed in a volume with its extents rounded up to multiples of 4, the
 * added voxels solid (mask 0).  max_voxels bounds the voxels of one batch
 * (B volumes; one volume for lbms_unet_warm_start), up to
 * LBMS_UNET_MAX_VOXELS.  Activation buffers are allocated for the largest
 * batch met, about 3.4 kB per voxel of it (8 volumes of 96^3: 27 GB).
 * width 4..32 (28 gives 1.05M parameters); weights He-uniform from a
 * counter-based generator keyed by seed, head and biases zero. */
typedef struct lbms_unet lbms_unet;

enum { LBMS_UNET_MAX_VOXELS = 8000000 };   /* the padded rows stay within 65535 tiles of 128 */

lbms_status lbms_unet_create(int width, int64_t max_voxels, uint64_t seed, lbms_unet **out);

/* Adds one case of a handle as a training volume: its inputs and, as the
 * target, 100 (X - X_profile) of the handle's current mole fractions on its
 * fluid voxels (call it on a steady state).  The case must have boundary
 * data and fit max_voxels. */
lbms_status lbms_unet_add_sample(lbms_unet *net, lbms_ctx *ctx, int case_index);

/* Adds a caller-given training volume: x FP32 [17][Z][Y][X] (channel 16 the
 * fluid mask), targets [3][Z][Y][X]; X, Y, Z multiples of 4. */
lbms_status lbms_unet_add_volume(lbms_unet *net, const float *x, const float *targets, int X, int Y, int Z);

/* iters steps of Adam on the mean-square error over fluid voxels.  Step i
 * takes the training volumes of group i mod G (volumes of equal extents, in
 * order of first addition): min(max_batch, volumes in the group,
 * max_voxels / voxels a volume) of them, drawn uniformly with replacement
 * by a counter-based generator.  The learning rate decays from lr by a
 * cosine to lr / 20 over the iterations of this call; last_loss (may be
 * NULL) receives the mean loss of the last 10 steps. */
lbms_status lbms_unet_train(lbms_unet *net, int iters, int max_batch, double lr, double *last_loss);

/* Predicts the steady mole fractions of one case and restarts that case
 * from them, as lbms_net_warm_start (clamped at 1e-6, renormalised; X may
 * be NULL or receives the dense field [3][N]). */
lbms_status lbms_unet_warm_start(lbms_unet *net, lbms_ctx *ctx, int case_index, double *X);

/* Inference and one training step on caller-given volumes, for tests: x
 * FP32 [B][17][Z][Y][X] (channel 16 the fluid mask), targets [B][3][Z][Y][X],
 * out [B][3][Z][Y][X]; X, Y, Z multiples of 4.  The loss is
 * sum((out - target)^2 mask) / (3 sum(mask)).  With lr = 0 the parameters
 * do not change; the gradients are kept for lbms_unet_get. */
lbms_status lbms_unet_forward(lbms_unet *net, const float *x, int B, int X, int Y, int Z, float *out);
lbms_status lbms_unet_train_batch(lbms_unet *net, const float *x, const float *targets, int B, int X, int Y, int Z,
                                  double lr, double *loss);

/* Parameters (what = 0) or the gradients of the last step (what = 1) in
 * the order and layouts of the PyTorch modules Conv3d / ConvTranspose3d:
 * per layer (e1a, e1b, e2a, e2b, e3a, e3b, u2, d2a, d2b, u1, d1a, d1b, head)
 * its weight ([co][ci][3][3][3]; transposed: [ci][co][2][2][2]; head
 * [3][width]) then its bias [co].  n = floats the buffer holds. */
lbms_status lbms_unet_get(const lbms_unet *net, int what, float *buf, int64_t n);
lbms_status lbms_unet_set(lbms_unet *net, const float *params, int64_t n);

lbms_status lbms_unet_info(const lbms_unet *net, int64_t *n_params, int64_t *n_samples);
/* Matrix products computed on the tcgen05 tensor cores since creation. */
lbms_status lbms_unet_gemm_calls(const lbms_unet *net, int64_t *tcgen05_calls);
const char *lbms_unet_last_error(const lbms_unet *net);
void lbms_unet_destroy(lbms_unet *net);

#ifdef __cplusplus
}
#endif

#endif
