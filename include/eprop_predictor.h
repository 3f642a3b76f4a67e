/*
 * Learned learning-signal predictor: C ABI.
 *
 * The paper has no counterpart; this is an addition beside plain e-prop.  A
 * small MLP estimates the error signal E_k^t (Methods, "Loss function":
 * E_k = pi_k - pi*_k for softmax cross-entropy) from the network's per-step
 * state, so that the learning signal L_j = sum_k B_jk E_k (Methods,
 * "Gradients") can be formed before a sample's target window opens.
 *
 *   input  x (n_in values per row): the K readout potentials y_k^t followed
 *          by 64 population rates r_g^t = beta r_g^{t-1} + (1 - beta) *
 *          (mean spike count of the neurons j with j mod 64 = g), beta =
 *          exp(-dt / 20 ms) (Eq. ema-rate applied to group means), in
 *          spikes per 1000 steps (the paper's rate unit);
 *   layers n_in -> hidden -> hidden -> n_out, GELU(x) = x Phi(x) between;
 *   output an estimate of E^t (n_out values per row).
 *
 * BF16 form: scaled inputs, weights, the hidden activations after GELU and the
 * backward deltas that enter a matrix product are rounded to BF16 (round to
 * nearest even); every product accumulates in FP32 on the tensor cores
 * (mma.sync m16n8k16); biases, pre-activations, outputs, gradients and the
 * Adam state are FP32.  Training minimises (1 / (2 R)) sum (Y - E)^2 over a
 * batch of R rows with Adam (Eq. adam1, Eq. adam2, Eq. adam; beta1 0.9,
 * beta2 0.999, eps 1e-8) on FP32 master weights.
 *
 * Parameters are packed, row-major, in the order W1 [n_in][hidden],
 * b1 [hidden], W2 [hidden][hidden], b2 [hidden], W3 [hidden][n_out],
 * b3 [n_out].
 *
 * Every call is asynchronous on the predictor's stream except where noted;
 * errors return a status (codes of eprop.h) and a message readable with
 * eprop_predictor_last_error.
 */
#ifndef EPROP_PREDICTOR_H
#define EPROP_PREDICTOR_H

#include <stdint.h>

#include "eprop.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eprop_predictor eprop_predictor;

/* Creates a predictor for up to max_rows rows per call.  params: n_params
 * packed FP32 values (host), or NULL for the seeded default (weights
 * N(0, 1 / fan_in) from a SplitMix64 hash of (seed, index) through the
 * Box-Muller transform, zero biases).  stream: a cudaStream_t or NULL (the
 * predictor then owns a stream).  Sizes: 1 <= n_in, n_out <= 1024,
 * 16 <= hidden <= 1024, 1 <= max_rows <= 65536; EPROP_EINVAL otherwise. */
eprop_status eprop_predictor_create(int32_t n_in, int32_t hidden, int32_t n_out, int32_t max_rows,
                                    const float *params, uint64_t seed, void *stream,
                                    eprop_predictor **out);

/* Number of packed parameters. */
int64_t eprop_predictor_num_params(const eprop_predictor *p);

/* Forward pass: y [rows][n_out] = MLP(x [rows][n_in]); pointers are host
 * pointers unless is_device (device pointers must stay valid until the
 * call's work is done).  Waits for completion when is_device = 0. */
eprop_status eprop_predictor_forward(eprop_predictor *p, const float *x, int32_t rows, float *y,
                                     int32_t is_device);

/* One training step on a batch: forward, loss (1/(2 rows)) sum (Y - e)^2,
 * backward and one Adam update with learning rate lr.  x [rows][n_in],
 * e [rows][n_out]; loss_out (host, may be NULL) receives the batch loss
 * before the update (the call then waits for completion). */
eprop_status eprop_predictor_train_step(eprop_predictor *p, const float *x, const float *e,
                                        int32_t rows, float lr, float *loss_out, int32_t is_device);

/* Copies an internal buffer of the last call to host memory (waits):
 *   0 parameters [n_params]      1 gradients of the last train step [n_params]
 *   2 A1 [rows][hidden] (FP32)   3 H1 [rows][hidden] (BF16 values)
 *   4 A2 [rows][hidden]          5 H2 [rows][hidden] (BF16 values)
 *   6 Y [rows][n_out]            7 dY [rows][n_out] (BF16 values)
 *   8 dA2 [rows][hidden] (BF16)  9 dA1 [rows][hidden] (BF16)
 *  10 Adam m [n_params]         11 Adam v [n_params]
 *  12 x as used, BF16 values [rows][n_in]
 * rows = the row count of the last forward or train call; count is the
 * number of floats the caller's buffer holds (EPROP_EINVAL if too small). */
eprop_status eprop_predictor_read(eprop_predictor *p, int32_t which, float *dst, int64_t count);

/* Sets the input scale s [n_in] (host FP32; part of the model, default 1):
 * the first layer sees bf16(x_c * s_c). */
eprop_status eprop_predictor_set_input_scale(eprop_predictor *p, const float *scale);

/* Replaces the packed parameters (host FP32) and resets the Adam state. */
eprop_status eprop_predictor_set_params(eprop_predictor *p, const float *params);

/* Attaches a predictor to a network (batch <= max_rows, n_in = n_out + 64,
 * n_out equal to the network's readouts) or detaches it (mode 0).  Each
 * step, after the readout, the inputs x^t of every sample are formed on the
 * GPU (its readout potentials and the 64 group rates of its recurrent
 * neurons, groups j mod 64).  mode bit 0: the predictor's output stands in
 * for E^t wherever the sample's target window is closed (window = 0),
 * both in the learning signal and in the readout gradient, so that weight
 * updates do not wait for the target window; bit 1: x^t of the last call
 * is recorded (eprop_read_predictor_inputs).  The predictor must outlive
 * the attachment; it runs on the network's stream and is captured with the
 * rest of a call in launch_mode 1.  Group rates restart from zero with the
 * network state (non-continuous calls). */
eprop_status eprop_attach_predictor(eprop_net *net, eprop_predictor *p, int32_t mode);

/* Copies the recorded predictor inputs of the last simulate call,
 * [batch][T][n_out + 64] (mode bit 1 needed).  Host pointer unless
 * is_device; waits. */
eprop_status eprop_read_predictor_inputs(eprop_net *net, float *x, int32_t is_device);

eprop_status eprop_predictor_sync(eprop_predictor *p);
void eprop_predictor_destroy(eprop_predictor *p);
const char *eprop_predictor_last_error(const eprop_predictor *p);

#ifdef __cplusplus
}
#endif

#endif /* EPROP_PREDICTOR_H */
