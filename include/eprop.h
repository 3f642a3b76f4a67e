/*
 * eprop.h -- C ABI of the GB300 event-driven e-prop library (libeprop.so).
 *
 * The library simulates recurrent spiking networks of LIF or ALIF neurons
 * with a leaky readout and trains every input, recurrent and readout weight
 * with eligibility propagation (e-prop), exactly as the time-driven
 * definition of the paper "Event-driven eligibility propagation in large
 * sparse networks" (Methods: neuron models, loss function, gradients,
 * optimization) but organised event by event: a synapse is touched only when
 * a presynaptic spike reaches it, and its eligibility trace is advanced in
 * closed form over the interval since its previous arrival (Results,
 * "Event-driven weight updates in e-prop"; Algorithm 5).
 *
 * Conventions for every call:
 *   - Returns EPROP_OK or an error code; no exception crosses the ABI.
 *     eprop_last_error() gives a human-readable message for the last error.
 *   - Pointer arguments are host pointers unless `is_device` is 1, in which
 *     case they must be device pointers valid on the network's device.
 *     Input arrays are copied (host) or read during the call (device) and
 *     stay owned by the caller.
 *   - All state is owned by the library; eprop_destroy frees it.
 *   - Work is issued asynchronously on the CUDA stream given at creation.
 *     Inside a simulate call part of it (the readout kernels) runs on a
 *     second stream the network owns, forked from and joined back into
 *     that stream with events, so that work the caller orders after the
 *     call on the given stream sees all of it.  eprop_sync waits for it and
 *     surfaces device errors.
 *   - After EPROP_ETIMEOUT or EPROP_ECUDA the network is in an error state
 *     and every further call except eprop_destroy / eprop_last_error
 *     returns EPROP_ESTATE.
 *   - Time is in steps of dt (ms).  Steps of one simulate call are numbered
 *     t = 1..T; state before t = 1 is zero for a fresh or reset network.
 */
#ifndef EPROP_H
#define EPROP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPROP_ABI_VERSION 2
#define EPROP_MAX_DRIVE_THR 64

typedef enum {
    EPROP_OK = 0,
    EPROP_EINVAL = 1,   /* invalid argument or unsupported combination      */
    EPROP_ENOMEM = 2,   /* device or host allocation failed                  */
    EPROP_ECUDA = 3,    /* a CUDA call or kernel failed                      */
    EPROP_ETIMEOUT = 4, /* a bounded device wait gave up                     */
    EPROP_ESTATE = 5    /* the network is in an error state / wrong order    */
} eprop_status;

typedef struct eprop_net eprop_net; /* opaque; owned by the library */

/*
 * Network and learning parameters (plain old data).
 *
 * Neuron model (Methods, "Neuron models", Eq. lif_update):
 *   a_j^t   = rho a_j^{t-1} + z_j^{t-1},          rho   = exp(-dt / tau_a)
 *   v_th^t  = v_th + beta_a a_j^t                 (beta_a used only for ALIF)
 *   v_j^t   = alpha v_j^{t-1} + I_j^t - z_j^{t-1} v_th^t,   alpha = exp(-dt / tau_m)
 *   z_j^t   = 1 iff v_j^t - v_th^t > 0 and the neuron is not refractory
 *   I_j^t   = sum over synapses of the weight carried by each spike arriving
 *             at t (emitted at t - d, d = the synapse's delay, 1 <= d <=
 *             max_delay) + drive_weight * n_j^t (external Poisson drive)
 * A neuron that spiked at t is refractory for t_ref steps: z = 0, psi = 0.
 * Surrogate (Eq. piecewise-linear-surrogate-gradient):
 *   psi_j^t = gamma * max(0, 1 - beta_sg |v_j^t - v_th^t|)
 * Readout (Eq. leaky_integrator): y_k^t = kappa y_k^{t-1} + sum_j W_out[j][k] z_j^t
 * Loss: 0 = MSE (Eq. mean-squared-error), 1 = softmax cross-entropy
 * (Eq. softmax, Eq. cross-entropy-loss); the error signal is multiplied by
 * the per-step learning window.
 * Learning signal: L_j^t = sum_k B[j][k] E_k^t with B = W_out (symmetric,
 * feedback = 0) or a fixed random matrix (feedback = 1).
 * Eligibility trace filter: kappa_e (Eq. filtered-eligibility-trace with
 * the filter decoupled from the readout, Results "Eligibility trace filter
 * decoupled from output time constant"); kappa_e < 0 means kappa_e = kappa.
 * Weight update (Eq. gradient-descent): W -= lr * (mean over the batch of
 * each sample's sum over the window of g^t), applied after the last step of
 * every update window.  update_interval = U steps (0: one window per
 * simulate call); windows are counted from the last state reset.
 *
 * Variants of the paper's e-prop+ and constraints (all 0 = the plain method):
 *   surrogate 1: psi = gamma exp(-beta_sg |v - v_th|) (Eq. exponential-
 *     surrogate-gradient);
 *   reset_mode 1: fixed reset (Methods, neuron models, e-prop+): the step
 *     after a spike the decayed membrane alpha v is replaced by v_reset,
 *     v^t = v_reset + I^t; like the soft reset it is a stop-gradient, so the
 *     eligibility trace is unchanged;
 *   loss 2: temporal MSE (1/K) sum_k (y_k - y*_k)^2, E_k = (2/K)(y_k - y*_k)
 *     (Eq. temporal-mse);
 *   c_reg != 0: firing-rate regularisation with the moving-average rate
 *     f_j^t = beta_reg f_j^{t-1} + (1 - beta_reg) z_j^t (Eq. ema-rate) in
 *     spikes per step and target f_target; adds c_reg (f_j^t - f_target)
 *     G_beta(e^t) to the gradient of every synapse onto neuron j
 *     (Eq. ema-gradient); needs continuous = 0 and update_interval = 0 (the
 *     second filtered trace is not carried between windows);
 *   sign_mask: weights keep the sign of their initial value (bit 0 input,
 *     bit 1 recurrent, bit 2 readout weights; Dale's law when the initial
 *     weights of each source share a sign); an update that would cross zero
 *     leaves a zero of that sign;
 *   optimizer 1: Adam (Eq. adam with the TensorFlow reordering Eq. eta-adam-
 *     fast, Eq. delta-w-adam-fast, constant eps_hat = adam_eps): one step per
 *     update window on the window's batch-mean gradient, k = steps taken,
 *     eta_k = lr sqrt(1 - b2^k) / (1 - b1^k), w -= eta_k m / (sqrt(v) + eps_hat);
 *   if_period > 0: ignore-and-fire neurons (Methods, "Scaling"): z_j^t = 1
 *     iff (t_abs + phase_j) mod if_period == 0 regardless of the membrane,
 *     phase_j = (upper 32 bits of mix(if_seed ^ j)) mod if_period; v and psi
 *     are still integrated.
 * sign_mask & 3 and optimizer 1 are not available with the lazy window form
 * that carries state (trace_kernel 1 with continuous or update_interval).
 *
 * External drive: n_j^t = #{m < n_drive_thr : u >= drive_thr[m]} with u the
 * upper 32 bits of h = mix(mix(mix(drive_seed ^ j) ^ t_abs) ^ sample),
 * mix = the SplitMix64 output function, t_abs = the network's absolute step
 * counter (1 for the first step after creation).  drive_thr[0 .. n_drive_thr)
 * must be non-decreasing (an inversion table of a CDF); creation fails with
 * EPROP_EINVAL otherwise.
 */
typedef struct eprop_config {
    int32_t abi_version;      /* must be EPROP_ABI_VERSION */
    int32_t n_in;             /* input channels (sources 0..n_in-1)          */
    int32_t n_rec;            /* recurrent neurons (< 2^24)                  */
    int32_t n_out;            /* readouts, 1..1024                           */
    int32_t batch;            /* samples simulated together, >= 1            */
    int32_t neuron_model;     /* 0 LIF, 1 ALIF                                */
    int32_t t_ref;            /* refractory steps, >= 0                       */
    int32_t loss;             /* 0 MSE, 1 softmax cross-entropy, 2 temporal MSE */
    int32_t feedback;         /* 0 symmetric B = W_out^T, 1 fixed random B    */
    int32_t update_interval;  /* U in steps; 0 = one window per call          */
    int32_t continuous;       /* 1: keep all state between simulate calls     */
    int32_t max_delay;        /* D, 1..8                                      */
    int32_t trace_dtype;      /* storage of per-synapse traces: 0 FP32, 1 BF16,
                                 2 FP16 (16-bit forms rounded to nearest even,
                                 arithmetic in FP32)                          */
    int32_t record_grad;      /* 1: keep per-synapse gradient sums             */
    int32_t record_raster;    /* 1: keep the spike raster of the last call     */
    int32_t record_psi;       /* 1: keep the surrogate values of the last call */
    int32_t n_drive_thr;      /* entries used in drive_thr (0: no drive)       */
    int32_t launch_mode;      /* 0: launch every kernel of a simulate call;
                                 1: capture a call once in a CUDA graph and
                                 replay it for later calls with the same T;
                                 2: as 1, with every step of the call in one
                                 persistent cooperative kernel (grid barriers
                                 between the neuron and the delivery phases,
                                 bounded waits: EPROP_ETIMEOUT); needs one
                                 update window per call (continuous = 0,
                                 update_interval = 0), n_out <= 256 and no
                                 predictor; results are bit-identical to 0/1 */
    int32_t trace_kernel;     /* synapse-trace kernel: 0 auto (3 when state is
                                 carried, else 2 for batch > 1, else 1);
                                 1 lazy window work queue (batch 1): only
                                 synapses with an arrival are touched, a
                                 skipped window is caught up at the next
                                 arrival; 2 batched single window (no state
                                 carried between windows); 3 dense window
                                 pass (carried state: continuous or
                                 update_interval > 0, else EPROP_EINVAL):
                                 every synapse is advanced at every window
                                 end; with batch > 1 every synapse carries
                                 one trace per sample and the weight steps
                                 with the batch mean; 4 the dense window pass
                                 with the synapse records kept by target band
                                 (12288 LIF / 4608 ALIF targets, a band's
                                 window coefficients in shared memory): same
                                 results bit for bit as 3; needs carried
                                 state, batch 1, optimizer 0 and free synapse
                                 signs (sign_mask & 3 == 0), else
                                 EPROP_EINVAL; eprop_read_weights_grads
                                 returns the creation order                  */
    int32_t blocks_per_sm;    /* CTAs per SM of the row kernels; 0 = 2        */
    int32_t profile;          /* 1: time the synapse-trace kernels of every
                                 window with CUDA events (see eprop_stats)    */
    float dt;                 /* ms                                           */
    float tau_m, tau_a, beta_a, v_th, tau_out, kappa_e;
    float gamma, beta_sg;
    float lr;
    float drive_weight;
    uint64_t drive_seed;
    uint32_t drive_thr[EPROP_MAX_DRIVE_THR];
    /* variants (see above) */
    int32_t surrogate;        /* 0 piecewise linear, 1 exponential            */
    int32_t reset_mode;       /* 0 subtract the threshold, 1 fixed v_reset     */
    float v_reset;
    float c_reg, f_target, beta_reg;
    int32_t sign_mask;        /* 1 input, 2 recurrent, 4 readout weights       */
    int32_t optimizer;        /* 0 SGD, 1 Adam                                 */
    float adam_b1, adam_b2, adam_eps;
    int32_t if_period;        /* ignore-and-fire period in steps, 0 = off      */
    uint64_t if_seed;
    /* generalized delays (Supplement "Generalized delays"), in steps 0..64:
       the readout receives the recurrent spikes d_out steps late (Eq.
       leaky_integrator_with_delay), and the learning signal of step tau
       reaches the recurrent layer at tau + d_ls, paired with the filtered
       eligibility trace of tau - d_out (Eq. eprop-learning-signal-delay);
       signals arriving after a sample's end are dropped.  Nonzero values
       need one update window per call (update_interval = 0, continuous =
       0) and launch_mode 0 or 1.                                          */
    int32_t d_out, d_ls;
} eprop_config;

/*
 * All input and recurrent synapses as one CSR matrix by source.  Sources
 * 0..n_in-1 are the input channels, n_in..n_in+n_rec-1 the recurrent neurons
 * (source n_in + j is neuron j).  Targets are recurrent neuron indices.
 * Rows may be empty; autapses are allowed by the library but not generated.
 */
typedef struct eprop_synapses {
    int64_t n_src;            /* must equal n_in + n_rec                      */
    int64_t nnz;              /* number of synapses                           */
    const int64_t *row_ptr;   /* [n_src + 1], row_ptr[0] = 0, non-decreasing  */
    const int32_t *target;    /* [nnz] in [0, n_rec)                          */
    const float *weight;      /* [nnz]                                        */
    const uint8_t *delay;     /* [nnz] in [1, max_delay]                      */
} eprop_synapses;

/*
 * Creates a network on the current CUDA device.
 *   w_out     [n_rec][n_out] readout weights (W_out[j][k] = weight j -> k)
 *   out_mask  [n_rec][n_out] 1 where the readout synapse j -> k exists: its
 *             weight W_out[j][k] learns; 0: the weight is held at its value
 *             and gets no gradient (a sparse readout, e.g. an output in-degree
 *             below n_rec, Methods "Scaling"); NULL = all 1
 *   feedback  [n_rec][n_out] fixed random B (required iff cfg->feedback == 1)
 *   cuda_stream  cudaStream_t to issue all work on (NULL: legacy stream);
 *             the network also creates one stream and two events of its own
 *             (readout work, see above), freed by eprop_destroy
 * Errors: EPROP_EINVAL (inconsistent sizes, delays out of range, unsupported
 * combination), EPROP_ENOMEM, EPROP_ECUDA.  On error *out is NULL.
 * Batches: batch > 1 needs continuous = 0 (every sample starts each call
 * from zero state); update windows inside a call (update_interval > 0) run
 * with batch <= 64 in the dense form (one trace per sample and synapse, the
 * shared weight steps with the batch mean at every window end, Eq.
 * accumulated-gradients); the lazy form (trace_kernel 1) needs batch 1.
 */
eprop_status eprop_create_network(const eprop_config *cfg, const eprop_synapses *syn,
                                  const float *w_out, const uint8_t *out_mask,
                                  const float *feedback, int32_t is_device,
                                  void *cuda_stream, eprop_net **out);

/*
 * Sets the inputs of the next simulate calls (copied into library memory).
 *   in_step_ptr [batch*T + 1]: input spikes of sample b emitted at step t are
 *               in_ids[in_step_ptr[b*T + t-1] .. in_step_ptr[b*T + t] - 1]
 *               (Methods: the input reaches the network one delay later)
 *   in_ids      input channel indices in [0, n_in)
 *   targets     [batch][T][n_out]: y*_k^t (MSE) or one-hot pi*_k^t (CE)
 *   window      [batch][T] learning window (0/1) or NULL = all ones
 *               (Results, "Learning window signal generator")
 *   lengths     [batch] steps of each sample, 1..T, or NULL = all T; steps
 *               after a sample's length leave that sample untouched
 * Errors: EPROP_EINVAL on out-of-range ids or lengths, EPROP_ENOMEM.
 */
eprop_status eprop_set_inputs_targets(eprop_net *net, const int64_t *in_step_ptr,
                                      const int32_t *in_ids, int64_t n_in_ids,
                                      const float *targets, const uint8_t *window,
                                      const int32_t *lengths, int32_t T,
                                      int32_t is_device);

/*
 * Simulates T steps (T = the value given to eprop_set_inputs_targets) of
 * every sample and applies the weight updates of every update window that
 * ends inside the call.  Unless continuous, all state is reset to zero first.
 *   forced_raster  NULL, or device pointer [batch][T][n_rec] (uint8): the
 *                  spikes z_j^t are taken from it (teacher forcing) while v,
 *                  psi and all traces are still computed.
 * T must be a multiple of update_interval when update_interval > 0.
 */
eprop_status eprop_simulate(eprop_net *net, int32_t T, const uint8_t *forced_raster);

/*
 * Copies weights and cumulative gradients of one projection.
 *   proj 0: input synapses (CSR entries of rows 0..n_in-1), length nnz_in
 *   proj 1: recurrent synapses (rows n_in..), length nnz_rec
 *   proj 2: readout weights W_out [n_rec][n_out]
 * Weights are those in effect after the last completed update window.
 * `grad` (optional, needs record_grad) receives, per weight, the sum over
 * all updates since creation of the applied batch-mean gradient
 * (sum_t g^t of Eq. accumulated-gradients).  Either pointer may be NULL.
 */
eprop_status eprop_read_weights_grads(eprop_net *net, int32_t proj, float *w, float *grad,
                                      int32_t is_device);

/*
 * Copies the outputs of the last simulate call.
 *   y     [batch][T][n_out] readout signal y_k^t, 0 after a sample's length
 *         (or NULL)
 *   loss_per_sample [batch] sum over steps of the (windowed) loss (or NULL)
 *   raster [batch][T][n_rec] uint8 spikes (needs record_raster; or NULL)
 * Pointers are host pointers unless is_device.
 */
eprop_status eprop_readout(eprop_net *net, float *y, float *loss_per_sample,
                           uint8_t *raster, int32_t is_device);

/*
 * Raster readout without allocation.  The paper has no counterpart: this is
 * an interface variant of the raster part of eprop_readout for callers that
 * cannot allocate device memory when they read (eprop_readout allocates a
 * device scratch buffer on first use; this call unpacks through a fixed
 * scratch array compiled into the library instead).
 *   raster [batch][T][n_rec] uint8 spikes of the last simulate call, written
 *          by the call (host pointer unless is_device); needs record_raster.
 * Limit: batch * T * n_rec <= EPROP_STATIC_RASTER_BYTES, else EPROP_EINVAL
 * with a message and nothing written.  The network's device must be the
 * current device (EPROP_EINVAL otherwise).  No device memory is allocated;
 * only a rejected call records its message in the network's error string.
 * The first call on each device resolves the scratch address once (with
 * lazy module loading this may load the library's device code): make that
 * first call before any stream capture.  The scratch needs no
 * initialisation (every byte read back is written first).  It is one
 * array per device shared by all networks of the process: calls that
 * overlap in time race on it and must be serialised by the caller.
 * Returns after the copy has completed.
 */
#define EPROP_STATIC_RASTER_BYTES (16 * 1024 * 1024)
eprop_status eprop_readout_raster_static(eprop_net *net, uint8_t *raster, int32_t is_device);

/*
 * Copies the surrogate derivatives psi_j^t of the last simulate call
 * (Eq. piecewise-linear-surrogate-gradient), [batch][T][n_rec], 0 where the
 * neuron is refractory or the sample has ended.  Needs record_psi = 1.
 */
eprop_status eprop_read_surrogate(eprop_net *net, float *psi, int32_t is_device);

/* Counters of the last simulate call. */
typedef struct eprop_stats {
    int64_t events;           /* synapse events: one presynaptic spike transmitted
                                 through one synapse (sum of the out-degrees of
                                 all spikes emitted in the call)              */
    int64_t kernel_launches;  /* CUDA kernels the call issued                  */
    int64_t trace_launches;   /* of which synapse-trace kernels                */
    int64_t windows;          /* update windows that ended in the call         */
    double trace_ms;          /* device time of the synapse-trace kernels
                                 (CUDA events on the network's stream; needs
                                 profile = 1, else 0)                          */
} eprop_stats;

/* Fills *out with the counters of the last simulate call (waits for it). */
eprop_status eprop_get_stats(eprop_net *net, eprop_stats *out);

/* Autotuner of the launch shapes (form 2: the shapes of a call are picked
 * by measurement, not by a table).  The paper has no counterpart.  For each
 * candidate it replays one simulate call of the current inputs (after one
 * warm-up call that captures the CUDA graph in launch_mode 1), timed with
 * CUDA events on the network's stream, and restores the complete network
 * state (a device snapshot of every buffer and the host-side clock) after
 * each; then it applies the fastest candidate and restores the state once
 * more, so the network continues exactly as before the call.  Candidates:
 * blocks_per_sm 1..4 of the row kernels (delivery and synapse trace) and,
 * before the first simulate call of a batch-1 network that carries state,
 * trace_kernel 3 (dense window pass) and 1 (lazy).  The snapshot needs as
 * much device memory as the network holds (EPROP_ENOMEM otherwise).  out
 * receives the chosen shape and every candidate's time (ms per call). */
#define EPROP_TUNE_MAX 16
typedef struct eprop_tune_result {
    int32_t trace_kernel;
    int32_t blocks_per_sm;
    int32_t n_candidates;
    int32_t cand_trace_kernel[EPROP_TUNE_MAX];
    int32_t cand_blocks_per_sm[EPROP_TUNE_MAX];
    double cand_ms[EPROP_TUNE_MAX];
} eprop_tune_result;

eprop_status eprop_autotune(eprop_net *net, eprop_tune_result *out);

/* Waits for all issued work; returns EPROP_ECUDA / EPROP_ETIMEOUT on a
 * device error or a bounded wait that gave up. */
eprop_status eprop_sync(eprop_net *net);

/* Frees all device and host memory of the network (NULL is ignored). */
void eprop_destroy(eprop_net *net);

/* Message of the last error of `net`, or of the last failed create when
 * net is NULL.  Never NULL; valid until the next call on the same net. */
const char *eprop_last_error(const eprop_net *net);

#ifdef __cplusplus
}
#endif
#endif /* EPROP_H */
