/*
 * FP64 time-driven e-prop oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the slow, obviously-correct CPU definition of what the CUDA
 * library computes.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may build, load or call it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Each simulated step follows the paper's Methods in order:
 *   - LIF / ALIF membrane, threshold adaptation and spike   (Eq. lif_update,
 *     Eq. binary-spike-state-variable, Eq. spike-threshold-adaptation)
 *   - piecewise-linear surrogate gradient psi               (Eq. piecewise-
 *     linear-surrogate-gradient)
 *   - leaky readout y, error signal E (MSE or softmax CE)   (Eq. leaky_
 *     integrator, Eq. mean-squared-error, Eq. softmax, Eq. cross-entropy-loss)
 *   - learning signal L_j = sum_k B_jk E_k                  (Eq. final-gradient)
 *   - eligibility vector, eligibility trace, low-pass filter and per-step
 *     gradient g^t = L^t F_kappa(e^t)                       (Eq. eligibility-
 *     vector-substituted, Eq. filtered-eligibility-trace, Eq. gradient-rec,
 *     Eq. gradient-in, Eq. filter)
 *   - output-weight gradient E_k^t F_kappa(z_j^t)           (Eq. eprop-output-
 *     new-subs-rewritten with d = 0)
 *   - accumulated gradient and gradient-descent update      (Eq. accumulated-
 *     gradients, Eq. gradient-descent), averaged over the mini-batch.
 * This is the time-driven gradient computation of Algorithm 1 with the
 * weight update applied at the end of each update window.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - spike iff v - v_th > 0 (strict);
 *   - refractory period: after a spike at t, z = 0 and psi = 0 for the next
 *     t_ref steps, v keeps integrating;
 *   - input and recurrent spikes act through integer delays d >= 1:
 *     a source spike emitted at step s reaches its target at step s + d, both
 *     in the membrane input and in the presynaptic trace F_alpha (d = 1 gives
 *     the paper's z_i^{t-1} and, for inputs, x_i^{t-1});
 *   - the weight carried by a spike is the weight in effect at the step the
 *     spike is emitted (weights change only at update-window ends);
 *   - an external Poisson drive (non-plastic) adds drive_weight * n_j^t to the
 *     membrane input, n_j^t drawn by the SplitMix64 counter hash;
 *   - batch gradient = mean over samples of each sample's sum over steps.
 *
 * Besides the method's results the oracle keeps, for the parity tolerance,
 * the sum of the magnitudes of the terms of every accumulated sum: sum_t
 * |g^t| per weight and |y| accumulated with |W_out| (the condition of each
 * sum: FP32 rounding of a sum is bounded relative to it, not to the sum's
 * possibly cancelled value), and the sensitivity of each gradient to a
 * relative perturbation of the error signal: sum_t Lsens_j^t |ebar^t| with
 * Lsens_j^t = sum_k |B_jk| Esens_k^t, Esens = |y|_k + |y*_k| for MSE and
 * pi_k (|y|_k + sum_l pi_l |y|_l) + pi_k + pi*_k for softmax CE.  They do
 * not feed back into any result.
 *
 * Variants (e-prop+, Methods and Supplement), each off by default:
 *   - exponential surrogate psi = gamma exp(-beta |v - v_th|)  (Eq. exponential-
 *     surrogate-gradient);
 *   - fixed reset: the step after a spike the decayed membrane alpha v is
 *     replaced by v_reset (v^t = v_reset + I^t instead of alpha v - v_th + I);
 *     the reset stays outside the eligibility (it is a stop-gradient, as the
 *     soft reset is), so the eligibility vector keeps F_alpha;
 *   - temporal MSE: loss (1/K) sum_k (y_k - y*_k)^2, E_k = (2/K)(y_k - y*_k)
 *     (Eq. temporal-mse);
 *   - firing-rate regularisation with the exponential moving average
 *     f_j^t = beta_reg f_j^{t-1} + (1 - beta_reg) z_j^t (Eq. ema-rate), adding
 *     c_reg (f_j^t - f*) G_beta(e^t) to every synapse onto neuron j
 *     (Eq. ema-gradient); G_beta(e^t) = (1 - beta_reg) F_beta(e^t) is a second
 *     filtered copy of the same eligibility trace e^t; rates are in spikes
 *     per step;
 *   - fixed weight signs (Dale's law when the initial weights of each source
 *     share a sign): bit 0 input, bit 1 recurrent, bit 2 readout weights keep
 *     the sign of their initial value; an update that would cross zero stops
 *     at zero (a signed zero, keeping the sign);
 *   - Adam (Eq. adam, Eq. eta-adam-fast, Eq. delta-w-adam-fast): one Adam step
 *     per update window on the window's batch-mean gradient, k = number of
 *     steps taken, eta_k = eta sqrt(1 - b2^k) / (1 - b1^k),
 *     w -= eta_k m / (sqrt(v) + eps_hat) with the TensorFlow constant eps_hat;
 *   - ignore-and-fire neurons (Methods, "Scaling"): z_j^t = 1 iff
 *     (t_abs + phase_j) mod period == 0, whatever the membrane does; v and psi
 *     are still integrated; phase_j = (upper 32 bits of mix(if_seed ^ j))
 *     mod period.
 *   - generalized delays (Supplement, "Generalized delays"): the readout
 *     receives the recurrent spikes d_out steps late (Eq. leaky_integrator_
 *     with_delay), so the output gradient filters z^{t-d_out}; the learning
 *     signal of step tau reaches the recurrent layer at tau + d_ls and is
 *     paired there with the filtered eligibility trace of step tau - d_out
 *     (Eq. eprop-learning-signal-delay); signals that would arrive after a
 *     sample's end are dropped.  Rings of the recent spikes, traces and
 *     signals (indexed by the absolute step) hold what the pairing needs.
 *
 * E_override (optional, [B][T][K]): where window = 0, E^t is taken from it
 * instead of from the loss (the learned predictor's error estimate).
 *
 * Threads: the per-synapse loop of each step may run on several host
 * threads (OpenMP, when built with it); every synapse is updated by exactly
 * one thread and no sum crosses synapses, so the results do not depend on
 * the thread count.
 *
 * Teacher forcing: `forced` replaces the spikes z; `forced_psi` (optional)
 * replaces the surrogate values psi used by the traces, so that the trace
 * and gradient arithmetic can be compared in isolation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the per-synapse loop (1 without OpenMP); returns the count in
   effect. */
int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

typedef struct {
    int32_t n_in, n_rec, n_out, batch;
    int32_t neuron_model;         /* 0 LIF, 1 ALIF */
    int32_t t_ref, loss, feedback, update_interval, continuous, max_delay;
    int32_t n_drive_thr;
    double alpha, rho, kappa, kappa_e, beta_a, v_th, gamma, beta_sg;
    double lr, drive_weight;
    uint64_t drive_seed;
    const uint32_t *drive_thr;
    /* variants (see the header comment) */
    int32_t surrogate;            /* 0 piecewise linear, 1 exponential */
    int32_t reset_mode;           /* 0 soft, 1 fixed value */
    double v_reset;
    double c_reg, f_target, beta_reg;
    int32_t sign_mask;            /* bit 0 input, bit 1 recurrent, bit 2 readout */
    int32_t optimizer;            /* 0 SGD, 1 Adam */
    double adam_b1, adam_b2, adam_eps;
    int32_t if_period;            /* ignore-and-fire period in steps, 0: off */
    uint64_t if_seed;
    int32_t d_out, d_ls;          /* generalized delays (see the header comment) */
} oracle_cfg;

typedef struct {
    /* network: synapses in CSR by source; sources are the n_in inputs
       followed by the n_rec recurrent neurons */
    int64_t n_src, nnz;
    const int64_t *ptr;
    const int32_t *col;
    const uint8_t *delay;
    double *w;                    /* [nnz], updated in place */
    double *w_out;                /* [n_rec][n_out], updated in place */
    const uint8_t *out_mask;      /* [n_rec][n_out] 1 = readout synapse j -> k exists */
    const double *fb;             /* [n_rec][n_out] or NULL (B = W_out^T) */
    /* persistent state */
    double *v, *a, *psi_prev;     /* [B][N] */
    int32_t *ref;                 /* [B][N] */
    uint8_t *z_prev;              /* [B][N] */
    double *ring;                 /* [B][D+1][N] pending membrane input */
    uint8_t *src_hist;            /* [B][D+1][n_src] source spikes of the last D+1 steps */
    double *zbar, *epsa, *ebar;   /* [B][nnz] eligibility state */
    double *g;                    /* [nnz]  sum over samples of sum_t g^t */
    double *y, *zk;               /* [B][K], [B][N] */
    double *g_out;                /* [N][K] */
    double *grad_acc, *grad_out_acc; /* applied batch-mean gradients, summed */
    int64_t *counters;            /* [0] absolute step, [1] step inside run */
    double *g_abs, *g_out_abs;    /* sum_t |g^t| of the current window      */
    double *grad_abs_acc, *grad_out_abs_acc; /* the same, batch mean, summed */
    double *y_abs;                /* [B][K] kappa-filtered sum of |W_out| z  */
    double *g_lsens, *g_out_lsens;        /* sensitivity sums, current window */
    double *grad_lsens_acc, *grad_out_lsens_acc; /* the same, batch mean, summed */
    double *rate;                 /* [B][N] f_j of the rate regularisation */
    double *ebar_reg;             /* [B][nnz] F_beta(e) of each synapse */
    const uint8_t *w_neg, *w_out_neg; /* [nnz], [N][K] 1 where the initial weight is negative */
    double *adam_m, *adam_v;      /* [nnz] */
    double *adam_m_out, *adam_v_out; /* [N][K] */
    /* generalized delays: rings indexed by the absolute step */
    uint8_t *z_hist;              /* [B][d_out+1][N] recurrent spikes */
    double *ebar_hist;            /* [B][nnz][d_out+d_ls+1] filtered eligibility traces */
    double *L_hist, *Ls_hist;     /* [B][d_ls+1][N] learning signals and their sensitivities */
} oracle_state;

/* SplitMix64 output function (Steele, Lea & Flood 2014). */
static uint64_t mix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int drive_count(const oracle_cfg *c, int64_t b, int64_t t_abs, int64_t j) {
    uint64_t h = mix64(mix64(mix64(c->drive_seed ^ (uint64_t)j) ^ (uint64_t)t_abs) ^ (uint64_t)b);
    uint32_t u = (uint32_t)(h >> 32);
    int n = 0;
    for (int m = 0; m < c->n_drive_thr; ++m)
        if (u >= c->drive_thr[m]) n++;
    return n;
}

/* Phase of ignore-and-fire neuron j: (upper 32 bits of mix(if_seed ^ j)) mod
   period. */
static int64_t if_phase(const oracle_cfg *c, int64_t j) {
    return (int64_t)((uint32_t)(mix64(c->if_seed ^ (uint64_t)j) >> 32) % (uint32_t)c->if_period);
}

/* Weight after an update w - dw, kept on the side of zero of its initial
   value when its sign is fixed (neg: initial weight negative). */
static double signed_update(double w, double dw, int fixed, int neg) {
    double x = w - dw;
    if (!fixed) return x;
    if (neg) return x < 0.0 ? x : -0.0;
    return x > 0.0 ? x : 0.0;
}

/* One step of the per-synapse eligibility recursion (Eq. eligibility-vector-
 * substituted and Eq. filtered-eligibility-trace):
 *   eps_a^t = psi^{t-1} zbar^{t-1} + (rho - psi^{t-1} beta_a) eps_a^{t-1}
 *   zbar^t  = alpha zbar^{t-1} + s^t          (F_alpha of the arriving spike)
 *   e^t     = psi^t (zbar^t - beta_a eps_a^t)
 *   ebar^t  = kappa_e ebar^{t-1} + e^t        (F_kappa)
 * and returns the per-step gradient g^t = L^t ebar^t. */
static double eligibility_e(double alpha, double rho, double beta_a, double kappa_e, double psi_prev,
                            double psi, double arrive, double *zbar, double *epsa, double *ebar) {
    double epsa_new = psi_prev * (*zbar) + (rho - psi_prev * beta_a) * (*epsa);
    *zbar = alpha * (*zbar) + arrive;
    *epsa = epsa_new;
    double e = psi * ((*zbar) - beta_a * (*epsa));
    *ebar = kappa_e * (*ebar) + e;
    return e;
}

double oracle_eligibility_step(double alpha, double rho, double beta_a,
                               double kappa_e, double psi_prev, double psi,
                               double L, double arrive, double *zbar,
                               double *epsa, double *ebar) {
    eligibility_e(alpha, rho, beta_a, kappa_e, psi_prev, psi, arrive, zbar, epsa, ebar);
    return L * (*ebar);
}

/* Contribution of one presynaptic arrival to a synapse gradient.  In the
   event-driven form (Sec. "From time-driven to event-driven e-prop",
   event-driven weight updates) the gradient of a synapse is a sum over its
   presynaptic events, each weighted from the postsynaptic history: by
   linearity of the eligibility recursion in zbar, an arrival at step a adds
   Q_j(a) = sum_{t = a}^{b} L_j^t ebar^t, where ebar is the response of the
   recursion above to one unit arrival at a from a zero state and b is the
   last step of a's update window (width U).  Computed here from that
   definition, one forward run of the recursion per (a, j).  psi, L: [T][N]
   of one sample (row t-1 holds step t); Q: [T][N] (row a-1 holds a).  The
   sum over a synapse's arrivals of |Q_j(a)| is the condition of the
   event-driven sum, used by the parity tolerance. */
void oracle_arrival_contrib(double alpha, double rho, double beta_a, double kappa_e,
                            int32_t T, int32_t U, int64_t N, const double *psi,
                            const double *L, double *Q) {
    for (int32_t a = 1; a <= T; ++a) {
        const int32_t b = ((a + U - 1) / U) * U < T ? ((a + U - 1) / U) * U : T;
        for (int64_t j = 0; j < N; ++j) {
            double zbar = 0.0, epsa = 0.0, ebar = 0.0, q = 0.0;
            for (int32_t t = a; t <= b; ++t) {
                const double pp = t > 1 ? psi[(int64_t)(t - 2) * N + j] : 0.0;
                q += oracle_eligibility_step(alpha, rho, beta_a, kappa_e, pp,
                                             psi[(int64_t)(t - 1) * N + j],
                                             L[(int64_t)(t - 1) * N + j],
                                             t == a ? 1.0 : 0.0, &zbar, &epsa, &ebar);
            }
            Q[(int64_t)(a - 1) * N + j] = q;
        }
    }
}

/* Sampled synapses of a run whose postsynaptic history is given (teacher
   forcing with the surrogate values and readout of another implementation):
   each synapse s runs the recursion above over steps t = 1..T of the run
   from a zero state (psi^0 = 0), with its arrivals arrive[s][t-1] (its
   source's spike d steps before t), its target's psi[s][t-1] and learning
   signal L[s][t-1], and the learning signal's sensitivity Ls[s][t-1].
   Returns per synapse G = sum_t g^t (the gradient summed over every update
   window of the run, batch of one), mag = sum_t |g^t| and
   sens = sum_t Ls^t |ebar^t|, the parity condition of the sum as
   oracle_simulate keeps it. */
void oracle_synapse_sample(double alpha, double rho, double beta_a, double kappa_e,
                           int64_t S, int32_t T, const uint8_t *arrive, const double *psi,
                           const double *L, const double *Ls, double *G, double *mag,
                           double *sens) {
    for (int64_t s = 0; s < S; ++s) {
        const int64_t o = s * (int64_t)T;
        double zbar = 0.0, epsa = 0.0, ebar = 0.0, g = 0.0, m = 0.0, se = 0.0;
        for (int32_t t = 1; t <= T; ++t) {
            const double pp = t > 1 ? psi[o + t - 2] : 0.0;
            const double gt = oracle_eligibility_step(alpha, rho, beta_a, kappa_e, pp, psi[o + t - 1],
                                                      L[o + t - 1], (double)arrive[o + t - 1],
                                                      &zbar, &epsa, &ebar);
            g += gt;
            m += fabs(gt);
            se += Ls[o + t - 1] * fabs(ebar);
        }
        G[s] = g;
        mag[s] = m;
        sens[s] = se;
    }
}

static void reset_state(const oracle_cfg *c, oracle_state *s) {
    int64_t B = c->batch, N = c->n_rec, K = c->n_out, D1 = c->max_delay + 1;
    memset(s->v, 0, sizeof(double) * B * N);
    memset(s->a, 0, sizeof(double) * B * N);
    memset(s->psi_prev, 0, sizeof(double) * B * N);
    memset(s->ref, 0, sizeof(int32_t) * B * N);
    memset(s->z_prev, 0, B * N);
    memset(s->ring, 0, sizeof(double) * B * D1 * N);
    memset(s->src_hist, 0, B * D1 * s->n_src);
    memset(s->zbar, 0, sizeof(double) * B * s->nnz);
    memset(s->epsa, 0, sizeof(double) * B * s->nnz);
    memset(s->ebar, 0, sizeof(double) * B * s->nnz);
    memset(s->y, 0, sizeof(double) * B * K);
    memset(s->y_abs, 0, sizeof(double) * B * K);
    memset(s->zk, 0, sizeof(double) * B * N);
    memset(s->rate, 0, sizeof(double) * B * N);
    memset(s->ebar_reg, 0, sizeof(double) * B * s->nnz);
    memset(s->z_hist, 0, (size_t)B * (c->d_out + 1) * N);
    memset(s->ebar_hist, 0, sizeof(double) * B * s->nnz * (c->d_out + c->d_ls + 1));
    memset(s->L_hist, 0, sizeof(double) * B * (c->d_ls + 1) * N);
    memset(s->Ls_hist, 0, sizeof(double) * B * (c->d_ls + 1) * N);
    s->counters[1] = 0;
}

/* Runs T steps for every sample; returns 0 on success. */
int oracle_simulate(const oracle_cfg *c, oracle_state *s, int32_t T,
                    const int64_t *x_ptr, const int32_t *x_ids,
                    const double *targets, const uint8_t *window,
                    const int32_t *lengths, const uint8_t *forced,
                    double *y_rec, double *loss, uint8_t *raster,
                    double *margin, double *psi_rec, double *L_rec,
                    double *y_abs_rec, const double *forced_psi,
                    const double *E_override) {
    const int64_t B = c->batch, N = c->n_rec, K = c->n_out, NI = c->n_in;
    const int64_t D1 = c->max_delay + 1, NS = s->n_src, NNZ = s->nnz;
    const int64_t U = c->update_interval > 0 ? c->update_interval : T;
    if (!c->continuous) reset_state(c, s);
    double *psi = (double *)calloc(N, sizeof(double));
    double *L = (double *)calloc(N, sizeof(double));
    double *E = (double *)calloc(K, sizeof(double));
    double *pi = (double *)calloc(K, sizeof(double));
    double *Esens = (double *)calloc(K, sizeof(double));
    double *Ls = (double *)calloc(N, sizeof(double));
    uint8_t *z = (uint8_t *)calloc(N, 1);
    if (!psi || !L || !E || !pi || !z || !Esens || !Ls) return 1;
    for (int64_t b = 0; b < B; ++b) loss[b] = 0.0;

    for (int32_t t = 1; t <= T; ++t) {
        const int64_t t_abs = ++s->counters[0];
        ++s->counters[1];
        const int64_t slot = t_abs % D1;
        for (int64_t b = 0; b < B; ++b) {
            if (t > lengths[b]) continue;
            double *v = s->v + b * N, *a = s->a + b * N;
            double *psi_prev = s->psi_prev + b * N;
            int32_t *ref = s->ref + b * N;
            uint8_t *z_prev = s->z_prev + b * N;
            double *ring = s->ring + b * D1 * N;
            uint8_t *hist = s->src_hist + b * D1 * NS;
            double *y = s->y + b * K, *zk = s->zk + b * N;
            double *y_abs = s->y_abs + b * K;
            double *rate = s->rate + b * N;
            const int64_t bt = b * (int64_t)T + (t - 1);

            /* sources that spike at this step: inputs from the raster */
            memset(hist + slot * NS, 0, NS);
            for (int64_t q = x_ptr[bt]; q < x_ptr[bt + 1]; ++q)
                hist[slot * NS + x_ids[q]] = 1;

            /* neurons */
            for (int64_t j = 0; j < N; ++j) {
                double I = ring[slot * N + j];
                ring[slot * N + j] = 0.0;
                if (c->drive_weight != 0.0)
                    I += c->drive_weight * drive_count(c, b, t_abs, j);
                a[j] = c->rho * a[j] + z_prev[j];
                double vth = c->v_th + c->beta_a * a[j];
                if (c->reset_mode == 1)           /* fixed reset value */
                    v[j] = (z_prev[j] ? c->v_reset : c->alpha * v[j]) + I;
                else                              /* reset by subtraction */
                    v[j] = c->alpha * v[j] + I - z_prev[j] * vth;
                int refractory = ref[j] > 0;
                double m = v[j] - vth;
                if (forced)
                    z[j] = forced[bt * N + j];
                else if (c->if_period > 0)        /* ignore-and-fire */
                    z[j] = ((t_abs + if_phase(c, j)) % c->if_period) == 0 ? 1 : 0;
                else
                    z[j] = (!refractory && m > 0.0) ? 1 : 0;
                if (c->surrogate == 1) {
                    psi[j] = refractory ? 0.0 : c->gamma * exp(-c->beta_sg * fabs(m));
                } else {
                    double h = 1.0 - c->beta_sg * fabs(m);
                    psi[j] = refractory ? 0.0 : c->gamma * (h > 0.0 ? h : 0.0);
                }
                if (forced_psi) psi[j] = forced_psi[bt * N + j];
                if (refractory) ref[j] -= 1;
                if (z[j]) ref[j] = c->t_ref;
                raster[bt * N + j] = z[j];
                margin[bt * N + j] = m;
                if (psi_rec) psi_rec[bt * N + j] = psi[j];
                hist[slot * NS + NI + j] = z[j];
                rate[j] = c->beta_reg * rate[j] + (1.0 - c->beta_reg) * z[j];
            }

            /* readout, error signal, loss; the readout sees the recurrent
               spikes d_out steps late (Eq. leaky_integrator_with_delay) */
            uint8_t *zh = s->z_hist + b * (c->d_out + 1) * N;
            memcpy(zh + (t_abs % (c->d_out + 1)) * N, z, N);
            const uint8_t *zd = (t_abs - c->d_out >= 1) ? zh + ((t_abs - c->d_out) % (c->d_out + 1)) * N : NULL;
            const double win = window ? (double)window[bt] : 1.0;
            const double *tgt = targets + bt * K;
            for (int64_t k = 0; k < K; ++k) {
                double acc = 0.0, acc_abs = 0.0;
                for (int64_t j = 0; j < N; ++j)
                    if (zd && zd[j]) {
                        acc += s->w_out[j * K + k];
                        acc_abs += fabs(s->w_out[j * K + k]);
                    }
                y[k] = c->kappa * y[k] + acc;
                y_abs[k] = c->kappa * y_abs[k] + acc_abs;
                y_rec[bt * K + k] = y[k];
                if (y_abs_rec) y_abs_rec[bt * K + k] = y_abs[k];
            }
            if (c->loss == 0) {
                for (int64_t k = 0; k < K; ++k) {
                    double diff = y[k] - tgt[k];
                    E[k] = win * diff;
                    loss[b] += 0.5 * win * diff * diff;
                }
            } else if (c->loss == 2) {            /* temporal MSE */
                for (int64_t k = 0; k < K; ++k) {
                    double diff = y[k] - tgt[k];
                    E[k] = win * (2.0 / (double)K) * diff;
                    loss[b] += win * diff * diff / (double)K;
                }
            } else {
                double mx = y[0];
                for (int64_t k = 1; k < K; ++k) mx = y[k] > mx ? y[k] : mx;
                double den = 0.0;
                for (int64_t k = 0; k < K; ++k) den += exp(y[k] - mx);
                for (int64_t k = 0; k < K; ++k) {
                    pi[k] = exp(y[k] - mx) / den;
                    E[k] = win * (pi[k] - tgt[k]);
                    loss[b] -= win * tgt[k] * ((y[k] - mx) - log(den));
                }
            }
            /* learning signal */
            const double *Bm = c->feedback ? s->fb : s->w_out;
            /* sensitivity of E_k to a relative perturbation of the readout
               (its inputs summed in magnitude, y_abs) and of the target:
               MSE  E_k = y_k - y*_k:      |y|_abs,k + |y*_k|;
               CE   E_k = pi_k - pi*_k:    d pi_k = pi_k (dy_k - sum_l pi_l dy_l),
                    so pi_k (|y|_abs,k + sum_l pi_l |y|_abs,l) + pi_k + pi*_k
                    (the last two: rounding of pi_k and of the difference) */
            if (c->loss == 0) {
                for (int64_t k = 0; k < K; ++k) Esens[k] = win * (y_abs[k] + fabs(tgt[k]));
            } else if (c->loss == 2) {
                for (int64_t k = 0; k < K; ++k) Esens[k] = win * (2.0 / (double)K) * (y_abs[k] + fabs(tgt[k]));
            } else {
                double pya = 0.0;
                for (int64_t k = 0; k < K; ++k) pya += pi[k] * y_abs[k];
                for (int64_t k = 0; k < K; ++k)
                    Esens[k] = win * (pi[k] * (y_abs[k] + pya) + pi[k] + fabs(tgt[k]));
            }
            /* an external error signal where the target window is closed
               (the learned predictor's form): it stands in for E there, in
               the learning signal and the readout gradient; it enters as
               given, so its sensitivity is its own magnitude */
            if (E_override && win == 0.0)
                for (int64_t k = 0; k < K; ++k) {
                    E[k] = E_override[bt * K + k];
                    Esens[k] = fabs(E[k]);
                }
            for (int64_t j = 0; j < N; ++j) {
                double acc = 0.0, accs = 0.0;
                for (int64_t k = 0; k < K; ++k) {
                    acc += Bm[j * K + k] * E[k];
                    accs += fabs(Bm[j * K + k]) * Esens[k];
                }
                L[j] = acc;
                Ls[j] = accs;
                if (L_rec) L_rec[bt * N + j] = acc;
            }
            /* generalized delays (Eq. eprop-learning-signal-delay): the
               learning signal of step tau reaches the synapses at tau + d_ls
               and is paired with their filtered eligibility of tau - d_out */
            const int64_t RH = c->d_out + c->d_ls + 1;
            const int delayed = c->d_out != 0 || c->d_ls != 0;
            double *Lh = s->L_hist + b * (c->d_ls + 1) * N, *Lsh = s->Ls_hist + b * (c->d_ls + 1) * N;
            if (delayed) {
                memcpy(Lh + (t_abs % (c->d_ls + 1)) * N, L, sizeof(double) * N);
                memcpy(Lsh + (t_abs % (c->d_ls + 1)) * N, Ls, sizeof(double) * N);
            }
            const int64_t t_sig = t_abs - c->d_ls;            /* step of the arriving learning signal */
            const int64_t t_eli = t_sig - c->d_out;           /* step of the paired eligibility */
            const double *Ld = t_sig >= 1 ? Lh + (t_sig % (c->d_ls + 1)) * N : NULL;
            const double *Lsd = t_sig >= 1 ? Lsh + (t_sig % (c->d_ls + 1)) * N : NULL;

            /* eligibility traces and gradients, every synapse, every step;
               each synapse's state and sums are its own, so the sources may
               be visited by several threads (OpenMP) with identical results */
#pragma omp parallel for schedule(dynamic, 64)
            for (int64_t i = 0; i < NS; ++i) {
                for (int64_t q = s->ptr[i]; q < s->ptr[i + 1]; ++q) {
                    const int64_t j = s->col[q];
                    const int64_t d = s->delay[q];
                    double arrive = 0.0;
                    if (t_abs - d >= 1) arrive = hist[((t_abs - d) % D1) * NS + i];
                    const double e = eligibility_e(c->alpha, c->rho, c->beta_a, c->kappa_e, psi_prev[j],
                                                   psi[j], arrive, s->zbar + b * NNZ + q,
                                                   s->epsa + b * NNZ + q, s->ebar + b * NNZ + q);
                    double gt, gabs, lsens;
                    if (!delayed) {
                        gt = L[j] * s->ebar[b * NNZ + q];
                        lsens = Ls[j] * fabs(s->ebar[b * NNZ + q]);
                    } else {
                        double *eh = s->ebar_hist + (b * NNZ + q) * RH;
                        eh[t_abs % RH] = s->ebar[b * NNZ + q];
                        const double ed = (Ld && t_eli >= 1) ? eh[t_eli % RH] : 0.0;
                        gt = Ld ? Ld[j] * ed : 0.0;
                        lsens = Lsd ? Lsd[j] * fabs(ed) : 0.0;
                    }
                    gabs = fabs(gt);
                    if (c->c_reg != 0.0) {        /* Eq. ema-gradient */
                        double *er = s->ebar_reg + b * NNZ + q;
                        *er = c->beta_reg * (*er) + e;
                        const double greg = c->c_reg * (rate[j] - c->f_target) * (1.0 - c->beta_reg) * (*er);
                        gt += greg;
                        gabs += fabs(greg);
                    }
                    s->g[q] += gt;
                    s->g_abs[q] += gabs;
                    s->g_lsens[q] += lsens;
                }
            }
            for (int64_t j = 0; j < N; ++j) {
                zk[j] = c->kappa * zk[j] + (zd ? zd[j] : 0);   /* F_kappa(z^{t-d_out}) */
                for (int64_t k = 0; k < K; ++k)
                    if (s->out_mask[j * K + k]) {
                        s->g_out[j * K + k] += E[k] * zk[j];
                        s->g_out_abs[j * K + k] += fabs(E[k] * zk[j]);
                        s->g_out_lsens[j * K + k] += Esens[k] * zk[j];
                    }
            }
            for (int64_t j = 0; j < N; ++j) {
                psi_prev[j] = psi[j];
                z_prev[j] = z[j];
            }

            /* transmission of this step's spikes with the current weights */
            for (int64_t i = 0; i < NS; ++i) {
                if (!hist[slot * NS + i]) continue;
                for (int64_t q = s->ptr[i]; q < s->ptr[i + 1]; ++q) {
                    const int64_t tgt_slot = (t_abs + s->delay[q]) % D1;
                    ring[tgt_slot * N + s->col[q]] += s->w[q];
                }
            }
        }

        /* end of an update window: gradient descent with the batch mean */
        if (s->counters[1] % U == 0) {
            double eta = c->lr;
            if (c->optimizer == 1) {              /* Eq. eta-adam-fast */
                const double k = (double)(++s->counters[2]);
                eta = c->lr * sqrt(1.0 - pow(c->adam_b2, k)) / (1.0 - pow(c->adam_b1, k));
            }
            const int64_t nnz_in = s->ptr[NI];
            for (int64_t q = 0; q < NNZ; ++q) {
                double gm = s->g[q] / (double)B;
                double dw = c->lr * gm;
                if (c->optimizer == 1) {          /* Eq. delta-w-adam-fast */
                    s->adam_m[q] = c->adam_b1 * s->adam_m[q] + (1.0 - c->adam_b1) * gm;
                    s->adam_v[q] = c->adam_b2 * s->adam_v[q] + (1.0 - c->adam_b2) * gm * gm;
                    dw = eta * s->adam_m[q] / (sqrt(s->adam_v[q]) + c->adam_eps);
                }
                const int fixed = (c->sign_mask >> (q < nnz_in ? 0 : 1)) & 1;
                s->w[q] = signed_update(s->w[q], dw, fixed, s->w_neg[q]);
                s->grad_acc[q] += gm;
                s->g[q] = 0.0;
                s->grad_abs_acc[q] += s->g_abs[q] / (double)B;
                s->g_abs[q] = 0.0;
                s->grad_lsens_acc[q] += s->g_lsens[q] / (double)B;
                s->g_lsens[q] = 0.0;
            }
            for (int64_t j = 0; j < N; ++j) {
                for (int64_t k = 0; k < K; ++k) {
                    if (!s->out_mask[j * K + k]) continue;
                    double gm = s->g_out[j * K + k] / (double)B;
                    double dw = c->lr * gm;
                    if (c->optimizer == 1) {
                        double *mo = s->adam_m_out + j * K + k, *vo = s->adam_v_out + j * K + k;
                        *mo = c->adam_b1 * (*mo) + (1.0 - c->adam_b1) * gm;
                        *vo = c->adam_b2 * (*vo) + (1.0 - c->adam_b2) * gm * gm;
                        dw = eta * (*mo) / (sqrt(*vo) + c->adam_eps);
                    }
                    s->w_out[j * K + k] = signed_update(s->w_out[j * K + k], dw, (c->sign_mask >> 2) & 1,
                                                        s->w_out_neg[j * K + k]);
                    s->grad_out_acc[j * K + k] += gm;
                    s->g_out[j * K + k] = 0.0;
                    s->grad_out_abs_acc[j * K + k] += s->g_out_abs[j * K + k] / (double)B;
                    s->g_out_abs[j * K + k] = 0.0;
                    s->grad_out_lsens_acc[j * K + k] += s->g_out_lsens[j * K + k] / (double)B;
                    s->g_out_lsens[j * K + k] = 0.0;
                }
            }
        }
    }
    free(psi); free(L); free(E); free(pi); free(z); free(Esens); free(Ls);
    return 0;
}
