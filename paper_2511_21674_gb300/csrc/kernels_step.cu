// Per-step kernels: input injection, neuron update, readout and error
// signal, spike transmission through the delayed synapses.
#include <cstddef>

#include "eprop.h"
#include "eprop_internal.cuh"
#include "eprop_launch.h"

namespace eprop {

// list slot / ring helpers -------------------------------------------------

__device__ __forceinline__ int run_step(const Net &n, int i) { return n.clock->r_base + i; }
__device__ __forceinline__ long long abs_step(const Net &n, int i) { return n.clock->t_abs_base + i; }
__device__ __forceinline__ int win_start(const Net &n, int r) { return ((r - 1) / n.U) * n.U; }

__device__ __forceinline__ uint32_t *src_words(const Net &n, int b, int src) {
    return n.bits + ((long long)b * n.n_src + src) * n.RW;
}

// Appends `src` to the spike list of run step r of sample b and sets its
// bit; returns without a second entry if the bit was already set.
__device__ __forceinline__ void mark_spike(const Net &n, int b, int src, int r) {
    const int p = r & (n.RW * 32 - 1);
    uint32_t *wd = src_words(n, b, src) + (p >> 5);
    const uint32_t m = 1u << (p & 31);
    const uint32_t old = atomicOr(wd, m);
    if (old & m) return;
    const long long li = list_index(n, b, r % n.RS) + ((src >> 8) & (kBkt - 1));
    const int pos = atomicAdd(&n.list_cnt[li], 1);
    n.list_ids[li * n.list_cap + pos] = src;
}

// K9: input spikes of call step i ------------------------------------------
__global__ void inject_kernel(Net n, int i) {
    const int b = blockIdx.y;
    if (i > n.lengths[b]) return;
    const long long q0 = n.x_ptr[(long long)b * n.T + i - 1];
    const long long q1 = n.x_ptr[(long long)b * n.T + i];
    const int r = run_step(n, i);
    for (long long q = q0 + blockIdx.x * blockDim.x + threadIdx.x; q < q1;
         q += (long long)gridDim.x * blockDim.x)
        mark_spike(n, b, n.x_ids[q], r);
}

// One neuron's update at call step i from its loaded state (Eq. lif_update,
// Eq. binary-spike-state-variable, Eq. spike-threshold-adaptation, the
// surrogate): clears its ring slot, writes v, a, ref, z_prev, psi and the
// rate regularisation signal, and marks a spike.  Shared by the per-step
// neuron kernel and the persistent step loop.
// VAR: the e-prop+ variants (fixed reset, ignore-and-fire, exponential
// surrogate, rate regularisation) are compiled in; the plain method's
// instance carries none of their code.
template <bool VAR>
__device__ __forceinline__ void neuron_update(const Net &n, int i, int b, int j, long long nb, int r, int a0,
                                              long long t_abs, const uint32_t *thr_s, float *psi_row,
                                              long long *ring_row, long long acc_q, float v_hi_q, float v_lo_q,
                                              float a_hi_q, float a_lo_q, int ref_q, uint8_t zp8_q) {
    ring_row[j] = 0;
    // exact fixed-point input split into an FP32 pair
    const float acc_hi = (float)acc_q;
    float u_hi = acc_hi * kFixInv;
    float u_lo = (float)(acc_q - (long long)acc_hi) * kFixInv;
    if (n.n_thr > 0) {
        const uint64_t h = mix64(mix64(mix64(n.drive_seed ^ (uint64_t)j) ^ (uint64_t)t_abs) ^ (uint64_t)b);
        const uint32_t u = (uint32_t)(h >> 32);
        // thresholds are non-decreasing (checked at creation): the count of
        // thresholds <= u is the index of the first one above u
        int cnt = 0;
        while (cnt < n.n_thr && u >= thr_s[cnt]) ++cnt;
        const float dv = n.drive_weight * (float)cnt;
        const float de = fmaf(n.drive_weight, (float)cnt, -dv);
        float e;
        two_sum(u_hi, dv, u_hi, e);
        u_lo += e + de;
    }
    const float zp = (float)zp8_q;
    float vth = n.v_th, vth_lo = 0.0f;
    if (n.alif) {
        comp_step(n.rho, n.rho_lo, zp, 0.0f, a_hi_q, a_lo_q);
        n.a[nb] = a_hi_q;
        n.a_lo[nb] = a_lo_q;
        vth = fmaf(n.beta_a, a_hi_q, n.v_th);
        vth_lo = fmaf(n.beta_a, a_hi_q, n.v_th - vth) + n.beta_a * a_lo_q;
    }
    if (VAR && n.reset_mode == 1 && zp != 0.0f) {
        // fixed reset: v' = v_reset + I (the decayed membrane is replaced)
        float s, e;
        two_sum(n.v_reset, u_hi, s, e);
        const float lo = e + u_lo;
        const float hi = s + lo;
        v_lo_q = lo - (hi - s);
        v_hi_q = hi;
    } else {
        // v' = alpha v + I - z_prev v_th (Eq. lif_update), input term as a pair
        if (!VAR || n.reset_mode == 0) {
            float e;
            two_sum(u_hi, -zp * vth, u_hi, e);
            u_lo += e - zp * vth_lo;
        }
        comp_step(n.alpha, n.alpha_lo, u_hi, u_lo, v_hi_q, v_lo_q);
    }
    n.v[nb] = v_hi_q;
    n.v_lo[nb] = v_lo_q;
    const float m = (v_hi_q - vth) + (v_lo_q - vth_lo);
    const bool refractory = ref_q > 0;
    int z;
    if (n.forced) {
        z = n.forced[((long long)b * n.T + (i - 1)) * n.n_rec + j] ? 1 : 0;
    } else if (VAR && n.if_period > 0) {
        // ignore-and-fire: a fixed schedule with the neuron's own phase
        const uint32_t ph = (uint32_t)(mix64(n.if_seed ^ (uint64_t)j) >> 32) % (uint32_t)n.if_period;
        z = ((t_abs + (long long)ph) % n.if_period) == 0 ? 1 : 0;
    } else {
        z = (!refractory && m > 0.0f) ? 1 : 0;
    }
    float psi;
    if (VAR && n.surrogate == 1) {      // Eq. exponential-surrogate-gradient
        psi = refractory ? 0.0f : n.gamma * expf(-n.beta_sg * fabsf(m));
    } else {                     // Eq. piecewise-linear-surrogate-gradient
        const float hh = 1.0f - n.beta_sg * fabsf(m);
        psi = refractory ? 0.0f : n.gamma * fmaxf(hh, 0.0f);
    }
    psi_row[j] = psi;
    if (VAR && n.R_win) {
        // moving-average rate (Eq. ema-rate) and the regularisation
        // signal of Eq. ema-gradient, with G_beta's factor (1 - beta)
        const float f = n.beta_reg * n.rate[nb] + (1.0f - n.beta_reg) * (float)z;
        n.rate[nb] = f;
        n.R_win[((long long)b * n.U + (r - a0 - 1)) * n.n_rec + j] =
            n.c_reg * (1.0f - n.beta_reg) * (f - n.f_target);
    }
    if (n.record_psi) n.rec_psi[((long long)b * n.T + (i - 1)) * n.n_rec + j] = psi;
    int rf = ref_q;
    if (refractory) rf -= 1;
    if (z) rf = n.t_ref;
    n.ref[nb] = rf;
    n.z_prev[nb] = (uint8_t)z;
    if (z) {
        mark_spike(n, b, n.n_in + j, r);
        if (n.pop_cnt) atomicAdd(&n.pop_cnt[b * kPopGroups + (j & (kPopGroups - 1))], 1);
        if (n.record_raster) {
            const int W32 = (n.T + 31) / 32;
            atomicOr(&n.rec_raster[((long long)b * W32 + ((i - 1) >> 5)) * n.n_rec + j],
                     1u << ((i - 1) & 31));
        }
    }
}

// K1: LIF / ALIF neuron update (Eq. lif_update, Eq. binary-spike-state-
// variable, Eq. spike-threshold-adaptation, Eq. piecewise-linear-surrogate-
// gradient).  Each thread updates kNPT neurons of one sample (strided by the
// block size, so every access stays coalesced): the clock and the drive
// table are read once per block, then the state of all kNPT neurons is
// loaded in one batch (one memory round trip for the batch), updated, and
// stored.  Two neurons per thread (twice the blocks of four per thread)
// measured faster on the million-neuron workload.
constexpr int kNPT = 2;
constexpr int kNeuronThreads = 256;

template <bool VAR>
__global__ void __launch_bounds__(kNeuronThreads) neuron_kernel(Net n, int i) {
    __shared__ uint32_t thr_s[EPROP_MAX_DRIVE_THR];
    __shared__ Clock ck_s;
    __shared__ int len_s;
    const int b = blockIdx.y;
    if (threadIdx.x == 0) {
        ck_s = *n.clock;
        len_s = n.lengths[b];
    }
    for (int m = threadIdx.x; m < n.n_thr; m += blockDim.x) thr_s[m] = n.drive_thr[m];
    __syncthreads();
    const Clock ck = ck_s;
    const int len = len_s;
    const int r = ck.r_base + i;
    const int a0 = ((r - 1) / n.U) * n.U;
    const long long t_abs = ck.t_abs_base + i;
    const int slot = (ck.ring0 + i) % (n.D + 1);
    float *psi_row = n.psi_hist + ((long long)b * (n.U + 1) + (r - a0)) * n.n_rec;
    long long *ring_row = n.ring + ((long long)b * (n.D + 1) + slot) * n.n_rec;
    const long long nb0 = (long long)b * n.n_rec;
    // the grid holds as many blocks as are resident at once; each block
    // walks groups of kNeuronThreads * kNPT neurons
    for (int jg = blockIdx.x * (kNeuronThreads * kNPT); jg < n.n_rec; jg += gridDim.x * (kNeuronThreads * kNPT)) {
    const int jb = jg + threadIdx.x;
    if (i > len) {               // sample already finished: frozen, silent
#pragma unroll
        for (int q = 0; q < kNPT; ++q) {
            const int j = jb + q * kNeuronThreads;
            if (j >= n.n_rec) break;
            psi_row[j] = 0.0f;
            if (n.R_win) n.R_win[((long long)b * n.U + (r - a0 - 1)) * n.n_rec + j] = 0.0f;
            if (n.record_psi) n.rec_psi[((long long)b * n.T + (i - 1)) * n.n_rec + j] = 0.0f;
        }
        continue;
    }
    // batch of loads
    float v_hi[kNPT], v_lo[kNPT], a_hi[kNPT], a_lo[kNPT];
    int ref[kNPT];
    uint8_t zp8[kNPT];
    long long acc[kNPT];
#pragma unroll
    for (int q = 0; q < kNPT; ++q) {
        const int j = jb + q * kNeuronThreads;
        const bool in = j < n.n_rec;
        const long long nb = nb0 + (in ? j : 0);
        v_hi[q] = in ? n.v[nb] : 0.f;
        v_lo[q] = in ? n.v_lo[nb] : 0.f;
        a_hi[q] = (in && n.alif) ? n.a[nb] : 0.f;
        a_lo[q] = (in && n.alif) ? n.a_lo[nb] : 0.f;
        ref[q] = in ? n.ref[nb] : 0;
        zp8[q] = in ? n.z_prev[nb] : 0;
        acc[q] = in ? ring_row[j] : 0;
    }
#pragma unroll
    for (int q = 0; q < kNPT; ++q) {
        const int j = jb + q * kNeuronThreads;
        if (j >= n.n_rec) break;
        const long long nb = nb0 + j;
        neuron_update<VAR>(n, i, b, j, nb, r, a0, t_abs, thr_s, psi_row, ring_row, acc[q], v_hi[q], v_lo[q],
                      a_hi[q], a_lo[q], ref[q], zp8[q]);
    }
    }
}

constexpr int kReadoutChunk = 16;    // spikes per readout block and round

__device__ float block_sum(float x, float *sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = x;
    __syncthreads();
    float t = 0.0f;
    const int nw = (blockDim.x + 31) >> 5;
    for (int q = 0; q < nw; ++q) t += sh[q];
    return t;
}

__device__ float block_max(float x, float *sh) {
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = x;
    __syncthreads();
    float t = -INFINITY;
    const int nw = (blockDim.x + 31) >> 5;
    for (int q = 0; q < nw; ++q) t = fmaxf(t, sh[q]);
    return t;
}

// K3b: leaky readout (Eq. leaky_integrator), error signal and loss
// (Eq. mean-squared-error / Eq. softmax, Eq. cross-entropy-loss) of sample b,
// by one whole CTA, thread = readout k (blockDim multiple of 32, >= n_out).
__device__ void readout_finish(const Net &n, int i, int b) {
    __shared__ float sh[32];
    const int k = threadIdx.x;
    const bool has_k = k < n.n_out;
    const int r = run_step(n, i);
    const int a0 = win_start(n, r);
    const long long bk = (long long)b * n.n_out + k;
    float *E = n.E_win + ((long long)b * n.U + (r - a0 - 1)) * n.n_out;
    if (i > n.lengths[b]) {      // after the sample's end: no error, no output
        if (has_k) {
            E[k] = 0.0f;
            n.y_rec[((long long)b * n.T + (i - 1)) * n.n_out + k] = 0.0f;
        }
        return;
    }
    float y = 0.0f;
    if (has_k) {
        const long long acc = __ldcg(n.y_acc + bk);     // summed by atomics in L2
        n.y_acc[bk] = 0;
        y = n.kappa * n.y[bk] + (float)acc * kFixInv;
        n.y[bk] = y;
        n.y_rec[((long long)b * n.T + (i - 1)) * n.n_out + k] = y;
    }
    const float win = n.window ? (float)n.window[(long long)b * n.T + (i - 1)] : 1.0f;
    const float tgt = has_k ? n.targets[((long long)b * n.T + (i - 1)) * n.n_out + k] : 0.0f;
    float l;
    if (n.loss == 0) {
        const float diff = y - tgt;
        if (has_k) E[k] = win * diff;
        l = has_k ? 0.5f * win * diff * diff : 0.0f;
    } else if (n.loss == 2) {        // temporal MSE (Eq. temporal-mse)
        const float diff = y - tgt;
        const float invK = 1.0f / (float)n.n_out;
        if (has_k) E[k] = win * (2.0f * invK) * diff;
        l = has_k ? win * diff * diff * invK : 0.0f;
    } else {
        const float mx = block_max(has_k ? y : -INFINITY, sh);
        const float ex = has_k ? expf(y - mx) : 0.0f;
        const float den = block_sum(ex, sh);
        if (has_k) E[k] = win * (ex / den - tgt);
        l = has_k ? -win * tgt * ((y - mx) - logf(den)) : 0.0f;
    }
    const float tot = block_sum(l, sh);
    if (threadIdx.x == 0) n.loss_acc[b] += tot;
}

// K3a: readout input sum_j W_out[j][k] z_j^t in exact fixed point; one CTA per
// (chunk of the step's spike list, sample); thread = readout k; the last CTA
// of a sample then runs K3b for it.
__global__ void readout_accum_kernel(Net n, int i, int chunk) {
    __shared__ int srcs[kReadoutChunk];
    __shared__ int incl[kBkt];
    __shared__ int last;
    const int b = blockIdx.y;
    if (i > n.lengths[b]) {                  // finished sample: block 0 writes the zeros
        if (blockIdx.x == 0) readout_finish(n, i, b);
        return;
    }
    // the readout receives the recurrent spikes d_out steps late (Eq.
    // leaky_integrator_with_delay): the spike list of run step r - d_out
    const int rs = run_step(n, i) - n.d_out;
    const long long li = list_index(n, b, (rs >= 1 ? rs : 1) % n.RS);
    const int *cnt = n.list_cnt + li;
    const int *ids = n.list_ids + li * n.list_cap;
    if (threadIdx.x < 32) {
        const BucketScan bs = bucket_scan(cnt);
        incl[threadIdx.x] = bs.incl;
    }
    __syncthreads();
    const int total = rs >= 1 ? incl[kBkt - 1] : 0;
    for (int c0 = blockIdx.x * chunk; c0 < total; c0 += gridDim.x * chunk) {
        const int c1 = min(c0 + chunk, total);
        // every entry of the chunk resolved in parallel: bucket = first
        // bucket whose inclusive count exceeds the entry's rank
        for (int t = threadIdx.x; t < c1 - c0; t += blockDim.x) {
            const int c = c0 + t;
            int bk = 0;
            while (incl[bk] <= c) ++bk;
            srcs[t] = ids[(long long)bk * n.list_cap + (c - (bk > 0 ? incl[bk - 1] : 0))];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < n.n_out; k += blockDim.x) {
            long long acc = 0;
            for (int c = 0; c < c1 - c0; ++c) {
                const int src = srcs[c];
                if (src < n.n_in) continue;
                acc += __float2ll_rn(n.w_out[(long long)(src - n.n_in) * n.n_out + k] * 4294967296.0f);
            }
            if (acc) atomicAdd(reinterpret_cast<unsigned long long *>(&n.y_acc[(long long)b * n.n_out + k]),
                               (unsigned long long)acc);
        }
        __syncthreads();
    }
    // the sample's last block to finish forms y, E and the loss
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&n.ro_done[b], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) n.ro_done[b] = 0;
    readout_finish(n, i, b);
}

// Predictor inputs of step i (one block per sample): the readout
// potentials y^t and the group rates r_g = beta r_g + (1 - beta) * (spikes of
// group g at this step) / |group| (Eq. ema-rate on group means), given in
// spikes per 1000 steps (the paper's rate unit).
__global__ void pred_input_kernel(Net n, int i) {
    const int b = blockIdx.x;
    const int K = n.n_out;
    const bool live = i <= n.lengths[b];
    float *x = n.pred_x + (long long)b * n.pred_in;
    for (int g = threadIdx.x; g < kPopGroups; g += blockDim.x) {
        const long long o = (long long)b * kPopGroups + g;
        const int c = n.pop_cnt[o];
        n.pop_cnt[o] = 0;
        const float rr = n.pop_beta * n.pop_rate[o] + (1.0f - n.pop_beta) * ((float)c * n.pop_inv[g]);
        n.pop_rate[o] = rr;
        x[K + g] = 1000.0f * rr;         // spikes per 1000 steps
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) x[k] = live ? n.y[(long long)b * K + k] : 0.0f;
    __syncthreads();
    if (n.pred_mode & 2) {
        float *rec = n.pred_rec + ((long long)b * n.T + (i - 1)) * n.pred_in;
        for (int q = threadIdx.x; q < n.pred_in; q += blockDim.x) rec[q] = x[q];
    }
}

// Where the sample's target window is closed, the predicted error signal
// stands in for E^t (learning signal and readout gradient of the window).
__global__ void pred_apply_kernel(Net n, int i) {
    const int b = blockIdx.x;
    const int k = threadIdx.x;
    if (k >= n.n_out || i > n.lengths[b]) return;
    if (n.window && n.window[(long long)b * n.T + (i - 1)]) return;
    const int r = run_step(n, i);
    const int a0 = win_start(n, r);
    n.E_win[((long long)b * n.U + (r - a0 - 1)) * n.n_out + k] = n.pred_y[(long long)b * n.n_out + k];
}

// Issues the bulk copies of one chunk (cnt records from q0) into a stage
// (one thread).  4-byte streams start at q_al = q0 rounded down to 4
// elements, the 2-byte trace stream at q0 rounded down to 8 elements, so
// every copy starts and ends on 16-byte boundaries (the record arrays are
// padded past nnz).
__device__ __forceinline__ void issue_chunk(const Net &n, StageBuf &sb, uint64_t *bar, long long q0, int cnt,
                                            bool with_trace, StageDesc &dsc) {
    const long long q_al = q0 & ~3LL;
    const uint32_t n4 = (uint32_t)((q0 + cnt - q_al + 3) & ~3LL);
    long long q_al2 = q_al;
    uint32_t tr_bytes = 0;
    if (with_trace) {
        if (n.trace_bf16) {
            q_al2 = q0 & ~7LL;
            tr_bytes = (uint32_t)((q0 + cnt - q_al2 + 7) & ~7LL) * 2u;
        } else {
            tr_bytes = n4 * 4u;
        }
    }
    mbar_expect_tx(bar, n4 * 8u + tr_bytes);
    bulk_g2s(sb.td, n.tgt_d + q_al, n4 * 4u, bar);
    bulk_g2s(sb.w, n.w + q_al, n4 * 4u, bar);
    if (with_trace) {
        if (n.trace_bf16) bulk_g2s(sb.tr, reinterpret_cast<const uint16_t *>(n.ebar) + q_al2, tr_bytes, bar);
        else bulk_g2s(sb.tr, reinterpret_cast<const float *>(n.ebar) + q_al, tr_bytes, bar);
    }
    dsc.q0 = q0;
    dsc.q_al = q_al;
    dsc.q_al2 = q_al2;
    dsc.n = cnt;
}

__device__ __forceinline__ float stage_trace(const Net &n, const StageBuf &sb, const StageDesc &d, long long q) {
    if (n.trace_bf16)
        return trace16_to_float(reinterpret_cast<const uint16_t *>(sb.tr)[q - d.q_al2], n.trace_type);
    return reinterpret_cast<const float *>(sb.tr)[q - d.q_al];
}

constexpr int kDStages = 3;
__host__ __device__ constexpr size_t deliver_stage_bytes(bool state) {
    return state ? sizeof(StageBuf) : offsetof(StageBuf, tr);
}

// K2: transmission of the spikes of call step i.  Each warp walks its share
// of the step's spiking rows as a sequence of chunks of kChunk synapse
// records; a kDStages-deep pipeline of bulk copies (TMA, 1-D) streams the
// records into shared memory while earlier chunks are delivered.  The
// weight carried is the weight in effect at emission: with per-synapse lazy
// updates, the gradient of update windows that closed since the synapse's
// last arrival is added on the fly (read-only).  Arrivals are summed in
// exact int64 fixed point.
template <bool ALIF, bool STATE>
__global__ void __launch_bounds__(256, STATE ? 2 : 4) deliver_kernel(Net n, int i) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ uint64_t bars[8][kDStages];
    __shared__ StageDesc desc[8][kDStages];
    __shared__ RowInfo info[8][STATE ? kDStages : 1][kMaxDelay + 1];
    __shared__ unsigned long long ev_block;
    __shared__ long long ring_off[kMaxDelay + 1];
    const int b = blockIdx.y;
    // the list slot of step r + 1 (filled by the next neuron update) was last
    // used RS steps ago; every reader of it has finished: the delivery and
    // window kernels of that step come earlier on this stream, its readout
    // before the last window end (RS = U + D + 1 > U), and with RS = 2 the
    // readout runs on this stream
    if (blockIdx.x == 0 && threadIdx.x < kBkt)
        n.list_cnt[list_index(n, b, (run_step(n, i) + 1) % n.RS) + threadIdx.x] = 0;
    if (i > n.lengths[b]) return;            // whole block: same sample
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // without carried state the trace stream is not staged: stages are the
    // (j|d, w) part of a StageBuf only
    constexpr size_t kStride = deliver_stage_bytes(STATE);
    auto buf = [&](int k) -> StageBuf & {
        return *reinterpret_cast<StageBuf *>(dsm + (size_t)(warp * kDStages + k) * kStride);
    };
    if (threadIdx.x == 0) ev_block = 0ULL;
    if (threadIdx.x <= n.D)                  // ring slot of an arrival d steps ahead
        ring_off[threadIdx.x] = (long long)((n.clock->ring0 + i + (int)threadIdx.x) % (n.D + 1)) * n.n_rec;
    if (lane < kDStages) mbar_init(&bars[warp][lane], 1);
    fence_mbar_init();
    __syncthreads();
    unsigned long long ev_warp = 0ULL;
    const int r = run_step(n, i);
    const int a0 = win_start(n, r);
    const int k1 = a0 / n.U;                 // windows < k1 are closed
    const long long li = list_index(n, b, r % n.RS);
    const int *ids = n.list_ids + li * n.list_cap;
    const BucketScan bs = bucket_scan(n.list_cnt + li);
    const int D1 = n.D + 1;
    long long *ring_b = n.ring + (long long)b * D1 * n.n_rec;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    const int nw = gridDim.x * (blockDim.x >> 5);
    // producer cursor (warp-uniform)
    // work items: (spiking row, one of kDParts equal parts of its synapses),
    // dealt round-robin to the warps; a step has about as many spiking rows
    // as there are warps, and whole rows would leave most warps idle while
    // a few finish a second row
    constexpr int kDParts = 4;
    int prow = gw;
    long long pq = 0, pre = 0;
    int psrc = -1, pfirst = 0;
    RowInfo rinfo;
    unsigned vmask = 0;
    auto next_item = [&]() -> bool {
        while (pq >= pre) {
            if (prow >= bs.total * kDParts) return false;
            const int row = prow / kDParts, part = prow % kDParts;
            psrc = bucket_entry(n, ids, bs, row);
            const long long rb = n.row_ptr[psrc], len = n.row_ptr[psrc + 1] - rb;
            pq = rb + len * part / kDParts;
            pre = rb + len * (part + 1) / kDParts;
            prow += nw;
            pfirst = 1;
            if (STATE && pre > pq && lane >= 1 && lane <= n.D)
                rinfo = row_info(n, src_words(n, b, psrc), n.anchor_t[(long long)b * n.n_src + psrc],
                                 n.anchor_z[(long long)b * n.n_src + psrc], a0, lane, false);
        }
        return true;
    };
    for (int k = 0; k < kDStages; ++k) {
        if (!next_item()) break;
        const int cnt = (int)min((long long)kChunk, pre - pq);
        if (STATE && lane >= 1 && lane <= n.D) info[warp][k][lane] = rinfo;
        if (lane == 0) {
            issue_chunk(n, buf(k), &bars[warp][k], pq, cnt, STATE, desc[warp][k]);
            desc[warp][k].first = pfirst;
            desc[warp][k].row = (int)(pre - pq);
        }
        pq += cnt;
        pfirst = 0;
        vmask |= 1u << k;
    }
    __syncwarp();
    int abort_c = -1;
    for (int c = 0;; ++c) {
        const int k = c % kDStages;
        if (!((vmask >> k) & 1u)) break;
        if (!mbar_wait(&bars[warp][k], (uint32_t)((c / kDStages) & 1), n.err_flags)) {
            abort_c = c;
            break;
        }
        const StageDesc d = desc[warp][k];
        if (d.first && lane == 0) ev_warp += (unsigned long long)d.row;
        const StageBuf &sb = buf(k);
#pragma unroll 2
        for (int h = 0; h < kChunk / 32; h += 4) {
            uint32_t td[4];
            float wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = lane + 32 * (h + u);
                const long long q = d.q0 + idx;
                td[u] = idx < d.n ? sb.td[q - d.q_al] : 0u;
                wv[u] = idx < d.n ? sb.w[q - d.q_al] : 0.f;
            }
            if (STATE) {
                // lazily pending windows k0 .. k1-1: prefetch the first two
                // windows' coefficients, then advance
                float eb[4];
                Coef cf0[4], cf1[4];
                int k0s[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    k0s[u] = -1;
                    eb[u] = 0.f;
                    if (td[u] == 0u) continue;
                    const RowInfo ri = info[warp][k][td[u] >> 24];
                    if (ri.b_prev == kNoSpike || ri.b_prev >= a0) continue;
                    const long long q = d.q0 + lane + 32 * (h + u);
                    const long long j = td[u] & 0xFFFFFFu;
                    int k0 = ri.k_prev;
                    if (k1 - k0 > n.RC) {
                        atomicOr(n.err_flags, 1u);
                        k0 = k1 - n.RC;
                    }
                    k0s[u] = k0;
                    eb[u] = stage_trace(n, sb, d, q);
                    cf0[u] = load_coef<ALIF>(n, j, k0);
                    if (k0 + 1 < k1) cf1[u] = load_coef<ALIF>(n, j, k0 + 1);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (k0s[u] < 0) continue;
                    const int k0 = k0s[u];
                    const long long q = d.q0 + lane + 32 * (h + u);
                    const long long j = td[u] & 0xFFFFFFu;
                    float zbar = info[warp][k][td[u] >> 24].zbar_bp;
                    float ebar = eb[u], G = 0.f;
                    float epsa = ALIF ? load_trace(n.epsa, q, n.trace_type) : 0.f;
                    apply_coef<ALIF>(n, cf0[u], zbar, epsa, ebar, G);
                    if (k0 + 1 < k1) apply_coef<ALIF>(n, cf1[u], zbar, epsa, ebar, G);
                    for (int kk = k0 + 2; kk < k1; ++kk) apply_window<ALIF>(n, j, kk, zbar, epsa, ebar, G);
                    wv[u] -= n.lr * G;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (td[u] == 0u) continue;
                const int j = (int)(td[u] & 0xFFFFFFu);
                const int dl = (int)(td[u] >> 24);
                const long long fx = __float2ll_rn(wv[u] * 4294967296.0f);
                atomicAdd(reinterpret_cast<unsigned long long *>(&ring_b[ring_off[dl] + j]),
                          (unsigned long long)fx);
            }
        }
        __syncwarp();
        // refill stage k with the next chunk
        vmask &= ~(1u << k);
        if (next_item()) {
            const int cnt = (int)min((long long)kChunk, pre - pq);
            if (STATE && lane >= 1 && lane <= n.D) info[warp][k][lane] = rinfo;
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async();
                issue_chunk(n, buf(k), &bars[warp][k], pq, cnt, STATE, desc[warp][k]);
                desc[warp][k].first = pfirst;
                desc[warp][k].row = (int)(pre - pq);
            }
            pq += cnt;
            pfirst = 0;
            vmask |= 1u << k;
        }
        __syncwarp();
    }
    if (abort_c >= 0) {                      // let copies in flight land first
        for (int c = abort_c + 1; c < abort_c + kDStages; ++c)
            if ((vmask >> (c % kDStages)) & 1u)
                mbar_wait(&bars[warp][c % kDStages], (uint32_t)((c / kDStages) & 1), n.err_flags);
    }
    if (lane == 0 && ev_warp) atomicAdd(&ev_block, ev_warp);
    __syncthreads();
    if (threadIdx.x == 0 && ev_block) atomicAdd(n.events, ev_block);
}

// ---------------------------------------------------- persistent step loop
//
// Form (2): all T steps of a single-window call in one cooperative launch
// (captured in the call's CUDA graph like any kernel).  Per step two phases
// separated by grid barriers:
//   A  readout finish of step i - 1 (one block per sample), input injection
//      and every neuron update of step i;
//   B  readout accumulation and spike delivery of step i (warps dealt to
//      samples, each warp walking its share of the sample's spike list).
// The arithmetic is that of the per-step kernels (the neuron update is the
// same device function, readout and ring sums are the same exact int64
// fixed-point additions), so the results are bit-identical to them.  The
// barrier waits are bounded: a wait that gives up sets error bit 2 and an
// abort flag that every block checks, so all blocks leave the loop.

constexpr int kPersThreads = 256;
constexpr unsigned kBarrierLimit = 1u << 22;

__device__ bool grid_barrier(GridBar *gb, unsigned nblocks, unsigned *err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        volatile unsigned *vgen = &gb->gen;
        volatile unsigned *vab = &gb->abort;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            unsigned it = 0;
            while (*vgen == g) {
                if (*vab || ++it > kBarrierLimit) {
                    atomicOr(err, 4u);
                    atomicExch(&gb->abort, 1u);
                    s_ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(kPersThreads) persistent_steps_kernel(Net n, int T, GridBar *gb) {
    __shared__ uint32_t thr_s[EPROP_MAX_DRIVE_THR];
    for (int m = threadIdx.x; m < n.n_thr; m += blockDim.x) thr_s[m] = n.drive_thr[m];
    const Clock ck = *n.clock;                   // constant during a call
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)(tid >> 5), nwarps = (int)(nth >> 5);
    const int ws = max(1, nwarps / n.B);         // warps per sample in phase B
    const int D1 = n.D + 1;
    __syncthreads();
    for (int i = 1; i <= T; ++i) {
        const int r = ck.r_base + i;
        const int a0 = ((r - 1) / n.U) * n.U;
        const long long t_abs = ck.t_abs_base + i;
        const int slot = (ck.ring0 + i) % D1;
        // ---- phase A
        if (i > 1)
            for (int b = blockIdx.x; b < n.B; b += gridDim.x) readout_finish(n, i - 1, b);
        if (n.n_in > 0)                          // input spikes: one warp per sample
            for (int b = gwarp; b < n.B; b += nwarps) {
                if (i > n.lengths[b]) continue;
                const long long q0 = n.x_ptr[(long long)b * n.T + i - 1];
                const long long q1 = n.x_ptr[(long long)b * n.T + i];
                for (long long q = q0 + lane; q < q1; q += 32) mark_spike(n, b, n.x_ids[q], r);
            }
        for (long long idx = tid; idx < (long long)n.B * n.n_rec; idx += nth) {
            const int b = (int)(idx / n.n_rec), j = (int)(idx - (long long)b * n.n_rec);
            float *psi_row = n.psi_hist + ((long long)b * (n.U + 1) + (r - a0)) * n.n_rec;
            long long *ring_row = n.ring + ((long long)b * D1 + slot) * n.n_rec;
            if (i > n.lengths[b]) {              // sample already finished: frozen, silent
                psi_row[j] = 0.0f;
                if (n.R_win) n.R_win[((long long)b * n.U + (r - a0 - 1)) * n.n_rec + j] = 0.0f;
                if (n.record_psi) n.rec_psi[((long long)b * n.T + (i - 1)) * n.n_rec + j] = 0.0f;
                continue;
            }
            neuron_update<true>(n, i, b, j, idx, r, a0, t_abs, thr_s, psi_row, ring_row, ring_row[j], n.v[idx],
                          n.v_lo[idx], n.alif ? n.a[idx] : 0.f, n.alif ? n.a_lo[idx] : 0.f, n.ref[idx],
                          n.z_prev[idx]);
        }
        if (!grid_barrier(gb, gridDim.x, n.err_flags)) return;
        // ---- phase B
        for (int vw = gwarp; vw < n.B * ws; vw += nwarps) {
            const int b = vw / ws, sub = vw - b * ws;
            const long long li = list_index(n, b, r % n.RS);
            if (sub == 0 && lane < kBkt)         // next step's list slot (its readers are done)
                n.list_cnt[list_index(n, b, (r + 1) % n.RS) + lane] = 0;
            if (i > n.lengths[b]) continue;
            const int *ids = n.list_ids + li * n.list_cap;
            const BucketScan bs = bucket_scan(n.list_cnt + li);
            long long *ring_b = n.ring + (long long)b * D1 * n.n_rec;
            unsigned long long ev = 0;
            for (int e = sub; e < bs.total; e += ws) {
                const int src = bucket_entry(n, ids, bs, e);
                const long long rb = n.row_ptr[src], re = n.row_ptr[src + 1];
                ev += (unsigned long long)(re - rb);
                if (src >= n.n_in)               // readout input sum_j W_out[j][k] z_j (exact)
                    for (int k = lane; k < n.n_out; k += 32) {
                        const long long fx =
                            __float2ll_rn(n.w_out[(long long)(src - n.n_in) * n.n_out + k] * 4294967296.0f);
                        if (fx) atomicAdd(reinterpret_cast<unsigned long long *>(&n.y_acc[(long long)b * n.n_out + k]),
                                          (unsigned long long)fx);
                    }
                for (long long q = rb + lane; q < re; q += 32) {
                    const uint32_t td = n.tgt_d[q];
                    const int j = (int)(td & 0xFFFFFFu), dl = (int)(td >> 24);
                    const long long fx = __float2ll_rn(n.w[q] * 4294967296.0f);
                    atomicAdd(reinterpret_cast<unsigned long long *>(
                                  &ring_b[(long long)((ck.ring0 + i + dl) % D1) * n.n_rec + j]),
                              (unsigned long long)fx);
                }
            }
            if (lane == 0 && ev) atomicAdd(n.events, ev);
        }
        if (!grid_barrier(gb, gridDim.x, n.err_flags)) return;
    }
    for (int b = blockIdx.x; b < n.B; b += gridDim.x) readout_finish(n, T, b);
}

// ----------------------------------------------------------------- launches

void launch_inject(const Net &n, int i, int max_events_per_step, cudaStream_t st) {
    if (n.n_in == 0) return;
    int blocks = (max_events_per_step + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 64) blocks = 64;
    inject_kernel<<<dim3(blocks, n.B), 256, 0, st>>>(n, i);
}

void launch_neuron(const Net &n, int i, int sm_count, cudaStream_t st) {
    const int per_block = kNeuronThreads * kNPT;
    // one group of kNeuronThreads * kNPT neurons per block (a grid capped at
    // the resident blocks, walking several groups per block, measured slower)
    (void)sm_count;
    const int blocks = (n.n_rec + per_block - 1) / per_block;
    if (n.surrogate || n.reset_mode || n.if_period || n.R_win)
        neuron_kernel<true><<<dim3(blocks, n.B), kNeuronThreads, 0, st>>>(n, i);
    else
        neuron_kernel<false><<<dim3(blocks, n.B), kNeuronThreads, 0, st>>>(n, i);
}

void launch_readout(const Net &n, int i, int sm_count, cudaStream_t st) {
    const int chunk = kReadoutChunk;
    int blocks = (n.n_src + chunk - 1) / chunk;
    const int cap = n.B > 1 ? 4 : 2 * sm_count;
    if (blocks > cap) blocks = cap;
    const int th = ((n.n_out + 31) / 32) * 32;     // >= n_out: one thread per readout
    readout_accum_kernel<<<dim3(blocks, n.B), th, 0, st>>>(n, i, chunk);
}

void launch_pred_input(const Net &n, int i, cudaStream_t st) { pred_input_kernel<<<n.B, 128, 0, st>>>(n, i); }

void launch_pred_apply(const Net &n, int i, cudaStream_t st) {
    pred_apply_kernel<<<n.B, ((n.n_out + 31) / 32) * 32, 0, st>>>(n, i);
}

void launch_deliver(const Net &n, int i, int grid_x, cudaStream_t st) {
    const dim3 grid(grid_x, n.B);
    if (n.has_state && !n.dense) {
        const size_t sm = deliver_stage_bytes(true) * 8 * kDStages;
        if (n.alif) deliver_kernel<true, true><<<grid, 256, sm, st>>>(n, i);
        else deliver_kernel<false, true><<<grid, 256, sm, st>>>(n, i);
    } else {
        const size_t sm = deliver_stage_bytes(false) * 8 * kDStages;
        deliver_kernel<false, false><<<grid, 256, sm, st>>>(n, i);
    }
}

int persistent_blocks(int sm_count) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_steps_kernel, kPersThreads, 0);
    return occ >= 1 ? sm_count : 0;          // one block per SM (all co-resident)
}

cudaError_t launch_persistent_steps(const Net &n, int T, GridBar *gb, int blocks, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kPersThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, persistent_steps_kernel, n, T, gb);
}

void prepare_step_kernel_attributes() {
    const int sm = (int)(deliver_stage_bytes(true) * 8 * kDStages);
    const int sm0 = (int)(deliver_stage_bytes(false) * 8 * kDStages);
    cudaFuncSetAttribute(deliver_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(deliver_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(deliver_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm0);
}

}  // namespace eprop
