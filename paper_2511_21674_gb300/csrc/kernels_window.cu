// Update-window kernels: learning-signal tables, event-driven synapse trace
// and gradient (the metric kernel), readout-weight gradient, window rollover.
//
// Closed form used by the synapse kernel.  Inside one update window
// (a0, b] the state of synapse j <- i, x = (zbar, eps_a, ebar), evolves as
// x^t = A^t x^{t-1} + s^t (1, 0, psi_j^t) with s^t the arrival indicator and
//   A^{t} = [[alpha, 0, 0],
//            [psi^{t-1}, rho - beta psi^{t-1}, 0],
//            [psi^t (alpha - beta psi^{t-1}), -beta psi^t (rho - beta psi^{t-1}), kappa_e]]
// (Eq. eligibility-vector-substituted, Eq. filtered-eligibility-trace), and the
// window's gradient is G = sum_t L^t ebar^t (Eq. final-gradient).  Everything
// is linear in x and in the arrivals and depends on the presynaptic side only
// through the arrival times, so for each postsynaptic neuron j one backward
// (adjoint) sweep over the window gives
//   Q(a)  = dG/d(arrival at a),  Pe(a), Pa(a) = d(ebar^b, eps_a^b)/d(arrival at a)
//   c     = dG/dx^{a0},          Phi = dx^b/dx^{a0}
// and an arrival costs one table lookup instead of a loop over the history.
// The paper's event-driven algorithm (Algorithm 5) instead loops over the
// archived psi/L history of the inter-spike interval; the sums are the same.
#include <type_traits>

#include "eprop_internal.cuh"
#include "eprop_launch.h"

namespace eprop {

__device__ __forceinline__ int run_step_w(const Net &n, int i) { return n.clock->r_base + i; }

__device__ __forceinline__ const uint32_t *src_words_c(const Net &n, int b, int src) {
    return n.bits + ((long long)b * n.n_src + src) * n.RW;
}

// Calls f(s) for every spike time s in [lo, hi] (hi - lo < ring span) in
// increasing order.
template <typename F>
__device__ __forceinline__ void for_each_spike(const uint32_t *words, int RW, int lo, int hi, F f) {
    const int mask = RW * 32 - 1;
    int r = lo < 1 ? 1 : lo;
    while (r <= hi) {
        const int p = r & mask;
        const int bit = p & 31;
        const int span = min(31 - bit, hi - r);        // bits bit..bit+span
        uint32_t m = words[p >> 5] >> bit;
        if (span < 31) m &= (2u << span) - 1u;
        while (m) {
            const int o = __ffs(m) - 1;
            f(r + o);
            m &= m - 1;
        }
        r += span + 1;
    }
}

// begin / end of a simulate call -------------------------------------------
__global__ void begin_call_kernel(Net n, int continuous) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (!continuous) n.clock->r_base = 0;
        *n.events = 0ULL;
    }
    for (int b = threadIdx.x; b < n.B; b += blockDim.x) n.loss_acc[b] = 0.0f;
}

__global__ void end_call_kernel(Net n, int T) {
    if (threadIdx.x == 0) {
        n.clock->t_abs_base += T;
        n.clock->r_base += T;
        n.clock->ring0 = (int)((n.clock->ring0 + (long long)T) % (n.D + 1));
    }
}

// filtered error for the readout gradient: Ebar(u) = sum_{t >= u} kappa^{t-u} E^t
// inside the window, and C = kappa * Ebar(a0 + 1) (Eq. eprop-output-new-subs-
// rewritten, index-flipped inside the window).
__global__ void filter_error_kernel(Net n) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n.B * n.n_out) return;
    const int b = idx / n.n_out, k = idx % n.n_out;
    const float *E = n.E_win + (long long)b * n.U * n.n_out + k;
    float *Eb = n.Ebar_win + (long long)b * n.U * n.n_out + k;
    // FP64 recursion with the FP64 filter constant (kappa + kappa_lo): over a
    // long window the FP32 chain of products would carry a relative error of
    // about (window length) x 2^-24 on errors that arrive late in the window
    const double kap = (double)n.kappa + (double)n.kappa_lo;
    double acc = 0.0;
    for (int u = n.U - 1; u >= 0; --u) {
        acc = (double)E[(long long)u * n.n_out] + kap * acc;
        Eb[(long long)u * n.n_out] = (float)acc;
    }
    n.Cwin[idx] = (float)(kap * acc);
}

// learning-signal tables: one thread per (sample, neuron), 128 neurons per
// block.  The window is swept backwards in chunks of steps: the chunk's
// learning signals L^t = sum_k B_jk E_k^t (Eq. final-gradient; formed for
// the whole window beforehand on the tensor cores, L_win) are
// loaded into registers, then the adjoint recursion writes the per-step
// tables and, at the window start, the window coefficients.
template <bool ALIF, bool REG, bool F64>
__global__ void __launch_bounds__(128, 4) tables_kernel(Net n, int i_end) {
    constexpr int kTC = ALIF ? 16 : 32;     // window steps per chunk
    const int b = blockIdx.y;
    const int U = n.U, N = n.n_rec;
    const int r_end = run_step_w(n, i_end);
    const int a0 = r_end - U;
    const int j = blockIdx.x * 128 + threadIdx.x;
    const bool act = j < N;
    const float *psi_g = n.psi_hist + (long long)b * (U + 1) * N + (act ? j : 0);
    const float *L_g = n.L_win + (long long)b * U * N + (act ? j : 0);    // [U][N], row u - 1 = step u
    // firing-rate regularisation (single-window calls only): a second
    // filtered copy of the eligibility trace, F_beta(e), weighted by the
    // signal R^t (Eq. ema-gradient); its adjoint mb joins me wherever the
    // eligibility e^t enters (e^t feeds both filters)
    const float *R_g = REG ? n.R_win + (long long)b * U * N + (act ? j : 0) : nullptr;
    // The adjoint sweep is the per-window reduction of the gradient.  For
    // ALIF the eligibility psi (zbar - beta eps_a) is a near-cancellation of
    // two long-memory traces, so the sweep runs in FP64 there (FP32 loses up
    // to 1e-1 relative on some elements over a few hundred steps); the LIF
    // sweep has no such cancellation and runs in FP32.
    // Long LIF windows (more than 128 steps) sweep in FP64 as well: the FP32
    // chain of decays carries a relative error of about (steps) x 2^-24 on
    // the contributions of early arrivals.
    using R = typename std::conditional<ALIF || F64, double, float>::type;
    const R alpha = (R)n.alpha + (R)n.alpha_lo;
    const R rho = ALIF ? (R)n.rho + (R)n.rho_lo : (R)0;
    const R beta = n.beta_a;
    // kappa_e^m over a window of hundreds of steps: in the FP64 sweep the
    // filter constant keeps its FP64 value (hi + lo), as alpha and rho do
    const R ke = (ALIF || F64) ? (R)n.kappa_e + (R)n.kappa_e_lo : (R)n.kappa_e;
    // adjoint of G (mz, ma, me); of ebar^b (ez, ea, ee); of eps_a^b (az, aa, ae)
    R mz = 0, ma = 0, me = 0;
    R ez = 0, ea = 0, ee = 1;
    R az = 0, aa = 1, ae = 0;
    R pn = 0;
    R mb = 0;                                  // adjoint of F_beta(e) (regularisation)
    const R breg = (R)n.beta_reg;
    const float psi_b = act ? psi_g[(long long)U * N] : 0.f;
    // generalized delays (one window per call): step u pairs with the
    // learning signal of u + d_out, which reaches the neuron only if it was
    // formed d_ls or more steps before the sample's end
    const int l_lim = (n.d_out | n.d_ls) ? min(U, n.lengths[b] - n.d_ls - a0) : U;
    const long long qbase = ((long long)b * U) * N + j;
    // Steps are taken backwards in chunks of kTC: the chunk's psi and
    // learning signals are loaded in one batch, then the recursion runs over
    // the chunk in registers.
    for (int u1 = U; u1 >= 1; u1 -= kTC) {
        const int u0 = max(1, u1 - kTC + 1);            // chunk = steps u0..u1
        float Lc[kTC], Pc[kTC + 1];
#pragma unroll
        for (int c = 0; c < kTC; ++c) {
            const int u = u1 - c;
            const bool in = act && u >= u0;
            const int ul = u + n.d_out;
            Lc[c] = (in && ul <= l_lim) ? L_g[(long long)(ul - 1) * N] : 0.f;
            Pc[c] = in ? psi_g[(long long)u * N] : 0.f;
        }
        float Rc[REG ? kTC : 1];
#pragma unroll
        for (int c = 0; c < (REG ? kTC : 1); ++c) {
            const int u = u1 - c;
            Rc[c] = (REG && act && u >= u0) ? R_g[(long long)(u - 1) * N] : 0.f;
        }
        Pc[kTC] = act ? psi_g[(long long)(u0 - 1) * N] : 0.f;   // psi of the step before the chunk
        if (!act) continue;
#pragma unroll
        for (int c = 0; c < kTC; ++c) {
            const int u = u1 - c;
            if (u < u0) break;
            const R p = Pc[c];                               // psi^{a0+u}
            if (u < U) {
                // x -> (A^{u+1})^T x with A^{u+1} from psi^u = p, psi^{u+1} = pn;
                // D = adjoint of e^{u+1} (both filters of the eligibility)
                const R D = REG ? me + mb : me;
                if (REG) mb = breg * mb;
                if (ALIF) {
                    const R g1 = alpha - beta * p, g2 = rho - beta * p;
                    R nz = alpha * mz + p * ma + pn * g1 * D;
                    R na = g2 * ma - beta * pn * g2 * D;
                    R ne = ke * me;
                    mz = nz; ma = na; me = ne;
                    nz = alpha * ez + p * ea + pn * g1 * ee;
                    na = g2 * ea - beta * pn * g2 * ee;
                    ne = ke * ee;
                    ez = nz; ea = na; ee = ne;
                    nz = alpha * az + p * aa + pn * g1 * ae;
                    na = g2 * aa - beta * pn * g2 * ae;
                    ne = ke * ae;
                    az = nz; aa = na; ae = ne;
                } else {
                    mz = alpha * mz + alpha * pn * D;
                    me = ke * me;
                    ez = alpha * ez + alpha * pn * ee;
                    ee = ke * ee;
                }
            }
            me += (R)Lc[c];
            if (REG) mb += (R)Rc[c];
            const R De = REG ? me + mb : me;           // adjoint of e^u
            if (ALIF) {
                reinterpret_cast<float4 *>(n.qp)[qbase + (long long)(u - 1) * N] =
                    make_float4((float)(mz + p * De), (float)(ez + p * ee), (float)(az + p * ae), 0.f);
            } else {
                reinterpret_cast<float2 *>(n.qp)[qbase + (long long)(u - 1) * N] =
                    make_float2((float)(mz + p * De), (float)(ez + p * ee));
            }
            pn = p;
        }
        if (u0 == 1) {
            // step a0 (u = 0): the window coefficients c = (A^{a0+1})^T mu^{a0+1}
            // (regularisation runs without carried state: no coefficients
            // of F_beta are kept, only G's adjoint sees it)
            const R p = Pc[kTC];
            const R D = REG ? me + mb : me;
            if (ALIF) {
                const R g1 = alpha - beta * p, g2 = rho - beta * p;
                R nz = alpha * mz + p * ma + pn * g1 * D;
                R na = g2 * ma - beta * pn * g2 * D;
                R ne = ke * me;
                mz = nz; ma = na; me = ne;
                nz = alpha * ez + p * ea + pn * g1 * ee;
                na = g2 * ea - beta * pn * g2 * ee;
                ne = ke * ee;
                ez = nz; ea = na; ee = ne;
                nz = alpha * az + p * aa + pn * g1 * ae;
                na = g2 * aa - beta * pn * g2 * ae;
                ne = ke * ae;
                az = nz; aa = na; ae = ne;
            } else {
                mz = alpha * mz + alpha * pn * D;
                me = ke * me;
                ez = alpha * ez + alpha * pn * ee;
                ee = ke * ee;
            }
        }
    }
    if (!act) return;
    // window coefficients: c = (mz, ma, me), Phi rows (ez, ea, .) and (az, aa, .);
    // one set per sample ([B][N][RC])
    if (n.has_state) {
        const int slot = (a0 / U) & (n.RC - 1);
        const long long cj = ((long long)b * N + j) * n.RC + slot;
        if (ALIF) {
            float4 *c = reinterpret_cast<float4 *>(n.coef) + cj * 2;
            c[0] = make_float4((float)mz, (float)ma, (float)me, (float)az);
            c[1] = make_float4((float)aa, (float)ez, (float)ea, 0.f);
        } else {
            reinterpret_cast<float4 *>(n.coef)[cj] = make_float4((float)mz, (float)me, (float)ez, 0.f);
        }
    }
    n.psi_hist[(long long)b * (U + 1) * N + j] = psi_b;     // slot 0 of the next window
}

// Work-item offsets of one window: for the emission steps s = s_lo..s_hi
// whose spikes arrive in the window, off[k] = sum_{k' < k} rows(s_lo + k').
__global__ void window_offsets_kernel(Net n, int i_end) {
    const int r_end = run_step_w(n, i_end);
    const int a0 = r_end - n.U;
    const int s_lo = max(a0 + 1 - n.D, 1);
    const int nsteps = r_end - 1 - s_lo + 1;
    const int lane = threadIdx.x & 31;
    long long acc = 0;
    for (int k = 0; k < nsteps; ++k) {
        int v = n.list_cnt[list_index(n, 0, (s_lo + k) % n.RS) + lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) n.win_off[k] = acc;
        acc += v;
    }
    if (lane == 0) n.win_off[nsteps > 0 ? nsteps : 0] = acc;
    // the row kernels' work counters (after the U + D + 2 offsets)
    if (lane < kWorkCounters) n.win_off[n.U + n.D + 2 + lane] = 0;
}

__device__ __forceinline__ bool any_spike(const uint32_t *words, int RW, int lo, int hi) {
    const int mask = RW * 32 - 1;
    int r = lo < 1 ? 1 : lo;
    while (r <= hi) {
        const int p = r & mask;
        const int bit = p & 31;
        const int span = min(31 - bit, hi - r);
        uint32_t m = words[p >> 5] >> bit;
        if (span < 31) m &= (2u << span) - 1u;
        if (m) return true;
        r += span + 1;
    }
    return false;
}


// Rare paths of the trace kernel kept out of line (instruction-cache
// footprint of the unrolled hot loop).
template <bool ALIF>
__device__ __noinline__ float catch_up(const Net n, int j, int k0, int kW, float zbar, float &epsa,
                                       float &ebar) {
    float G = 0.f;
    if (kW - k0 > n.RC - 1) {
        atomicOr(n.err_flags, 1u);
        k0 = kW - (n.RC - 1);
    }
    for (int k = k0; k <= kW; ++k) apply_window<ALIF>(n, j, k, zbar, epsa, ebar, G);
    return G;
}

template <bool ALIF>
__device__ __noinline__ void scan_arrivals(const Net n, const uint32_t *words, int lo, int hi, int d,
                                           long long qrow, float &G, float &ebar, float &epsa) {
    const int N = n.n_rec;
    const int mask = n.RW * 32 - 1;
    int r = lo;
    while (r <= hi) {
        const int p = r & mask;
        const int bit = p & 31;
        const int span = min(31 - bit, hi - r);
        uint32_t m = words[p >> 5] >> bit;
        if (span < 31) m &= (2u << span) - 1u;
        while (m) {
            const int a = r + __ffs(m) - 1 + d;
            m &= m - 1;
            if (ALIF) {
                const float4 t = reinterpret_cast<const float4 *>(n.qp)[qrow + (long long)a * N];
                G += t.x; ebar += t.y; epsa += t.z;
            } else {
                const float2 t = reinterpret_cast<const float2 *>(n.qp)[qrow + (long long)a * N];
                G += t.x; ebar += t.y;
            }
        }
        r += span + 1;
    }
}

// Event-driven synapse trace + gradient of one update window (the metric
// kernel).  Work items are (spiking row, segment of kSeg synapses) in
// ascending emission step; the item of a row's first spike among the
// window's emission steps advances every synapse of its segment over all of
// the row's arrivals in the window, in order, so each synapse is touched by
// exactly one warp per window.  A synapse's first arrival restores its state
// from the end of the window of its previous arrival (catch-up through the
// skipped windows' coefficients); every arrival a adds Q(a) to the window's
// gradient and Pe(a), Pa(a) to the state.  Record streams are read once
// (tgt_d evict-first); the table slabs of the steps in flight stay in L2.

// Bulk copies of one chunk of synapse records into a stage (one thread);
// see the delivery kernel for the alignment rule.
__device__ __forceinline__ void issue_chunk_w(const Net &n, StageBuf &sb, uint64_t *bar, long long q0, int cnt,
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

__device__ __forceinline__ float stage_trace_w(const Net &n, const StageBuf &sb, const StageDesc &d, long long q) {
    if (n.trace_bf16)
        return trace16_to_float(reinterpret_cast<const uint16_t *>(sb.tr)[q - d.q_al2], n.trace_type);
    return reinterpret_cast<const float *>(sb.tr)[q - d.q_al];
}

constexpr int kTStages = 3;

// shared-memory layout of the trace kernel (dynamic): per warp kTStages
// stage buffers, then the window's work-item offsets
template <bool ALIF, bool STATE>
__global__ void __launch_bounds__(256, 2) trace_window_kernel(Net n, int i_end) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ uint64_t bars[8][kTStages];
    __shared__ StageDesc desc[8][kTStages];
    __shared__ RowInfo info[8][kTStages][kMaxDelay + 1];
    __shared__ int spk[8][kTStages][kSpikeCap];
    __shared__ int nspk[8][kTStages];
    __shared__ int rspk[8][kSpikeCap];          // the producer's current row
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StageBuf *buf = reinterpret_cast<StageBuf *>(dsm) + warp * kTStages;
    long long *off = reinterpret_cast<long long *>(dsm + sizeof(StageBuf) * 8 * kTStages);
    const int U = n.U, N = n.n_rec;
    const int r_end = run_step_w(n, i_end);
    const int a0 = r_end - U;
    const int s_lo = max(a0 + 1 - n.D, 1);
    const int s_hi = r_end - 1;
    const int nsteps = s_hi - s_lo + 1;
    if (nsteps <= 0) return;
    for (int k = threadIdx.x; k <= nsteps; k += blockDim.x) off[k] = n.win_off[k];
    if (lane < kTStages) mbar_init(&bars[warp][lane], 1);
    fence_mbar_init();
    __syncthreads();
    const long long total = off[nsteps];
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    const int kW = a0 / U;
    const float step = n.lr * n.inv_B;
    const long long qa = (long long)(-a0 - 1) * N;     // table index = qa + a * N + j
    // producer cursor (warp-uniform): work item, current row and its range;
    // items are handed out in order by a counter, so the warps in flight
    // stay within about one emission step (their table slabs stay in L2)
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(n.win_off + n.U + n.D + 2);
    long long pit = 0;
    long long pq = 0, pre = 0;
    int psrc = -1, ps = 0, pns = 0;
    RowInfo rinfo;
    unsigned vmask = 0;
    (void)gw;
    (void)nw;
    // advances the producer to the next chunk; false when the window is done
    auto next_row = [&]() -> bool {
        while (pq >= pre) {
            {
                long long v = 0;
                if (lane == 0) v = (long long)atomicAdd(ctr, 1ULL);
                pit = __shfl_sync(0xffffffffu, v, 0);
            }
            if (pit >= total) return false;
            int lo = 0, hi = nsteps;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (off[mid] <= pit) lo = mid; else hi = mid;
            }
            const int s = s_lo + lo;
            const long long li = list_index(n, 0, s % n.RS);
            const BucketScan bs = bucket_scan(n.list_cnt + li);
            const int src = bucket_entry(n, n.list_ids + li * n.list_cap, bs, (int)(pit - off[lo]));
            const long long rb = n.row_ptr[src], re = n.row_ptr[src + 1];
            if (re <= rb) continue;
            const uint32_t *words = src_words_c(n, 0, src);
            if (any_spike(words, n.RW, s_lo, s - 1)) continue;   // another item owns the row
            int ns = 0;
            if (lane == 0) {             // the row's spikes in [s, s_hi], ascending
                const int mask = n.RW * 32 - 1;
                int r = s;
                while (r <= s_hi) {
                    const int p = r & mask;
                    const int bit = p & 31;
                    const int span = min(31 - bit, s_hi - r);
                    uint32_t m = words[p >> 5] >> bit;
                    if (span < 31) m &= (2u << span) - 1u;
                    while (m) {
                        if (ns < kSpikeCap) rspk[warp][ns] = r + __ffs(m) - 1;
                        ++ns;
                        m &= m - 1;
                    }
                    r += span + 1;
                }
            }
            pns = __shfl_sync(0xffffffffu, ns, 0);
            if (STATE && lane >= 1 && lane <= n.D)
                rinfo = row_info(n, words, n.anchor_t[src], n.anchor_z[src], a0, lane, false);
            psrc = src;
            ps = s;
            pq = rb;
            pre = re;
        }
        return true;
    };
    auto produce = [&](int k) {
        const int cnt = (int)min((long long)kChunk, pre - pq);
        if (STATE && lane >= 1 && lane <= n.D) info[warp][k][lane] = rinfo;
        for (int c = lane; c < min(pns, kSpikeCap); c += 32) spk[warp][k][c] = rspk[warp][c];
        if (lane == 0) nspk[warp][k] = pns;
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async();
            issue_chunk_w(n, buf[k], &bars[warp][k], pq, cnt, STATE, desc[warp][k]);
            desc[warp][k].src = psrc;
            desc[warp][k].row = ps;
        }
        pq += cnt;
    };
    for (int k = 0; k < kTStages; ++k) {
        if (!next_row()) break;
        produce(k);
        vmask |= 1u << k;
    }
    __syncwarp();
    int abort_c = -1;
    for (int c = 0;; ++c) {
        const int k = c % kTStages;
        if (!((vmask >> k) & 1u)) break;
        if (!mbar_wait(&bars[warp][k], (uint32_t)((c / kTStages) & 1), n.err_flags)) {
            abort_c = c;
            break;
        }
        const StageDesc d = desc[warp][k];
        const StageBuf &sb = buf[k];
        const int ns = nspk[warp][k];
        const bool listed = ns <= kSpikeCap;
        const int s = d.row;
        const uint32_t *words = src_words_c(n, 0, d.src);
        const int *sp = spk[warp][k];
#pragma unroll 1
        for (int h = 0; h < kChunk / 32; h += 4) {
            uint32_t td[4];
            float wv[4], eb[4], ep[4];
            float4 t0[4];
            Coef cf0[4], cf1[4];
            int c0[4], k0s[4];
            // phase 1: which synapses have arrivals; issue every load they need
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = lane + 32 * (h + u);
                const long long q = d.q0 + idx;
                td[u] = idx < d.n ? sb.td[q - d.q_al] : 0u;
                const int dl = (int)(td[u] >> 24);
                const long long j = td[u] & 0xFFFFFFu;
                bool has = false;
                int cc = 0;
                if (td[u] != 0u) {
                    if (listed) {       // first listed spike whose arrival lies after a0
                        while (cc < ns && sp[cc] + dl <= a0) ++cc;
                        has = cc < ns && sp[cc] + dl <= r_end;
                    } else {
                        has = any_spike(words, n.RW, max(s, a0 + 1 - dl), r_end - dl);
                    }
                }
                c0[u] = has ? cc : -1;
                k0s[u] = -1;
                wv[u] = has ? sb.w[q - d.q_al] : 0.f;
                eb[u] = (STATE && has) ? stage_trace_w(n, sb, d, q) : 0.f;
                ep[u] = (STATE && ALIF && has) ? load_trace(n.epsa, q, n.trace_type) : 0.f;
                t0[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (has && listed) {
                    const long long qi = qa + (long long)(sp[cc] + dl) * N + j;
                    if (ALIF) t0[u] = __ldg(reinterpret_cast<const float4 *>(n.qp) + qi);
                    else {
                        const float2 t = __ldg(reinterpret_cast<const float2 *>(n.qp) + qi);
                        t0[u] = make_float4(t.x, t.y, 0.f, 0.f);
                    }
                }
                if (STATE && has) {
                    const RowInfo ri = info[warp][k][dl];
                    if (ri.b_prev != kNoSpike) {
                        int k0 = ri.k_prev;
                        if (kW - k0 > n.RC - 1) {
                            atomicOr(n.err_flags, 1u);
                            k0 = kW - (n.RC - 1);
                        }
                        k0s[u] = k0;
                        cf0[u] = load_coef<ALIF>(n, j, k0);
                        if (k0 + 1 <= kW) cf1[u] = load_coef<ALIF>(n, j, k0 + 1);
                    }
                }
            }
            // phase 2: closed-form advance and weight update
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (c0[u] < 0) continue;
                const long long q = d.q0 + lane + 32 * (h + u);
                const long long j = td[u] & 0xFFFFFFu;
                const int dl = (int)(td[u] >> 24);
                float G = 0.f, ebar = eb[u], epsa = ep[u];
                if (STATE) {            // the window's first arrival: restore the state
                    const int k0 = k0s[u];
                    if (k0 >= 0) {
                        float zbar = info[warp][k][dl].zbar_bp;
                        apply_coef<ALIF>(n, cf0[u], zbar, epsa, ebar, G);
                        if (k0 + 1 <= kW) apply_coef<ALIF>(n, cf1[u], zbar, epsa, ebar, G);
                        for (int kk = k0 + 2; kk <= kW; ++kk) apply_window<ALIF>(n, j, kk, zbar, epsa, ebar, G);
                    } else {
                        ebar = 0.f;
                        epsa = 0.f;
                    }
                }
                if (listed) {
                    G += t0[u].x;
                    ebar += t0[u].y;
                    if (ALIF) epsa += t0[u].z;
                    for (int cc = c0[u] + 1; cc < ns; ++cc) {
                        const int a = sp[cc] + dl;
                        if (a > r_end) break;
                        if (ALIF) {
                            const float4 t = __ldg(reinterpret_cast<const float4 *>(n.qp) + qa + (long long)a * N + j);
                            G += t.x; ebar += t.y; epsa += t.z;
                        } else {
                            const float2 t = __ldg(reinterpret_cast<const float2 *>(n.qp) + qa + (long long)a * N + j);
                            G += t.x; ebar += t.y;
                        }
                    }
                } else {            // rows with more spikes than the cache holds
                    scan_arrivals<ALIF>(n, words, max(s, a0 + 1 - dl), r_end - dl, dl, qa + j, G, ebar, epsa);
                }
                {
                    const float wn = window_update(n, q, wv[u], G);
                    if (!n.adam) __stcs(n.w + q, wn);
                }
                if (STATE) {
                    store_trace(n.ebar, q, ebar, n.trace_type);
                    if (ALIF) store_trace(n.epsa, q, epsa, n.trace_type);
                }
                if (n.record_grad) n.grad[q] = grad_add(n.grad[q], n.inv_B, G);
            }
        }
        __syncwarp();
        vmask &= ~(1u << k);
        if (next_row()) {
            produce(k);
            vmask |= 1u << k;
        }
        __syncwarp();
    }
    if (abort_c >= 0) {                      // let copies in flight land first
        for (int c = abort_c + 1; c < abort_c + kTStages; ++c)
            if ((vmask >> (c % kTStages)) & 1u)
                mbar_wait(&bars[warp][c % kTStages], (uint32_t)((c / kTStages) & 1), n.err_flags);
    }
}

// Dense form of the window update.  Every synapse is advanced to the end
// of every window, so the stored weight and traces are always those of the
// window start and spike delivery reads the weight as it is (no catch-up).
// The state x = (zbar, eps_a, ebar) at a0 passes through the window's
// coefficients (G += c . x, x <- Phi x); each arrival a in the window adds
// Q(a) to G and Pe(a), Pa(a) to the traces (event-driven weight update from
// the archived postsynaptic history, Sec. "From time-driven to event-driven
// e-prop"; the per-window tables stand for that history).  Two launches:
//   kPassFirst: rows with a spike whose arrival can fall in the window,
//     taken from the per-step spike lists in ascending emission step (the
//     row belongs to its first such spike), so the table slabs in use stay
//     in L2: the coefficient step and every arrival of the window (the
//     first one's table entry loaded with the rest of the synapse batch);
//   kPassIdle: all other rows, in index order (coefficient step only).
// Warps take work items in batches (one atomic per batch; the lanes resolve
// and filter the items in parallel) and advance the accepted rows in item
// order: 32 rows per batch in the idle launch, one spike-list item per
// batch in the spiking-row launch, whose warps in flight must stay within
// about one emission step (larger batches spread them over many steps,
// whose table slabs then no longer fit in L2: measured slower).  Per warp
// a kPStages-deep pipeline of bulk copies brings the (j|d, w, ebar) streams
// of the next chunks into shared memory while the current chunk is
// advanced; what stays on the critical path are the targets' window
// coefficients and the table entries (L2).
// two stages per warp: enough copies in flight for the streams, and the
// smaller shared-memory carve-out leaves more L1 for the coefficient and
// table lookups (measured faster than three or four stages)
constexpr int kPStages = 2;
constexpr int kPassIdle = 0, kPassFirst = 1;

// table entry (Q, Pe, Pa) of one arrival (Pa = 0 for LIF)
template <bool ALIF>
__device__ __forceinline__ float4 load_table(const Net &n, long long qi) {
    if (ALIF) return __ldg(reinterpret_cast<const float4 *>(n.qp) + qi);
    const float2 t = __ldg(reinterpret_cast<const float2 *>(n.qp) + qi);
    return make_float4(t.x, t.y, 0.f, 0.f);
}

// The idle-row launch fits three blocks per SM (more warps for its
// coefficient gathers); the spiking-row launch keeps two (it needs the
// registers of its table lookups).
// TB: trace storage (0 FP32, 1 BF16, 2 FP16); GEN: the general weight update
// (Adam or fixed signs), else plain gradient descent in place.
template <bool ALIF, int MODE, int TB, bool GEN>
__global__ void __launch_bounds__(256, MODE == kPassIdle ? 3 : 2) window_pass_kernel(Net n, int i_end) {
    constexpr bool LISTS = MODE != kPassIdle;        // work items from the spike lists
    constexpr int kBatch = LISTS ? 1 : 32;           // work items per fetch
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ uint64_t bars[8][kPStages];
    __shared__ StageDesc desc[8][kPStages];
    __shared__ float zbs[8][kPStages][kMaxDelay + 1];
    __shared__ int spk[8][LISTS ? kPStages : 1][kSpikeCap];
    __shared__ int nspk[8][kPStages];
    __shared__ int rspk[8][kSpikeCap];          // the producer's current row
    // per stage and delay d: step of the first arrival of the row's delay-d
    // synapses in the window (-1: none) and its index in the spike list
    __shared__ int2 arr[8][LISTS ? kPStages : 1][kMaxDelay + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StageBuf *buf = reinterpret_cast<StageBuf *>(dsm) + warp * kPStages;
    long long *off = reinterpret_cast<long long *>(dsm + sizeof(StageBuf) * 8 * kPStages);
    const int U = n.U, N = n.n_rec;
    const int r_end = run_step_w(n, i_end);
    const int a0 = r_end - U;
    const int s_lo = max(a0 + 1 - n.D, 1);
    const int s_hi = r_end - 1;
    const int nsteps = s_hi - s_lo + 1;
    if (LISTS && nsteps <= 0) return;
    if (LISTS)
        for (int k = threadIdx.x; k <= nsteps; k += blockDim.x) off[k] = n.win_off[k];
    if (lane < kPStages) mbar_init(&bars[warp][lane], 1);
    fence_mbar_init();
    __syncthreads();
    const long long total = LISTS ? off[nsteps] : (long long)n.n_src;
    const float step = n.lr * n.inv_B;
    const long long qa = (long long)(-a0 - 1) * N;     // table index = qa + a * N + j
    // work items are handed out in order by a counter, so the warps in
    // flight stay within about one emission step (their table slabs stay
    // in L2)
    unsigned long long *ctr =
        reinterpret_cast<unsigned long long *>(n.win_off + n.U + n.D + 2) + (MODE == kPassFirst ? 0 : 1);
    // candidates of the current batch: lane l < kBatch holds item base + l
    // (its row, emission step and synapse range); amask = accepted rows not
    // yet taken
    int csrc = 0, cstep = s_lo;
    long long crb = 0, cre = 0;
    unsigned amask = 0;
    bool drained = false;
    // producer cursor (warp-uniform): current row and its remaining range
    long long pq = 0, pre = 0;
    int psrc = -1, ps = s_lo, pns = 0;
    float pzb = 0.f;            // lane d: zbar at a0 of the row's delay-d synapses
    unsigned vmask = 0;
    // the next batch's counter value is fetched one row ahead (lane 0), so
    // the atomic's round trip overlaps the current row's chunks
    long long pf_base = -1;
    auto prefetch = [&]() {
        if (lane == 0 && pf_base < 0 && !drained) pf_base = (long long)atomicAdd(ctr, (unsigned long long)kBatch);
    };
    auto refill = [&]() -> bool {
        long long base = 0;
        if (lane == 0) {
            base = pf_base >= 0 ? pf_base : (long long)atomicAdd(ctr, (unsigned long long)kBatch);
            pf_base = -1;
        }
        base = __shfl_sync(kFull, base, 0);
        if (base >= total) {
            drained = true;
            return false;
        }
        const long long it = base + lane;
        const bool valid = lane < kBatch && it < total;
        int src = 0, s = s_lo;
        if (LISTS) {
            int lo = 0;
            if (valid) {
                int hi = nsteps;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (off[mid] <= it) lo = mid; else hi = mid;
                }
            }
            s = s_lo + lo;
            // list entries, one emission step at a time (a batch spans few)
            const int s_first = __shfl_sync(kFull, s, 0);
            const int s_last = __reduce_max_sync(kFull, valid ? s : s_first);
            for (int ss = s_first; ss <= s_last; ++ss) {
                const long long li = list_index(n, 0, ss % n.RS);
                const BucketScan bs = bucket_scan(n.list_cnt + li);
                const long long r = it - off[ss - s_lo];      // entry index (lanes of step ss)
                int bk = 0;                                   // buckets with incl <= r
#pragma unroll
                for (int w = 16; w > 0; w >>= 1)
                    if ((long long)__shfl_sync(kFull, bs.incl, bk + w - 1) <= r) bk += w;
                const int prev = __shfl_sync(kFull, bs.incl, bk > 0 ? bk - 1 : 0);
                if (valid && s == ss)
                    src = n.list_ids[(li + bk) * n.list_cap + (r - (bk > 0 ? prev : 0))];
            }
        } else {
            src = valid ? (int)it : 0;
        }
        bool ok = false;
        long long rb = 0, re = 0;
        if (valid) {
            rb = n.row_ptr[src];
            re = n.row_ptr[src + 1];
            if (re > rb) {
                const uint32_t *words = src_words_c(n, 0, src);
                if (MODE == kPassIdle)        // rows of the list launch excluded
                    ok = !(nsteps > 0 && any_spike(words, n.RW, s_lo, s_hi));
                else                          // the row's first spike of the window
                    ok = !any_spike(words, n.RW, s_lo, s - 1);
            }
        }
        csrc = src;
        cstep = s;
        crb = rb;
        cre = re;
        amask = __ballot_sync(kFull, ok);
        return true;
    };
    auto next_row = [&]() -> bool {
        if (pq < pre) return true;
        while (amask == 0)
            if (drained || !refill()) return false;
        const int l = __ffs(amask) - 1;
        amask &= amask - 1;
        const int src = __shfl_sync(kFull, csrc, l);
        const int s = __shfl_sync(kFull, cstep, l);
        const long long rb = __shfl_sync(kFull, crb, l), re = __shfl_sync(kFull, cre, l);
        const uint32_t *words = src_words_c(n, 0, src);
        if (LISTS) {
            int ns = 0;
            if (lane == 0) {         // the row's spikes of the window, ascending
                const int mask = n.RW * 32 - 1;
                int r = s;
                while (r <= s_hi) {
                    const int p = r & mask;
                    const int bit = p & 31;
                    const int span = min(31 - bit, s_hi - r);
                    uint32_t m = words[p >> 5] >> bit;
                    if (span < 31) m &= (2u << span) - 1u;
                    while (m) {
                        if (ns < kSpikeCap) rspk[warp][ns] = r + __ffs(m) - 1;
                        ++ns;
                        m &= m - 1;
                    }
                    r += span + 1;
                }
            }
            __syncwarp();
            pns = __shfl_sync(kFull, ns, 0);
        }
        pzb = (lane >= 1 && lane <= n.D)
                  ? row_info(n, words, n.anchor_t[src], n.anchor_z[src], a0, lane, false).zbar_a0
                  : 0.f;
        psrc = src;
        ps = s;
        pq = rb;
        pre = re;
        if (amask == 0) prefetch();        // this batch is used up: fetch the next one
        return true;
    };
    auto produce = [&](int k) {
        const int cnt = (int)min((long long)kChunk, pre - pq);
        if (lane <= n.D) zbs[warp][k][lane] = pzb;
        if (LISTS) {
            for (int c = lane; c < min(pns, kSpikeCap); c += 32) spk[warp][k][c] = rspk[warp][c];
            if (lane == 0) nspk[warp][k] = pns;
            if (lane >= 1 && lane <= n.D) {
                const int nsc = min(pns, kSpikeCap);
                int cc = 0;
                while (cc < nsc && rspk[warp][cc] + lane <= a0) ++cc;
                const int a1 = (cc < nsc && rspk[warp][cc] + lane <= r_end) ? rspk[warp][cc] + lane : -1;
                arr[warp][LISTS ? k : 0][lane] = make_int2(a1, cc);
            }
        }
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async();
            issue_chunk_w(n, buf[k], &bars[warp][k], pq, cnt, true, desc[warp][k]);
            desc[warp][k].src = psrc;
            desc[warp][k].row = ps;
        }
        pq += cnt;
    };
    for (int k = 0; k < kPStages; ++k) {
        if (!next_row()) break;
        produce(k);
        vmask |= 1u << k;
    }
    __syncwarp();
    int abort_c = -1;
    for (int c = 0;; ++c) {
        const int k = c % kPStages;
        if (!((vmask >> k) & 1u)) break;
        if (!mbar_wait(&bars[warp][k], (uint32_t)((c / kPStages) & 1), n.err_flags)) {
            abort_c = c;
            break;
        }
        const StageDesc d = desc[warp][k];
        const StageBuf &sb = buf[k];
        const int ns = LISTS ? nspk[warp][k] : 0;
        const bool listed = ns <= kSpikeCap;
        const int *sp = spk[warp][LISTS ? k : 0];
        const float *zrow = zbs[warp][k];
        // chunk-relative addressing: shared offsets and global bases of the chunk
        const int o4 = (int)(d.q0 - d.q_al), o2 = (int)(d.q0 - d.q_al2);
        float *wq = n.w + d.q0;
        float *gq = n.grad + d.q0;
        constexpr int kB = 4;                  // synapses per lane in flight
#pragma unroll 1
        for (int h = 0; h < kChunk / 32; h += kB) {
            uint32_t td[kB];
            float wv[kB], zr[kB], eb[kB], ep[kB];
            Coef cf[kB];
            float4 t0[kB];                     // table entry of the first arrival
            int c0[kB];                        // its index in the row's spike list (-1: none)
            bool live[kB];
            // phase 1: every load the synapses need is issued before any is used
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int idx = lane + 32 * (h + u);
                const bool in = idx < d.n;
                td[u] = in ? sb.td[o4 + idx] : 0u;
                const int dl = (int)(td[u] >> 24);
                wv[u] = in ? sb.w[o4 + idx] : 0.f;
                if (TB) eb[u] = in ? trace16_to_float(reinterpret_cast<const uint16_t *>(sb.tr)[o2 + idx], TB)
                                   : 0.f;
                else eb[u] = in ? reinterpret_cast<const float *>(sb.tr)[o4 + idx] : 0.f;
                c0[u] = -1;
                t0[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                int a1 = -1;
                if (LISTS && listed && in) {               // first arrival in the window
                    const int2 ar = arr[warp][LISTS ? k : 0][dl];
                    a1 = ar.x;
                    c0[u] = a1 >= 0 ? ar.y : -1;
                }
                zr[u] = zrow[dl];
                ep[u] = (ALIF && in) ? load_trace(n.epsa, d.q0 + idx, TB) : 0.f;
                live[u] = in && (LISTS || zr[u] != 0.f || eb[u] != 0.f || ep[u] != 0.f);
                if (live[u]) cf[u] = load_coef_dense<ALIF>(n, td[u] & 0xFFFFFFu);
                if (c0[u] >= 0) t0[u] = load_table<ALIF>(n, qa + (long long)a1 * N + (td[u] & 0xFFFFFFu));
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                if (!live[u]) continue;
                const int idx = lane + 32 * (h + u);
                const int j = (int)(td[u] & 0xFFFFFFu);
                const int dl = (int)(td[u] >> 24);
                float G = 0.f, zbar = zr[u], ebar = eb[u], epsa = ep[u];
                apply_coef<ALIF>(n, cf[u], zbar, epsa, ebar, G);
                if (LISTS) {
                    if (listed) {
                        if (c0[u] >= 0) {
                            G += t0[u].x;
                            ebar += t0[u].y;
                            if (ALIF) epsa += t0[u].z;
                        }
                        // further arrivals (rows with more than one spike)
                        for (int cc = (c0[u] >= 0 ? c0[u] + 1 : ns); cc < ns; ++cc) {
                            const int a = sp[cc] + dl;
                            if (a > r_end) break;
                            const float4 t = load_table<ALIF>(n, qa + (long long)a * N + j);
                            G += t.x;
                            ebar += t.y;
                            if (ALIF) epsa += t.z;
                        }
                    } else {
                        // rows with more spikes than the cache holds
                        scan_arrivals<ALIF>(n, src_words_c(n, 0, d.src), max(d.row, a0 + 1 - dl), r_end - dl, dl,
                                            qa + j, G, ebar, epsa);
                    }
                }
                if (G != 0.f) {
                    if (GEN) {
                        const float wn = window_update(n, d.q0 + idx, wv[u], G);
                        if (!n.adam) __stcs(wq + idx, wn);
                    } else {
                        __stcs(wq + idx, sgd_step(wv[u], step, G));
                    }
                }
                if (TB) __stcs(reinterpret_cast<uint16_t *>(n.ebar) + d.q0 + idx, float_to_trace16(ebar, TB));
                else __stcs(reinterpret_cast<float *>(n.ebar) + d.q0 + idx, ebar);
                if (ALIF) store_trace(n.epsa, d.q0 + idx, epsa, TB);
                if (n.record_grad) gq[idx] = grad_add(gq[idx], n.inv_B, G);
            }
        }
        __syncwarp();
        vmask &= ~(1u << k);
        if (next_row()) {
            produce(k);
            vmask |= 1u << k;
        }
        __syncwarp();
    }
    if (abort_c >= 0) {                      // let copies in flight land first
        for (int c = abort_c + 1; c < abort_c + kPStages; ++c)
            if ((vmask >> (c % kPStages)) & 1u)
                mbar_wait(&bars[warp][c % kPStages], (uint32_t)((c / kPStages) & 1), n.err_flags);
    }
}

// event-driven synapse gradient, batched single-window form (no carried
// state: each arrival contributes Q(a) independently).  One warp per source
// row; the row's spikes of every sample are gathered into shared memory and
// every synapse sums the table entries of its arrivals over all samples.
template <int QP_STRIDE>
__global__ void __launch_bounds__(256) trace_batched_kernel(Net n) {
    constexpr int CAP = 512;
    __shared__ int sp[8][CAP];      // (sample << 20) | step
    __shared__ int ncount[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int U = n.U, N = n.n_rec, T = n.T;
    for (int src = gw; src < n.n_src; src += nw) {
        const long long q0 = n.row_ptr[src], q1 = n.row_ptr[src + 1];
        if (q1 == q0) continue;
        // gather (sample, step) pairs; lanes split the samples
        if (lane == 0) ncount[warp] = 0;
        __syncwarp();
        for (int b = lane; b < n.B; b += 32) {
            const uint32_t *words = src_words_c(n, b, src);
            for_each_spike(words, n.RW, 1, T, [&](int st) {
                const int pos = atomicAdd(&ncount[warp], 1);
                if (pos < CAP) sp[warp][pos] = (b << 20) | st;
            });
        }
        __syncwarp();
        const int ns = ncount[warp];
        if (ns == 0) continue;
        for (long long q = q0 + lane; q < q1; q += 32) {
            const uint32_t td = n.tgt_d[q];
            const int j = (int)(td & 0xFFFFFFu);
            const int d = (int)(td >> 24);
            // the batch's sum of arrival terms (up to samples x arrivals of
            // them) is reduced in FP64
            double G = 0.0;
            if (ns <= CAP) {
                for (int c = 0; c < ns; ++c) {
                    const int v = sp[warp][c];
                    const int b = v >> 20, a = (v & 0xFFFFF) + d;
                    if (a <= T) G += (double)n.qp[(((long long)b * U + (a - 1)) * N + j) * QP_STRIDE];
                }
            } else {
                for (int b = 0; b < n.B; ++b) {
                    const uint32_t *words = src_words_c(n, b, src);
                    for_each_spike(words, n.RW, 1, T - d, [&](int st) {
                        G += (double)n.qp[(((long long)b * U + (st + d - 1)) * N + j) * QP_STRIDE];
                    });
                }
            }
            {
                const float w0 = n.w[q];
                const float wn = window_update(n, q, w0, (float)G);
                if (!n.adam) n.w[q] = wn;
            }
            if (n.record_grad) n.grad[q] += n.inv_B * (float)G;
        }
        __syncwarp();
    }
}

// Dense window update of a mini-batch (batch > 1 with update windows inside
// a call; Eq. accumulated-gradients, Eq. gradient-descent).  Every synapse
// carries one state per sample (ebar, eps_a of sample b at b * nnz + q).
// At a window end each sample's state passes through that sample's window
// coefficients and arrival tables -- the arithmetic of the single-sample
// window pass -- and the weight takes one step with the sum over samples
// (the batch mean).  One warp per source row: the lanes first form each
// (sample, delay)'s presynaptic trace at the window start and gather the
// row's spikes of the window per sample (grouped by sample, ascending),
// then walk the row's synapses.
template <bool ALIF, int TB, bool GEN>
__global__ void __launch_bounds__(256) window_batched_kernel(Net n, int i_end) {
    constexpr int kCap = 256;                    // spikes of one row (all samples) cached per warp
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ float zb[8][kBatchWindowMax][kMaxDelay + 1];
    __shared__ int sp[8][kCap];
    __shared__ int soff[8][kBatchWindowMax + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp, nw = gridDim.x * (blockDim.x >> 5);
    const int U = n.U, N = n.n_rec, B = n.B, D = n.D;
    const int r_end = run_step_w(n, i_end);
    const int a0 = r_end - U;
    const int s_lo = max(a0 + 1 - D, 1), s_hi = r_end - 1;
    const float step = n.lr * n.inv_B;
    const long long nnz = n.nnz;
    const long long cstride = (long long)N * n.RC;
    for (int src = gw; src < n.n_src; src += nw) {
        const long long q0 = n.row_ptr[src], q1 = n.row_ptr[src + 1];
        if (q1 == q0) continue;
        for (int e = lane; e < B * D; e += 32) {
            const int b = e / D, d = e % D + 1;
            const long long sb = (long long)b * n.n_src + src;
            zb[warp][b][d] = row_info(n, src_words_c(n, b, src), n.anchor_t[sb], n.anchor_z[sb], a0, d, false).zbar_a0;
        }
        // lane l owns samples l and l + 32: counts, then offsets in sample order
        int cnt[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int b = lane + 32 * h;
            if (b < B && s_lo <= s_hi) for_each_spike(src_words_c(n, b, src), n.RW, s_lo, s_hi, [&](int) { ++cnt[h]; });
        }
        int base = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int v = cnt[h];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, v, o);
                if (lane >= o) v += t;
            }
            const int b = lane + 32 * h;
            if (b < B) soff[warp][b] = base + v - cnt[h];
            base += __shfl_sync(kFull, v, 31);
        }
        if (lane == 0) soff[warp][B] = base;
        __syncwarp();
        const int total = base;
        if (total <= kCap) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = lane + 32 * h;
                if (b < B && s_lo <= s_hi) {
                    int pos = soff[warp][b];
                    for_each_spike(src_words_c(n, b, src), n.RW, s_lo, s_hi, [&](int st) { sp[warp][pos++] = st; });
                }
            }
        }
        __syncwarp();
        for (long long q = q0 + lane; q < q1; q += 32) {
            const uint32_t td = n.tgt_d[q];
            const int j = (int)(td & 0xFFFFFFu);
            const int dl = (int)(td >> 24);
            // the sum over samples is reduced in FP64
            double Gt = 0.0;
            for (int b = 0; b < B; ++b) {
                const long long qb = (long long)b * nnz + q;
                float ebar = load_trace(n.ebar, qb, TB);
                float epsa = ALIF ? load_trace(n.epsa, qb, TB) : 0.f;
                float zbar = zb[warp][b][dl];
                Coef cf;
                if (ALIF) {
                    const float4 *p = reinterpret_cast<const float4 *>(n.coef) + ((long long)b * cstride + j) * 2;
                    cf.c0 = __ldg(p);
                    cf.c1 = __ldg(p + 1);
                } else {
                    cf.c0 = __ldg(reinterpret_cast<const float4 *>(n.coef) + (long long)b * cstride + j);
                    cf.c1 = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                float G = 0.f;
                apply_coef<ALIF>(n, cf, zbar, epsa, ebar, G);
                const long long qa = ((long long)b * U - a0 - 1) * N;   // table index qa + a * N + j
                if (total <= kCap) {
                    for (int c = soff[warp][b]; c < soff[warp][b + 1]; ++c) {
                        const int a = sp[warp][c] + dl;
                        if (a <= a0) continue;
                        if (a > r_end) break;
                        if (ALIF) {
                            const float4 t = __ldg(reinterpret_cast<const float4 *>(n.qp) + qa + (long long)a * N + j);
                            G += t.x; ebar += t.y; epsa += t.z;
                        } else {
                            const float2 t = __ldg(reinterpret_cast<const float2 *>(n.qp) + qa + (long long)a * N + j);
                            G += t.x; ebar += t.y;
                        }
                    }
                } else {            // rows with more spikes than the cache holds
                    scan_arrivals<ALIF>(n, src_words_c(n, b, src), max(a0 + 1 - dl, 1), r_end - dl, dl, qa + j, G,
                                        ebar, epsa);
                }
                store_trace(n.ebar, qb, ebar, TB);
                if (ALIF) store_trace(n.epsa, qb, epsa, TB);
                Gt += (double)G;
            }
            const float Gf = (float)Gt;
            if (Gf != 0.f) {
                const float w = n.w[q];
                if (GEN) {
                    const float wn = window_update(n, q, w, Gf);
                    if (!n.adam) n.w[q] = wn;
                } else {
                    n.w[q] = sgd_step(w, step, Gf);
                }
            }
            if (n.record_grad) n.grad[q] = grad_add(n.grad[q], n.inv_B, Gf);
        }
        __syncwarp();
    }
}

// readout weights: g_kj = sum_b [zk_j^{a0} C_k + sum_{spikes s in window} Ebar_k(s)]
// (Eq. eprop-output-new-subs-rewritten), one thread per (j, k).
__global__ void readout_weights_kernel(Net n, int i_end) {
    // one warp per recurrent neuron j, lanes over the readouts k (coalesced
    // rows of W_out); the neuron's spikes in the window are scanned once per
    // group of 32 readouts
    const int lane = threadIdx.x & 31;
    const long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int K = n.n_out, N = n.n_rec, U = n.U;
    if (j >= N) return;
    const int r_end = run_step_w(n, i_end);
    const int a0 = r_end - U;
    const int par = (a0 / U) & 1;
    const float *zk_cur = n.zk + (long long)par * n.B * N;
    float *zk_nxt = n.zk + (long long)(par ^ 1) * n.B * N;
    const float kU = exp2f(n.log2_kappa * (float)U);
    const uint8_t *mrow = n.out_mask + j * K;          // per-weight readout mask
    if ((K & 3) == 0) {
        // four readouts per lane (float4 rows; K % 4 == 0 keeps every row
        // 16-byte aligned).  The weight row is requested first and the
        // window's spike words one per lane, so the neuron's memory round
        // trips overlap instead of following one another.
        const int mask = n.RW * 32 - 1;
        const int base = (a0 + 1) & ~31;                 // step of the first word's bit 0
        const int nwd = (r_end - base) / 32 + 1;         // words covering a0+1 .. r_end
        const float s = n.lr * n.inv_B;
        for (int k0 = 0; k0 < K; k0 += 128) {
            const int k = k0 + 4 * lane;
            const bool has_k = k < K;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f), gg = w;
            float4 *wp = reinterpret_cast<float4 *>(n.w_out + j * K + k);
            float4 *gp = reinterpret_cast<float4 *>(n.grad_out + j * K + k);
            uchar4 mk = make_uchar4(0, 0, 0, 0);
            if (has_k) mk = *reinterpret_cast<const uchar4 *>(mrow + k);
            const bool upd = (mk.x | mk.y | mk.z | mk.w) != 0;
            if (upd && has_k) {
                w = *wp;
                if (n.record_grad) gg = *gp;
            }
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int b = 0; b < n.B; ++b) {
                const float z0 = zk_cur[(long long)b * N + j];
                const uint32_t *words = src_words_c(n, b, n.n_in + (int)j);
                const float *Eb = n.Ebar_win + (long long)b * U * K + k;
                float4 gb = make_float4(0.f, 0.f, 0.f, 0.f);
                if (has_k) {
                    const float4 cw = *reinterpret_cast<const float4 *>(n.Cwin + b * K + k);
                    gb = make_float4(z0 * cw.x, z0 * cw.y, z0 * cw.z, z0 * cw.w);
                }
                float zn = kU * z0;
                for (int g0 = 0; g0 < nwd; g0 += 32) {
                    const int st0 = base + 32 * (g0 + lane);     // this lane's word
                    const uint32_t wd = g0 + lane < nwd ? words[(st0 & mask) >> 5] : 0u;
                    for (int l = 0; l < min(32, nwd - g0); ++l) {
                        const int sb = base + 32 * (g0 + l);
                        uint32_t m = __shfl_sync(0xffffffffu, wd, l);
                        const int lo = max(a0 + 1 - sb, 0), hi = min(r_end - sb, 31);
                        m = (m >> lo) << lo;
                        if (hi < 31) m &= (2u << hi) - 1u;
                        while (m) {
                            const int st = sb + __ffs(m) - 1;
                            m &= m - 1;
                            // the spike reaches the readout d_out steps later
                            // (Eq. eprop-output-new-subs-rewritten with delay)
                            if (has_k && st + n.d_out <= r_end) {
                                const float4 e =
                                    *reinterpret_cast<const float4 *>(Eb + (long long)(st + n.d_out - a0 - 1) * K);
                                gb.x += e.x; gb.y += e.y; gb.z += e.z; gb.w += e.w;
                            }
                            zn += exp2f(n.log2_kappa * (float)(r_end - st));
                        }
                    }
                }
                g.x += gb.x; g.y += gb.y; g.z += gb.z; g.w += gb.w;
                if (k0 == 0 && lane == 0) zk_nxt[(long long)b * N + j] = zn;
            }
            if (upd && has_k) {
                // weights without a synapse (mask 0) keep their value and get
                // no gradient
                if (!mk.x) g.x = 0.f;
                if (!mk.y) g.y = 0.f;
                if (!mk.z) g.z = 0.f;
                if (!mk.w) g.w = 0.f;
                if (n.adam) {
                    *reinterpret_cast<float4 *>(n.gwin_out + j * K + k) =
                        make_float4(n.inv_B * g.x, n.inv_B * g.y, n.inv_B * g.z, n.inv_B * g.w);
                } else {
                    const float4 w0 = w;
                    if (mk.x) w.x -= s * g.x;
                    if (mk.y) w.y -= s * g.y;
                    if (mk.z) w.z -= s * g.z;
                    if (mk.w) w.w -= s * g.w;
                    if (n.sign_mask & 4) {
                        w.x = keep_sign(w0.x, w.x); w.y = keep_sign(w0.y, w.y);
                        w.z = keep_sign(w0.z, w.z); w.w = keep_sign(w0.w, w.w);
                    }
                    *wp = w;
                }
                if (n.record_grad) {
                    gg.x += n.inv_B * g.x; gg.y += n.inv_B * g.y; gg.z += n.inv_B * g.z; gg.w += n.inv_B * g.w;
                    *gp = gg;
                }
            }
        }
        return;
    }
    for (int k0 = 0; k0 < K; k0 += 32) {
        const int k = k0 + lane;
        const bool has_k = k < K;
        float g = 0.f;
        for (int b = 0; b < n.B; ++b) {
            const float z0 = zk_cur[(long long)b * N + j];
            const float *Eb = n.Ebar_win + (long long)b * U * K + k;
            float gb = has_k ? z0 * n.Cwin[b * K + k] : 0.f;
            float zn = kU * z0;
            for_each_spike(src_words_c(n, b, n.n_in + (int)j), n.RW, a0 + 1, r_end, [&](int st) {
                if (has_k && st + n.d_out <= r_end) gb += Eb[(long long)(st + n.d_out - a0 - 1) * K];
                zn += exp2f(n.log2_kappa * (float)(r_end - st));
            });
            g += gb;
            if (k0 == 0 && lane == 0) zk_nxt[(long long)b * N + j] = zn;
        }
        if (has_k && mrow[k]) {
            const long long idx = j * K + k;
            if (n.adam) {
                n.gwin_out[idx] = n.inv_B * g;
            } else {
                const float w0 = n.w_out[idx];
                const float wn = w0 - n.lr * n.inv_B * g;
                n.w_out[idx] = (n.sign_mask & 4) ? keep_sign(w0, wn) : wn;
            }
            if (n.record_grad) n.grad_out[idx] += n.inv_B * g;
        }
    }
}

// rollover to the next window: move each source's anchor to its last spike
// <= b - D and clear the bit positions of steps b+1 .. b+U.
__global__ void rollover_kernel(Net n, int i_end) {
    extern __shared__ uint32_t clear_mask[];
    const int U = n.U;
    const int r_end = run_step_w(n, i_end);
    const int a0 = r_end - U;
    const int S = n.RW * 32;
    for (int w = threadIdx.x; w < n.RW; w += blockDim.x) clear_mask[w] = 0u;
    __syncthreads();
    for (int r = r_end + 1 + threadIdx.x; r <= r_end + U; r += blockDim.x) {
        const int p = r & (S - 1);
        atomicOr(&clear_mask[p >> 5], 1u << (p & 31));
    }
    __syncthreads();
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n.B * n.n_src) return;
    uint32_t *words = n.bits + idx * n.RW;
    int at = n.anchor_t[idx];
    float az = n.anchor_z[idx];
    for_each_spike(words, n.RW, a0 + 1 - n.D, r_end - n.D, [&](int st) {
        az = (at == kNoSpike ? 0.f : az * exp2f(n.log2_alpha * (float)(st - at))) + 1.f;
        at = st;
    });
    n.anchor_t[idx] = at;
    n.anchor_z[idx] = az;
    for (int w = 0; w < n.RW; ++w) words[w] &= ~clear_mask[w];
    (void)a0;
}

// catch-up of every synapse to the last closed window boundary (a0 = r_base):
// write_back = 1 applies the pending gradient to the weights (end of a
// non-continuous call), else exports the effective weights and gradients
// without touching the state.
template <bool ALIF>
__global__ void flush_kernel(Net n, int i_end, float *w_dst, float *g_dst, long long q_begin,
                             long long q_end, int write_back) {
    __shared__ RowInfo info[8][kMaxDelay + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int a0 = n.clock->r_base + i_end;
    const int U = n.U;
    for (int src = gw; src < n.n_src; src += nw) {
        const long long q0 = max(n.row_ptr[src], q_begin), q1 = min(n.row_ptr[src + 1], q_end);
        if (q1 <= q0) continue;
        if (lane >= 1 && lane <= n.D)
            info[warp][lane] = row_info(n, src_words_c(n, 0, src), n.anchor_t[src],
                                        n.anchor_z[src], a0, lane, false);
        __syncwarp();
        for (long long q = q0 + lane; q < q1; q += 32) {
            const uint32_t td = n.tgt_d[q];
            const int j = (int)(td & 0xFFFFFFu);
            const int d = (int)(td >> 24);
            const RowInfo ri = info[warp][d];
            float G = 0.f;
            if (ri.b_prev != kNoSpike && ri.b_prev < a0) {
                float zbar = ri.zbar_bp;
                float ebar = load_trace(n.ebar, q, n.trace_type);
                float epsa = ALIF ? load_trace(n.epsa, q, n.trace_type) : 0.f;
                int k0 = ri.k_prev;
                const int k1 = a0 / U;
                if (k1 - k0 > n.RC) {
                    atomicOr(n.err_flags, 1u);
                    k0 = k1 - n.RC;
                }
                for (int k = k0; k < k1; ++k) apply_window<ALIF>(n, j, k, zbar, epsa, ebar, G);
            }
            const float wv = n.w[q] - n.lr * G;
            const float gv = n.record_grad ? n.grad[q] + G : 0.f;
            if (write_back) {
                n.w[q] = wv;
                if (n.record_grad) n.grad[q] = gv;
            } else {
                if (w_dst) w_dst[q - q_begin] = wv;
                if (g_dst) g_dst[q - q_begin] = gv;
            }
        }
        __syncwarp();
    }
}

__global__ void fill_int_kernel(int *p, long long count, int value) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        p[q] = value;
}

__global__ void unpack_raster_kernel(Net n, unsigned char *dst) {
    const long long total = (long long)n.B * n.T * n.n_rec;
    const int W32 = (n.T + 31) / 32;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q % n.n_rec);
        const long long bt = q / n.n_rec;
        const int t = (int)(bt % n.T);
        const int b = (int)(bt / n.T);
        dst[q] = (n.rec_raster[((long long)b * W32 + (t >> 5)) * n.n_rec + j] >> (t & 31)) & 1u;
    }
}

// Adam step at a window end (Eq. adam with the reordering of Eq. eta-adam-
// fast and Eq. delta-w-adam-fast, constant eps_hat): every synapse and every
// readout weight of a projecting neuron, from the window's batch-mean
// gradient left by the trace and readout kernels (cleared here for the next
// window).  k = the network's Adam steps so far + 1 (device counter, so a
// captured call replays correctly); the counter advances in the next kernel.
__global__ void adam_kernel(Net n) {
    const int k = n.clock->adam_k + 1;
    const double bc = sqrt(1.0 - pow((double)n.adam_b2, (double)k)) / (1.0 - pow((double)n.adam_b1, (double)k));
    const float eta = (float)((double)n.lr * bc);
    const long long nout = (long long)n.n_rec * n.n_out;
    const long long tot = n.nnz + nout;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        float *gp, *mp, *vp, *wp;
        bool fixed;
        if (i < n.nnz) {
            gp = n.gwin + i; mp = n.adam_m + i; vp = n.adam_v + i; wp = n.w + i;
            fixed = n.sign_mask && sign_fixed(n, i);
        } else {
            const long long o = i - n.nnz;
            if (!n.out_mask[o]) continue;
            gp = n.gwin_out + o; mp = n.adam_m_out + o; vp = n.adam_v_out + o; wp = n.w_out + o;
            fixed = (n.sign_mask & 4) != 0;
        }
        const float g = *gp;
        *gp = 0.0f;
        const float m = n.adam_b1 * *mp + (1.0f - n.adam_b1) * g;
        const float v = n.adam_b2 * *vp + (1.0f - n.adam_b2) * g * g;
        *mp = m;
        *vp = v;
        const float w0 = *wp;
        const float w = w0 - eta * m / (sqrtf(v) + n.adam_eps);
        *wp = fixed ? keep_sign(w0, w) : w;
    }
}

__global__ void adam_count_kernel(Net n) {
    if (threadIdx.x == 0) n.clock->adam_k += 1;
}

// ----------------------------------------------------------------- launches

void launch_adam(const Net &n, int sm_count, cudaStream_t st) {
    const long long tot = n.nnz + (long long)n.n_rec * n.n_out;
    long long blocks = (tot + 255) / 256;
    if (blocks > 8LL * sm_count) blocks = 8LL * sm_count;
    if (blocks < 1) blocks = 1;
    adam_kernel<<<(unsigned)blocks, 256, 0, st>>>(n);
    adam_count_kernel<<<1, 32, 0, st>>>(n);
}

void prepare_kernel_attributes() {
    const int tl = 200 * 1024;
#define EPROP_PASS_ATTR(A, P, T, G) \
    cudaFuncSetAttribute(window_pass_kernel<A, P, T, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, tl)
#define EPROP_PASS_ATTR2(A, T, G) EPROP_PASS_ATTR(A, kPassIdle, T, G); EPROP_PASS_ATTR(A, kPassFirst, T, G)
#define EPROP_PASS_ATTR3(A, G) EPROP_PASS_ATTR2(A, 0, G); EPROP_PASS_ATTR2(A, 1, G); EPROP_PASS_ATTR2(A, 2, G)
    EPROP_PASS_ATTR3(true, true); EPROP_PASS_ATTR3(true, false);
    EPROP_PASS_ATTR3(false, true); EPROP_PASS_ATTR3(false, false);
#undef EPROP_PASS_ATTR3
#undef EPROP_PASS_ATTR2
#undef EPROP_PASS_ATTR
    cudaFuncSetAttribute(trace_window_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tl);
    cudaFuncSetAttribute(trace_window_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tl);
    cudaFuncSetAttribute(trace_window_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, tl);
    cudaFuncSetAttribute(trace_window_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, tl);
}

void launch_begin_call(const Net &n, int continuous, cudaStream_t st) {
    begin_call_kernel<<<1, 64, 0, st>>>(n, continuous);
}

void launch_end_call(const Net &n, int T, cudaStream_t st) { end_call_kernel<<<1, 32, 0, st>>>(n, T); }

void launch_filter_error(const Net &n, int i_end, cudaStream_t st) {
    (void)i_end;
    const int tot = n.B * n.n_out;
    filter_error_kernel<<<(tot + 127) / 128, 128, 0, st>>>(n);
}

int launch_tables(const Net &n, int i_end, cudaStream_t st) {
    const int bd = 128;
    const dim3 grid((n.n_rec + bd - 1) / bd, n.B);
    const bool f64 = n.U > 128;          // long LIF windows sweep in FP64 (ALIF always does)
    if (n.R_win) {
        if (n.alif) tables_kernel<true, true, true><<<grid, bd, 0, st>>>(n, i_end);
        else if (f64) tables_kernel<false, true, true><<<grid, bd, 0, st>>>(n, i_end);
        else tables_kernel<false, true, false><<<grid, bd, 0, st>>>(n, i_end);
    } else {
        if (n.alif) tables_kernel<true, false, true><<<grid, bd, 0, st>>>(n, i_end);
        else if (f64) tables_kernel<false, false, true><<<grid, bd, 0, st>>>(n, i_end);
        else tables_kernel<false, false, false><<<grid, bd, 0, st>>>(n, i_end);
    }
    return 0;
}

void launch_trace_window(const Net &n, int i_end, int grid_x, cudaStream_t st) {
    window_offsets_kernel<<<1, 32, 0, st>>>(n, i_end);
    const size_t sm = sizeof(StageBuf) * 8 * kTStages + (size_t)(n.U + n.D + 1) * sizeof(long long);
    if (n.has_state) {
        if (n.alif) trace_window_kernel<true, true><<<grid_x, 256, sm, st>>>(n, i_end);
        else trace_window_kernel<false, true><<<grid_x, 256, sm, st>>>(n, i_end);
    } else {
        if (n.alif) trace_window_kernel<true, false><<<grid_x, 256, sm, st>>>(n, i_end);
        else trace_window_kernel<false, false><<<grid_x, 256, sm, st>>>(n, i_end);
    }
}

void launch_window_pass(const Net &n, int i_end, int grid_x, int grid_idle, cudaStream_t st) {
    window_offsets_kernel<<<1, 32, 0, st>>>(n, i_end);
    const size_t sb = sizeof(StageBuf) * 8 * kPStages;
    const size_t sm = sb + (size_t)(n.U + n.D + 2) * sizeof(long long);
#define EPROP_PASS(A, T, G)                                                             \
    do {                                                                                \
        window_pass_kernel<A, kPassFirst, T, G><<<grid_x, 256, sm, st>>>(n, i_end);     \
        window_pass_kernel<A, kPassIdle, T, G><<<grid_idle, 256, sb, st>>>(n, i_end);   \
    } while (0)
#define EPROP_PASS_T(A, G)                                        \
    do {                                                          \
        if (n.trace_type == 1) EPROP_PASS(A, 1, G);               \
        else if (n.trace_type == 2) EPROP_PASS(A, 2, G);          \
        else EPROP_PASS(A, 0, G);                                 \
    } while (0)
    const bool gen = n.adam || n.sign_mask;
    if (n.alif) {
        if (gen) EPROP_PASS_T(true, true); else EPROP_PASS_T(true, false);
    } else {
        if (gen) EPROP_PASS_T(false, true); else EPROP_PASS_T(false, false);
    }
#undef EPROP_PASS_T
#undef EPROP_PASS
}

void launch_window_batched(const Net &n, int i_end, int sm_count, cudaStream_t st) {
    int blocks = (n.n_src + 7) / 8;
    if (blocks > 8 * sm_count) blocks = 8 * sm_count;
#define EPROP_WB(A, T)                                                                                   \
    do {                                                                                                 \
        if (n.adam || n.sign_mask) window_batched_kernel<A, T, true><<<blocks, 256, 0, st>>>(n, i_end);  \
        else window_batched_kernel<A, T, false><<<blocks, 256, 0, st>>>(n, i_end);                       \
    } while (0)
#define EPROP_WB_T(A)                                  \
    do {                                               \
        if (n.trace_type == 1) EPROP_WB(A, 1);         \
        else if (n.trace_type == 2) EPROP_WB(A, 2);    \
        else EPROP_WB(A, 0);                           \
    } while (0)
    if (n.alif) EPROP_WB_T(true);
    else EPROP_WB_T(false);
#undef EPROP_WB_T
#undef EPROP_WB
}

void launch_trace_batched(const Net &n, int sm_count, cudaStream_t st) {
    int blocks = (n.n_src + 7) / 8;
    if (blocks > 8 * sm_count) blocks = 8 * sm_count;
    if (n.alif) trace_batched_kernel<4><<<blocks, 256, 0, st>>>(n);
    else trace_batched_kernel<2><<<blocks, 256, 0, st>>>(n);
}

void launch_readout_weights(const Net &n, int i_end, cudaStream_t st) {
    readout_weights_kernel<<<(unsigned)(((long long)n.n_rec * 32 + 255) / 256), 256, 0, st>>>(n, i_end);
}

void launch_rollover(const Net &n, int i_end, cudaStream_t st) {
    const long long tot = (long long)n.B * n.n_src;
    rollover_kernel<<<(unsigned)((tot + 255) / 256), 256, n.RW * sizeof(uint32_t), st>>>(n, i_end);
}

void launch_flush(const Net &n, int i_end, float *w_dst, float *g_dst, long long q_begin, long long q_end,
                  int write_back, int sm_count, cudaStream_t st) {
    int blocks = (n.n_src + 7) / 8;
    if (blocks > 8 * sm_count) blocks = 8 * sm_count;
    if (n.alif) flush_kernel<true><<<blocks, 256, 0, st>>>(n, i_end, w_dst, g_dst, q_begin, q_end, write_back);
    else flush_kernel<false><<<blocks, 256, 0, st>>>(n, i_end, w_dst, g_dst, q_begin, q_end, write_back);
}

void launch_fill_int(int *p, long long count, int value, cudaStream_t st) {
    if (count <= 0) return;
    long long blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    fill_int_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, count, value);
}

void launch_unpack_raster(const Net &n, unsigned char *dst, cudaStream_t st) {
    unpack_raster_kernel<<<1024, 256, 0, st>>>(n, dst);
}

}  // namespace eprop
