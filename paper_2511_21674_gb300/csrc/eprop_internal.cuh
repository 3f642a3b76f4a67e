// Internal definitions shared by the CUDA translation units of libeprop.
//
// Data layout in HBM (one network, batch B, N recurrent neurons, S = n_in + N
// sources, nnz synapses, D = max delay, U = update window in steps):
//   synapse records, CSR by source (SoA, 4-byte aligned streams):
//     tgt_d [nnz] u32   target | delay << 24
//     w     [nnz] f32   weight in effect after the synapse's last update
//     ebar  [nnz] f32/bf16  filtered eligibility trace at the end of the
//                       update window of the synapse's last arrival
//     epsa  [nnz] f32/bf16  adaptation eligibility (ALIF only)
//     grad  [nnz] f32   cumulative applied gradient (optional)
//   neurons [B][N]: v, a, ref, z_prev; psi history [B][U+1][N] (slot 0 =
//     last step of the previous window)
//   membrane input ring [B][D+1][N] int64 fixed point (2^-32): arrivals are
//     summed exactly, so the result does not depend on the atomic order
//   source spike bits [B][S][RW] u32: a ring of RW*32 >= U+D steps per source
//   source anchor [B][S]: last spike before the ring range and the
//     presynaptic trace sum_s alpha^{t-s} right after it
//   per-step spike lists (ring of RS steps) [B][RS][kBkt][cap] i32 with
//     counts [B][RS][kBkt]: a source appends to bucket (src >> 8) % kBkt, so
//     the appends of one step spread over kBkt counters
//   window tables [B][U][N] float2 (LIF: Q, Pe) or float4 (ALIF: Q, Pe, Pa)
//   window coefficients (ring of RC windows) [N][RC] float4 (LIF) or
//     2 x float4 (ALIF): neuron-major, so a catch-up over consecutive
//     windows reads contiguous entries
//   readout: W_out [N][K], B [N][K], y [B][K], error window [B][U][K]
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace eprop {

constexpr int kMaxDelay = 8;
constexpr int kSeg = 128;          // synapses per segment of the row kernels
constexpr int kSegPerLane = kSeg / 32;
constexpr int kSpikeCap = 64;      // spikes of one row cached per warp
constexpr int kMaxOut = 1024;
constexpr double kFixScale = 4294967296.0;          // 2^32
constexpr float kFixInv = 2.3283064365386963e-10f;  // 2^-32
constexpr int kNoSpike = -1073741824;               // "no spike" time

struct Clock {            // device-resident time base (graph-safe)
    long long t_abs_base; // absolute steps completed before the current call
    int r_base;           // steps since the last state reset before the call
    int ring0;            // t_abs_base mod (D + 1): ring slot of absolute step t_abs_base
    int adam_k;           // Adam steps taken
};

struct GridBar {           // grid barrier of the persistent step loop
    unsigned count, gen, abort;
};

struct Net {
    // sizes
    int n_in, n_rec, n_out, n_src, B, D, U, RW, RS, RC;
    long long nnz;
    // model switches
    int alif, t_ref, loss, feedback, has_state, trace_bf16, record_grad, record_raster, record_psi;
    int trace_type;           // trace storage: 0 FP32, 1 BF16, 2 FP16 (trace_bf16: any 16-bit form)
    int dense;                // 1: every synapse advanced at every window end (no catch-up)
    int n_thr, T;             // T of the current call
    int segs;                 // segments per row: ceil(max out-degree / kSeg)
    int list_cap;             // entries per spike-list bucket
    // constants (float, computed on the host in double)
    float alpha, rho, kappa, kappa_e, beta_a, v_th, gamma, beta_sg, lr, drive_weight;
    float alpha_lo, rho_lo;   // alpha - (float)alpha, rho - (float)rho
    float kappa_e_lo;         // kappa_e - (float)kappa_e (the FP64 adjoint sweep uses both)
    float kappa_lo;           // kappa - (float)kappa (the FP64 error filter uses both)
    float log2_alpha, log2_kappa, alphaU, kappaeU, inv_B;
    unsigned long long drive_seed;
    const uint32_t *drive_thr;
    // synapses
    const long long *row_ptr;
    const uint32_t *tgt_d;
    float *w;
    void *ebar;
    void *epsa;
    float *grad;
    // neurons: v and a are carried as unevaluated FP32 pairs (hi + lo)
    float *v, *a, *v_lo, *a_lo, *psi_hist;
    int *ref;
    uint8_t *z_prev;
    long long *ring;
    // sources
    uint32_t *bits;
    int *anchor_t;
    float *anchor_z;
    int *list_ids;
    int *list_cnt;
    // readout
    float *w_out;
    const uint8_t *out_mask;
    const float *fb;          // feedback matrix (== w_out when symmetric)
    float *grad_out;
    float *y;
    long long *y_acc;
    float *E_win, *Ebar_win, *Cwin;
    float *L_win;             // [B][U][N] learning signals L = B E of the window (tensor cores)
    float *zk, *zk_next;
    float *y_rec, *loss_acc;
    // window tables
    float *qp;
    float *coef;
    long long *win_off;       // [U + D + 2] work-item offsets of the window, then
                              // kWorkCounters work counters of the row kernels
    // inputs of the current call
    const long long *x_ptr;
    const int *x_ids;
    const float *targets;
    const uint8_t *window;
    const int *lengths;
    const uint8_t *forced;
    uint32_t *rec_raster;     // [B][T/32+1][N] bits (record_raster)
    float *rec_psi;           // [B][T][N] (record_psi)
    // learned learning-signal predictor (attached with eprop_attach_predictor)
    int pred_mode;            // 0 none; bit 0 predict E outside the target window; bit 1 record inputs
    int pred_in;              // n_out + kPopGroups inputs per row
    float pop_beta;           // exp(-dt / 20 ms)
    int *pop_cnt;             // [B][kPopGroups] spikes of the step per group
    float *pop_rate;          // [B][kPopGroups] filtered group rates
    const float *pop_inv;     // [kPopGroups] 1 / group size
    float *pred_x;            // [B][pred_in] inputs of the current step
    float *pred_rec;          // [B][T][pred_in] recorded inputs (bit 1)
    const float *pred_y;      // [B][n_out] predictor outputs of the current step
    int *ro_done;             // [B] readout blocks finished in the current step
    unsigned long long *events;
    unsigned int *err_flags;  // bit 0: catch-up ring overflow
    Clock *clock;
    // e-prop+ variants and constraints
    int surrogate;            // 0 piecewise linear, 1 exponential
    int reset_mode;           // 0 subtract the threshold, 1 fixed value
    float v_reset;
    float c_reg, f_target, beta_reg;   // firing-rate regularisation (c_reg 0: off)
    float *rate;              // [B][N] moving-average rate f_j
    float *R_win;             // [B][U][N] c_reg (1 - beta_reg) (f_j^t - f_target) of the window
    int sign_mask;            // fixed weight signs: 1 input, 2 recurrent, 4 readout
    long long nnz_in;         // input synapses come first in the CSR order
    int adam;                 // 1: Adam steps at window ends
    float adam_b1, adam_b2, adam_eps;
    float *gwin, *gwin_out;   // [nnz], [N][K] batch-mean gradient of the window (Adam)
    float *adam_m, *adam_v, *adam_m_out, *adam_v_out;
    int if_period;            // ignore-and-fire period (0: off)
    unsigned long long if_seed;
    int d_out, d_ls;          // generalized delays: readout input, learning signal
    // band-major learning state (trace_kernel 4, kernels_band.cu): w, ebar,
    // epsa and grad above are then in band-major order, tgt_d stays the
    // source-major packing of the creation arrays (read-back order)
    int band;                 // 1: band-major synapse records
    int band_w, nb;           // targets per band, number of bands
    int rr_stride, rr_cap;    // bytes per row record, spikes kept per record
    int band_stages;          // shared-memory stages of the band window kernel
    unsigned band_stage_b;    // bytes per stage
    long long nnz_b;          // band-major records incl. padding (multiple of kBandTile)
    long long n_tiles;        // nnz_b / kBandTile
    const uint32_t *bd_td;    // [nnz_b] (target - band start) | (delay - 1) << 14 | (row - tile row0) << 17
    const int *seg;           // [n_src + 1][nb] first position of each row inside each band
    const long long *band_base;   // [nb + 1] first record of each band (padded)
    const int4 *tiles;        // [n_tiles] (first row, rows spanned, band, 0)
    unsigned char *rrec;      // [n_src][rr_stride] row records of the current window
};

// Band-major form: records of one band (a range of band_w targets) are
// contiguous, by source row, padded to whole tiles of kBandTile records.
// two records per consumer thread of the band window kernel (16 consumer
// warps); a tile's 4-byte and 2-byte streams start on 16-byte boundaries
constexpr int kBandTile = 1024;
constexpr uint32_t kBandPad = 0xFFFFFFFFu;     // bd_td of a padding record

// ----------------------------------------------------------------- helpers

// ---- bulk asynchronous copies (TMA, 1-D) into shared memory, completed on
// an mbarrier.  Every wait is bounded: after kWaitLimit polls the kernel
// records an error flag (bit 1) and stops waiting.
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// L2 policy for data read once (synapse record streams): evicted first, so
// the streams do not push the tables and ring buffers out of L2
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// dst, src and bytes multiples of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(l2_evict_first())
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false (and error bit 1) when the limit is reached
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err) {
    for (unsigned it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(err, 2u);
    return false;
}

// One pipeline stage of a row kernel: kChunk synapse records of one row.
// Each stream is copied from the 16-byte-aligned start at or before the
// chunk (q_al for 4-byte streams, q_al2 for 2-byte streams).
constexpr int kChunk = 256;
constexpr int kChunkPad = kChunk + 8;
struct alignas(16) StageBuf {
    uint32_t td[kChunkPad];
    float w[kChunkPad];
    uint32_t tr[kChunkPad];       // trace stream: kChunkPad floats or 2*kChunkPad bf16
};
struct StageDesc {
    long long q0, q_al, q_al2;
    int n, src, first, row;
};

constexpr int kBkt = 32;           // spike-list buckets per step
constexpr int kPopGroups = 64;     // population-rate groups of the predictor inputs (j mod 64)
constexpr int kWorkCounters = 2;   // row-kernel work counters kept after the window offsets

__device__ __forceinline__ long long list_index(const Net &n, int b, int slot) {
    return (long long)(b * n.RS + slot) * kBkt;
}

// Warp-cooperative view of the kBkt buckets of one spike list: lane k holds
// the inclusive prefix of the counts of buckets 0..k.
struct BucketScan {
    int incl, total;
};
__device__ __forceinline__ BucketScan bucket_scan(const int *cnt) {
    const int lane = threadIdx.x & 31;
    int v = cnt[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    BucketScan bs;
    bs.incl = v;
    bs.total = __shfl_sync(0xffffffffu, v, 31);
    return bs;
}
// Entry r (warp-uniform, < total) of the list: its source id.
__device__ __forceinline__ int bucket_entry(const Net &n, const int *ids, const BucketScan &bs, int r) {
    const int bk = __popc(__ballot_sync(0xffffffffu, bs.incl <= r));
    const int prev = __shfl_sync(0xffffffffu, bs.incl, bk > 0 ? bk - 1 : 0);
    const int idx = r - (bk > 0 ? prev : 0);
    return ids[(long long)bk * n.list_cap + idx];
}

// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated first-order recursion x' = c * x + u in FP32 pairs:
// (x_hi + x_lo) and (c_hi + c_lo), u = u_hi + u_lo; error-free product
// (FMA) and TwoSum, then renormalisation (Fast2Sum).  Keeps the recursion's
// rounding error at the level of the FP32 pair instead of accumulating one
// FP32 rounding of |x| per step.
__device__ __forceinline__ void comp_step(float c_hi, float c_lo, float u_hi, float u_lo,
                                          float &x_hi, float &x_lo) {
    const float p = c_hi * x_hi;
    const float pe = fmaf(c_hi, x_hi, -p);
    const float small = fmaf(c_hi, x_lo, fmaf(c_lo, x_hi, pe)) + u_lo;
    const float s = p + u_hi;
    const float bb = s - p;
    const float err = (p - (s - bb)) + (u_hi - bb);
    const float lo = err + small;
    const float hi = s + lo;
    x_lo = lo - (hi - s);
    x_hi = hi;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    // SplitMix64 output function (Steele, Lea & Flood 2014)
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float pow_alpha(const Net &n, int k) {
    return k <= 0 ? 1.0f : exp2f(n.log2_alpha * (float)k);
}
__device__ __forceinline__ float pow_kappa(const Net &n, int k) {
    return k <= 0 ? 1.0f : exp2f(n.log2_kappa * (float)k);
}

__device__ __forceinline__ bool bit_at(const uint32_t *words, int RW, int r) {
    int p = r & (RW * 32 - 1);
    return (words[p >> 5] >> (p & 31)) & 1u;
}

// Record streams are touched once per event: evict-first loads and
// streaming stores keep them from displacing the lookup tables in L2.
// 16-bit trace values: BF16 (type 1) or FP16 (type 2), rounded to nearest
// even on the way in
__device__ __forceinline__ float trace16_to_float(unsigned short h, int type) {
    return type == 2 ? __half2float(__ushort_as_half(h)) : __bfloat162float(__ushort_as_bfloat16(h));
}
__device__ __forceinline__ unsigned short float_to_trace16(float x, int type) {
    return type == 2 ? __half_as_ushort(__float2half_rn(x)) : __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float load_trace(const void *base, long long q, int type) {
    if (type) {
        const unsigned short h = __ldcs(reinterpret_cast<const unsigned short *>(base) + q);
        return trace16_to_float(h, type);
    }
    return __ldcs(reinterpret_cast<const float *>(base) + q);
}
__device__ __forceinline__ void store_trace(void *base, long long q, float x, int type) {
    if (type) __stcs(reinterpret_cast<unsigned short *>(base) + q, float_to_trace16(x, type));
    else __stcs(reinterpret_cast<float *>(base) + q, x);
}

// Weight after an update, kept on the side of zero of the old weight (the
// old weight's sign bit is the synapse's fixed sign: a weight that reaches
// zero becomes a zero of its own sign, so the sign survives).
__device__ __forceinline__ float keep_sign(float w_old, float w_new) {
    if (signbit(w_old)) return w_new < 0.0f ? w_new : -0.0f;
    return w_new > 0.0f ? w_new : 0.0f;
}
__device__ __forceinline__ bool sign_fixed(const Net &n, long long q) {
    return (n.sign_mask >> (q < n.nnz_in ? 0 : 1)) & 1;
}
// Window-end update of synapse q from its batch-summed gradient G (Eq.
// gradient-descent): returns the new weight, or, with Adam, records the
// batch mean for the Adam step and returns the weight unchanged.
__device__ __forceinline__ float window_update(const Net &n, long long q, float w_old, float G) {
    if (n.adam) {
        n.gwin[q] = n.inv_B * G;
        return w_old;
    }
    const float w = w_old - n.lr * n.inv_B * G;
    return (n.sign_mask && sign_fixed(n, q)) ? keep_sign(w_old, w) : w;
}

// Presynaptic summary of one source row for one delay d, relative to the
// update window (a0, a0 + U]:
//   zbar_a0  presynaptic trace F_alpha of the arrivals up to a0, at a0
//   b_prev   end of the window holding the last arrival <= a0 (kNoSpike: none)
//   zbar_bp  trace at b_prev
//   k_prev   index of the first window after b_prev (b_prev / U)
struct RowInfo {
    float zbar_a0, zbar_bp;
    int b_prev, k_prev;      // k_prev = b_prev / U (window index after b_prev)
};

// Computes RowInfo for delay d from the source's spike bits and anchor.
// The bit ring covers run steps [a0 + 1 - D, a0 + U].
__device__ __forceinline__ RowInfo row_info(const Net &n, const uint32_t *words, int anchor_t,
                                            float anchor_z, int a0, int d, bool want_first) {
    RowInfo ri;
    const int lo = a0 + 1 - n.D;
    const int lim = a0 - d;            // last emission whose arrival is <= a0
    int s_p = anchor_t;
    float z_p = anchor_z;
    for (int s = (lo > 1 ? lo : 1); s <= lim; ++s) {
        if (bit_at(words, n.RW, s)) {
            z_p = s_p == kNoSpike ? 1.0f : __fmaf_rn(z_p, pow_alpha(n, s - s_p), 1.0f);
            s_p = s;
        }
    }
    if (s_p == kNoSpike) {
        ri.zbar_a0 = 0.0f;
        ri.zbar_bp = 0.0f;
        ri.b_prev = kNoSpike;
        ri.k_prev = 0;
    } else {
        const int a_p = s_p + d;
        const int b_p = ((a_p + n.U - 1) / n.U) * n.U;
        ri.b_prev = b_p;
        ri.k_prev = b_p / n.U;
        ri.zbar_bp = __fmul_rn(z_p, pow_alpha(n, b_p - a_p));
        ri.zbar_a0 = __fmul_rn(z_p, pow_alpha(n, a0 - a_p));
    }
    (void)want_first;
    return ri;
}

// Coefficients of one window of one neuron: LIF (cz, ce, mez, -); ALIF
// (cz, ca, ce, maz), (maa, mez, mea, -).
struct Coef {
    float4 c0, c1;
};
template <bool ALIF>
__device__ __forceinline__ Coef load_coef(const Net &n, long long j, int k) {
    Coef c;
    const int slot = k & (n.RC - 1);
    if (ALIF) {
        const float4 *p = reinterpret_cast<const float4 *>(n.coef) + ((long long)j * n.RC + slot) * 2;
        c.c0 = __ldg(p);
        c.c1 = __ldg(p + 1);
    } else {
        c.c0 = __ldg(reinterpret_cast<const float4 *>(n.coef) + (long long)j * n.RC + slot);
        c.c1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return c;
}
// The dense window pass keeps one window of coefficients (RC = 1): target
// j's entry is entry j.
template <bool ALIF>
__device__ __forceinline__ Coef load_coef_dense(const Net &n, uint32_t j) {
    Coef c;
    if (ALIF) {
        const float4 *p = reinterpret_cast<const float4 *>(n.coef) + 2u * j;
        c.c0 = __ldg(p);
        c.c1 = __ldg(p + 1);
    } else {
        c.c0 = __ldg(reinterpret_cast<const float4 *>(n.coef) + j);
        c.c1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return c;
}
// The window transfer's products and sums are spelled out with explicit
// rounding (fmaf / fmul intrinsics, never contracted or reordered by the
// compiler), so every kernel that applies it (source-major and band-major
// window passes, lazy catch-up) rounds the same way.
__device__ __forceinline__ float dot2_rn(float a, float x, float b, float y) {
    return __fmaf_rn(a, x, __fmul_rn(b, y));
}
__device__ __forceinline__ float dot3_rn(float a, float x, float b, float y, float c, float z) {
    return __fmaf_rn(a, x, __fmaf_rn(b, y, __fmul_rn(c, z)));
}
// plain window-end step w - step G and the gradient record g + G / B, one
// rounding each (see dot2_rn)
__device__ __forceinline__ float sgd_step(float w, float step, float G) { return __fmaf_rn(-step, G, w); }
__device__ __forceinline__ float grad_add(float g, float inv_B, float G) { return __fmaf_rn(inv_B, G, g); }
template <bool ALIF>
__device__ __forceinline__ void apply_coef(const Net &n, const Coef &c, float &zbar, float &epsa,
                                           float &ebar, float &G) {
    if (ALIF) {
        G = __fadd_rn(G, dot3_rn(c.c0.x, zbar, c.c0.y, epsa, c.c0.z, ebar));
        const float ea = dot2_rn(c.c0.w, zbar, c.c1.x, epsa);
        const float ee = dot3_rn(c.c1.y, zbar, c.c1.z, epsa, n.kappaeU, ebar);
        epsa = ea;
        ebar = ee;
    } else {
        G = __fadd_rn(G, dot2_rn(c.c0.x, zbar, c.c0.y, ebar));
        ebar = dot2_rn(c.c0.z, zbar, n.kappaeU, ebar);
    }
    zbar = __fmul_rn(zbar, n.alphaU);
}

// Window transfer of one synapse state x = (zbar, eps_a, ebar) over window
// index k (coefficients c, Phi from the coefficient ring); adds c . x to G.
template <bool ALIF>
__device__ __forceinline__ void apply_window(const Net &n, long long j, int k, float &zbar,
                                             float &epsa, float &ebar, float &G) {
    const int slot = k & (n.RC - 1);
    Coef cf;
    if (ALIF) {
        const float4 *c = reinterpret_cast<const float4 *>(n.coef) + ((long long)j * n.RC + slot) * 2;
        cf.c0 = c[0];                        // (cz, ca, ce, maz), (maa, mez, mea, -)
        cf.c1 = c[1];
    } else {
        cf.c0 = __ldg(reinterpret_cast<const float4 *>(n.coef) + (long long)j * n.RC + slot);   // (cz, ce, mez, -)
        cf.c1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    apply_coef<ALIF>(n, cf, zbar, epsa, ebar, G);
}

}  // namespace eprop
