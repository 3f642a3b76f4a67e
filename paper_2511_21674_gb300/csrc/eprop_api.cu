// C ABI of libeprop (see include/eprop.h): argument checks, device memory,
// and the launch schedule of one simulate call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "eprop.h"
#include "eprop_internal.cuh"
#include "eprop_launch.h"
#include "eprop_predictor.h"
#include "predictor_internal.h"

using eprop::Net;

struct DevAlloc {          // one device allocation of the network and its size
    void *p;
    size_t bytes;
};

struct eprop_net {
    eprop_config cfg;
    Net n;
    cudaStream_t st = nullptr;
    int dev = 0, sm_count = 1;
    std::string err;
    int bad = 0;
    std::vector<DevAlloc> fixed_allocs;   // freed at destroy
    std::vector<DevAlloc> win_allocs;     // window-sized buffers
    std::vector<DevAlloc> in_allocs;      // per-T input buffers
    long long nnz_in = 0;
    int U_alloc = 0, T_alloc = 0, T_in = 0, U_fixed = 0;
    int trace_mode = 0;                 // 0 window work queue, 1 batched, 2 dense window pass,
                                        // 3 band-major dense window pass
    int qp_stride = 2;
    long long x_cap = 0;
    long long max_in_per_step = 0;
    long long t_abs = 0;
    int r_base = 0;
    cudaGraphExec_t gexec = nullptr;
    int g_T = -1;
    int have_inputs = 0;
    int have_sim = 0;                   // a simulate call ran since the last set_inputs
    int own_stream = 0;
    // the readout work of a call runs on a second stream, forked from and
    // joined back into st by events (also inside a captured graph)
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    float *tmp_w = nullptr, *tmp_g = nullptr;
    std::vector<cudaEvent_t> ev;        // [2 * windows] trace timing events
    long long launches = 0, trace_launches = 0, windows = 0;
    unsigned char *tmp_raster = nullptr;
    long long tmp_raster_bytes = 0;
    eprop_predictor *pred = nullptr;    // attached learned learning-signal predictor
    int *pop_cnt_buf = nullptr;
    eprop::GridBar *gridbar = nullptr;  // persistent step loop (launch_mode 2)
    int pers_blocks = 0;
    cudaError_t launch_err = cudaSuccess;
};

static thread_local std::string g_create_err;

static eprop_status fail(eprop_net *net, eprop_status s, const std::string &msg) {
    if (net) net->err = msg;
    else g_create_err = msg;
    return s;
}

static eprop_status cuda_fail(eprop_net *net, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (net) {
        net->bad = 1;
        net->err = m;
    } else {
        g_create_err = m;
    }
    return e == cudaErrorMemoryAllocation ? EPROP_ENOMEM : EPROP_ECUDA;
}

#define CK(net, call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return cuda_fail((net), _e, #call); \
    } while (0)

static cudaError_t dalloc(std::vector<DevAlloc> &owner, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    owner.push_back(DevAlloc{*p, bytes});
    return cudaMemset(*p, 0, bytes);
}

static void free_all(std::vector<DevAlloc> &v) {
    for (const DevAlloc &a : v) cudaFree(a.p);
    v.clear();
}

static int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// ------------------------------------------------------- validation kernels

__global__ void check_synapses_kernel(const int32_t *tgt, const uint8_t *dly, long long nnz, int n_rec,
                                      int D, unsigned int *flag) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nnz;
         q += (long long)gridDim.x * blockDim.x) {
        if (tgt[q] < 0 || tgt[q] >= n_rec) atomicOr(flag, 1u);
        if (dly[q] < 1 || dly[q] > D) atomicOr(flag, 2u);
    }
}

__global__ void pack_synapses_kernel(const int32_t *tgt, const uint8_t *dly, const float *w, long long nnz,
                                     uint32_t *tgt_d, float *w_dst) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nnz;
         q += (long long)gridDim.x * blockDim.x) {
        tgt_d[q] = (uint32_t)tgt[q] | ((uint32_t)dly[q] << 24);
        w_dst[q] = w[q];
    }
}

__global__ void check_inputs_kernel(const long long *ptr, long long nptr, const int32_t *ids, long long nids,
                                    const int32_t *lengths, int B, int T, int n_in, unsigned int *flag) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = tid; q < nids; q += stride)
        if (ids[q] < 0 || ids[q] >= n_in) atomicOr(flag, 1u);
    for (long long q = tid; q + 1 < nptr; q += stride)
        if (ptr[q + 1] < ptr[q]) atomicOr(flag, 2u);
    if (tid == 0 && (ptr[0] != 0 || ptr[nptr - 1] != nids)) atomicOr(flag, 2u);
    if (lengths)
        for (long long b = tid; b < B; b += stride)
            if (lengths[b] < 1 || lengths[b] > T) atomicOr(flag, 4u);
}

// ------------------------------------------------------------- allocation

static eprop_status alloc_window(eprop_net *net, int U, int T) {
    Net &n = net->n;
    const eprop_config &c = net->cfg;
    if (net->U_alloc == U) return EPROP_OK;
    cudaStreamSynchronize(net->st);
    free_all(net->win_allocs);
    if (net->gexec) {
        cudaGraphExecDestroy(net->gexec);
        net->gexec = nullptr;
        net->g_T = -1;
    }
    const long long B = c.batch, N = c.n_rec, K = c.n_out, S = n.n_src;
    const int D = c.max_delay;
    n.U = U;
    n.alphaU = (float)std::exp(-(double)c.dt / c.tau_m * U);
    n.kappaeU = (float)(c.kappa_e < 0.f ? std::exp(-(double)c.dt / c.tau_out * U)
                                        : std::pow((double)c.kappa_e, (double)U));
    n.RW = next_pow2((U + D + 31) / 32);
    net->qp_stride = c.neuron_model == 1 ? 4 : 2;
    const double qp_bytes = (double)U * N * net->qp_stride * 4.0 * B;
    if (c.trace_kernel == 1) net->trace_mode = 0;
    else if (c.trace_kernel == 2) net->trace_mode = 1;
    else if (c.trace_kernel == 3) net->trace_mode = 2;
    else if (c.trace_kernel == 4) net->trace_mode = 3;
    else net->trace_mode = n.has_state ? 2 : (B > 1 ? 1 : 0);
    (void)qp_bytes;
    // row records keep spike steps as 16-bit offsets inside the window
    if (net->trace_mode == 3 && U + D > 65536)
        return fail(net, EPROP_EINVAL, "trace_kernel 4 needs update windows of at most 65536 - max_delay steps");
    n.dense = (net->trace_mode == 2 || net->trace_mode == 3) ? 1 : 0;
    // the readout reads the spike list of the step d_out back
    n.RS = std::max(net->trace_mode != 1 ? U + D + 1 : 2, c.d_out + 2);
    n.RC = 0;
    if (n.has_state && n.dense) {
        n.RC = 1;                       // only the current window's coefficients
    } else if (n.has_state) {
        // keep the coefficients of every window whose state can still matter:
        // a state skipped for RC windows has decayed by exp(-RC U / tau) with
        // the slowest synaptic time constant; RC is a power of two >= 4
        const double tau = std::max({(double)c.tau_m, (double)c.tau_out,
                                     c.neuron_model == 1 ? (double)c.tau_a : 0.0}) / c.dt;
        int rc = 4;
        while (rc < 256 && std::exp(-(double)rc * U / tau) > 1e-30) rc <<= 1;
        n.RC = rc;
    }
    std::vector<DevAlloc> &o = net->win_allocs;
    void *p;
#define WA(field, type, count)                                                   \
    do {                                                                         \
        cudaError_t _e = dalloc(o, &p, (size_t)(count) * sizeof(type));          \
        if (_e != cudaSuccess) return cuda_fail(net, _e, "window allocation");   \
        n.field = reinterpret_cast<decltype(n.field)>(p);                        \
    } while (0)
    WA(bits, uint32_t, B * S * n.RW);
    n.list_cap = (int)((((S + 255) / 256) + eprop::kBkt - 1) / eprop::kBkt * 256);
    WA(list_ids, int, B * n.RS * eprop::kBkt * (long long)n.list_cap);
    WA(list_cnt, int, B * n.RS * eprop::kBkt);
    WA(psi_hist, float, B * (U + 1) * N);
    WA(E_win, float, B * U * K);
    WA(L_win, float, B * (long long)U * N);
    if (c.c_reg != 0.f) WA(R_win, float, B * (long long)U * N);
    WA(Ebar_win, float, B * U * K);
    WA(qp, float, B * (long long)U * N * net->qp_stride);
    WA(win_off, long long, U + D + 2 + eprop::kWorkCounters);
    if (n.has_state) WA(coef, float, B * n.RC * N * (c.neuron_model == 1 ? 8 : 4));   // [B][N][RC]
#undef WA
    net->U_alloc = U;
    net->T_alloc = T;
    return EPROP_OK;
}

// Band-major records (trace_kernel 4, kernels_band.cu), built from the
// source-major packing (n.tgt_d, n.w): per row and band the count and first
// position (seg), bands padded to whole tiles, per tile its first row and
// band, then every record placed.  The source-major weights are freed; n.w
// becomes the band-major array.
static eprop_status build_band(eprop_net *net) {
    Net &n = net->n;
    std::vector<DevAlloc> &o = net->fixed_allocs;
    eprop::prepare_band_attributes();
    const int S = n.n_src, N = n.n_rec;
    const int Wmax = eprop::band_width(n.alif != 0);
    // the kernels use the band width as a compile-time constant
    const int nb = (N + Wmax - 1) / Wmax;
    const int W = Wmax;
    n.band = 1;
    n.band_w = W;
    n.nb = nb;
    // row record: zbar per delay, arrival range per delay, >= 8 spike steps
    n.rr_stride = (6 * n.D + 16 + 15) & ~15;
    n.rr_cap = (n.rr_stride - 6 * n.D) / 2;
    n.band_stages = eprop::band_stages_fit(n.alif != 0, n.rr_stride);
    n.band_stage_b = eprop::band_stage_size(n.alif != 0, n.rr_stride);
    std::vector<DevAlloc> tmp;
    auto nomem = [&]() {
        free_all(tmp);
        return fail(nullptr, EPROP_ENOMEM, "band layout allocation");
    };
    void *p;
    if (dalloc(o, &p, (size_t)(S + 1) * nb * 4) != cudaSuccess) return nomem();
    int *seg = static_cast<int *>(p);
    n.seg = seg;
    if (S > 0) eprop::launch_band_count(n.row_ptr, n.tgt_d, S, W, nb, seg);
    const int chunk = 1024;
    const int nch = std::max(1, (S + chunk - 1) / chunk);
    if (dalloc(tmp, &p, (size_t)nch * nb * 8) != cudaSuccess) return nomem();
    long long *part = static_cast<long long *>(p);
    if (S > 0) eprop::launch_band_chunk_sum(seg, S, nb, chunk, part);
    std::vector<long long> hp((size_t)nch * nb), tot(nb, 0);
    cudaError_t e = cudaMemcpy(hp.data(), part, hp.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        free_all(tmp);
        return cuda_fail(nullptr, e, "band layout counts");
    }
    for (int c = 0; c < nch; ++c)
        for (int b = 0; b < nb; ++b) {
            const long long v = hp[(size_t)c * nb + b];
            hp[(size_t)c * nb + b] = tot[b];
            tot[b] += v;
        }
    for (int b = 0; b < nb; ++b)
        if (tot[b] > (long long)INT32_MAX - eprop::kBandTile) {
            free_all(tmp);
            return fail(nullptr, EPROP_EINVAL, "trace_kernel 4: a band holds 2^31 synapses or more");
        }
    cudaMemcpy(part, hp.data(), hp.size() * 8, cudaMemcpyHostToDevice);
    if (S > 0) eprop::launch_band_chunk_scan(seg, S, nb, chunk, part);
    std::vector<int> last(nb);
    for (int b = 0; b < nb; ++b) last[b] = (int)tot[b];
    cudaMemcpy(seg + (size_t)S * nb, last.data(), (size_t)nb * 4, cudaMemcpyHostToDevice);
    std::vector<long long> t0(nb + 1, 0), base(nb + 1);
    for (int b = 0; b < nb; ++b) t0[b + 1] = t0[b] + (tot[b] + eprop::kBandTile - 1) / eprop::kBandTile;
    for (int b = 0; b <= nb; ++b) base[b] = t0[b] * eprop::kBandTile;
    n.n_tiles = t0[nb];
    n.nnz_b = n.n_tiles * eprop::kBandTile;
    if (dalloc(o, &p, (size_t)(nb + 1) * 8) != cudaSuccess) return nomem();
    cudaMemcpy(p, base.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice);
    n.band_base = static_cast<const long long *>(p);
    if (dalloc(tmp, &p, (size_t)(nb + 1) * 8) != cudaSuccess) return nomem();
    long long *tile0 = static_cast<long long *>(p);
    cudaMemcpy(tile0, t0.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice);
    if (dalloc(o, &p, (size_t)std::max(1LL, n.n_tiles) * sizeof(int4)) != cudaSuccess) return nomem();
    int4 *tiles = static_cast<int4 *>(p);
    n.tiles = tiles;
    if (dalloc(tmp, &p, 4) != cudaSuccess) return nomem();
    unsigned *flag = static_cast<unsigned *>(p);
    if (n.n_tiles > 0) eprop::launch_band_tiles(seg, tile0, S, nb, n.n_tiles, tiles, flag);
    if (dalloc(o, &p, (size_t)(n.nnz_b + 16) * 4) != cudaSuccess) return nomem();
    uint32_t *bd_td = static_cast<uint32_t *>(p);
    cudaMemset(bd_td, 0xFF, (size_t)(n.nnz_b + 16) * 4);
    n.bd_td = bd_td;
    if (dalloc(o, &p, (size_t)(n.nnz_b + 16) * 4) != cudaSuccess) return nomem();
    float *w_b = static_cast<float *>(p);
    if (S > 0 && n.nnz > 0) eprop::launch_band_scatter(n, n.w, bd_td, w_b);
    unsigned hflag = 0;
    e = cudaMemcpy(&hflag, flag, 4, cudaMemcpyDeviceToHost);
    free_all(tmp);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "band layout build");
    if (hflag)
        return fail(nullptr, EPROP_EINVAL,
                    "trace_kernel 4: a tile of a band spans 2^15 source rows or more (rows too sparse per band)");
    for (size_t q = 0; q < o.size(); ++q)
        if (o[q].p == n.w) {
            cudaFree(o[q].p);
            o.erase(o.begin() + (long long)q);
            break;
        }
    n.w = w_b;
    if (dalloc(o, &p, (size_t)std::max(1, S) * n.rr_stride) != cudaSuccess)
        return fail(nullptr, EPROP_ENOMEM, "band layout allocation");
    n.rrec = static_cast<unsigned char *>(p);
    return EPROP_OK;
}

extern "C" eprop_status eprop_create_network(const eprop_config *cfg, const eprop_synapses *syn,
                                             const float *w_out, const uint8_t *out_mask,
                                             const float *feedback, int32_t is_device,
                                             void *cuda_stream, eprop_net **out) {
    if (!out) return fail(nullptr, EPROP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg || !syn || !w_out) return fail(nullptr, EPROP_EINVAL, "cfg, syn and w_out are required");
    const eprop_config &c = *cfg;
    if (c.abi_version != EPROP_ABI_VERSION) return fail(nullptr, EPROP_EINVAL, "abi_version mismatch");
    if (c.n_in < 0 || c.n_rec < 1 || c.n_rec >= (1 << 24) || c.n_out < 1 || c.n_out > eprop::kMaxOut ||
        c.batch < 1 || c.batch >= (1 << 11))
        return fail(nullptr, EPROP_EINVAL, "sizes out of range (n_rec < 2^24, 1 <= n_out <= 1024, batch < 2048)");
    if (c.max_delay < 1 || c.max_delay > eprop::kMaxDelay) return fail(nullptr, EPROP_EINVAL, "max_delay must be 1..8");
    if (c.neuron_model < 0 || c.neuron_model > 1 || c.loss < 0 || c.loss > 2 || c.feedback < 0 ||
        c.feedback > 1 || c.trace_dtype < 0 || c.trace_dtype > 2 || c.t_ref < 0 || c.update_interval < 0)
        return fail(nullptr, EPROP_EINVAL, "invalid enum or negative parameter");
    if (c.batch > 1 && c.continuous)
        return fail(nullptr, EPROP_EINVAL, "batch > 1 needs continuous = 0 (every sample starts from zero state)");
    if (c.batch > eprop::kBatchWindowMax && c.update_interval > 0)
        return fail(nullptr, EPROP_EINVAL, "update windows inside a call need batch <= 64");
    if (c.d_out < 0 || c.d_out > 64 || c.d_ls < 0 || c.d_ls > 64)
        return fail(nullptr, EPROP_EINVAL, "d_out and d_ls must be 0..64");
    if ((c.d_out || c.d_ls) && (c.update_interval > 0 || c.continuous || c.launch_mode == 2))
        return fail(nullptr, EPROP_EINVAL,
                    "generalized delays need one update window per call (update_interval = 0, continuous = 0) "
                    "and launch_mode 0 or 1");
    if (c.launch_mode < 0 || c.launch_mode > 2)
        return fail(nullptr, EPROP_EINVAL, "launch_mode must be 0, 1 or 2");
    if (c.launch_mode == 2 && (c.continuous || c.update_interval > 0 || c.n_out > 256))
        return fail(nullptr, EPROP_EINVAL,
                    "launch_mode 2 (persistent step loop) needs one update window per call and n_out <= 256");
    if (c.trace_kernel < 0 || c.trace_kernel > 4 || c.blocks_per_sm < 0 || c.blocks_per_sm > 64)
        return fail(nullptr, EPROP_EINVAL, "trace_kernel must be 0..4 and blocks_per_sm 0..64");
    if (c.trace_kernel == 3 && !(c.continuous || c.update_interval > 0))
        return fail(nullptr, EPROP_EINVAL,
                    "trace_kernel 3 (dense window pass) advances carried state: it needs continuous or update_interval > 0");
    if (c.trace_kernel == 4 && (!(c.continuous || c.update_interval > 0) || c.batch != 1 || c.optimizer != 0 ||
                                (c.sign_mask & 3)))
        return fail(nullptr, EPROP_EINVAL,
                    "trace_kernel 4 (band-major dense window pass) needs carried state (continuous or "
                    "update_interval > 0), batch 1, optimizer 0 and free synapse signs");
    if (c.trace_kernel == 1 && c.batch > 1)
        return fail(nullptr, EPROP_EINVAL, "the lazy trace form (trace_kernel 1) needs batch = 1");
    if (c.trace_kernel == 2 && (c.continuous || c.update_interval > 0))
        return fail(nullptr, EPROP_EINVAL, "the batched trace kernel cannot carry state between windows");
    if (c.surrogate < 0 || c.surrogate > 1 || c.reset_mode < 0 || c.reset_mode > 1 || c.sign_mask < 0 ||
        c.sign_mask > 7 || c.optimizer < 0 || c.optimizer > 1 || c.if_period < 0)
        return fail(nullptr, EPROP_EINVAL, "invalid variant switch (surrogate, reset_mode, sign_mask, optimizer, if_period)");
    if (c.c_reg != 0.f && (!(c.beta_reg >= 0.f && c.beta_reg < 1.f) || c.continuous || c.update_interval > 0))
        return fail(nullptr, EPROP_EINVAL,
                    "rate regularisation needs 0 <= beta_reg < 1, continuous = 0 and update_interval = 0");
    if (c.optimizer == 1 && !(c.adam_b1 >= 0.f && c.adam_b1 < 1.f && c.adam_b2 >= 0.f && c.adam_b2 < 1.f &&
                              c.adam_eps > 0.f))
        return fail(nullptr, EPROP_EINVAL, "Adam needs 0 <= b1, b2 < 1 and eps > 0");
    if ((c.optimizer == 1 || (c.sign_mask & 3)) && c.trace_kernel == 1 && (c.continuous || c.update_interval > 0))
        return fail(nullptr, EPROP_EINVAL,
                    "Adam and fixed synapse signs need a trace form without lazy catch-up (not trace_kernel 1 with state)");
    if (c.n_drive_thr < 0 || c.n_drive_thr > EPROP_MAX_DRIVE_THR)
        return fail(nullptr, EPROP_EINVAL, "n_drive_thr out of range");
    for (int m = 1; m < c.n_drive_thr; ++m)
        if (c.drive_thr[m] < c.drive_thr[m - 1])
            return fail(nullptr, EPROP_EINVAL, "drive_thr must be non-decreasing");
    if (!(c.dt > 0.f) || !(c.tau_m > 0.f) || !(c.tau_out > 0.f) || (c.neuron_model == 1 && !(c.tau_a > 0.f)))
        return fail(nullptr, EPROP_EINVAL, "dt and time constants must be positive");
    if (syn->n_src != (int64_t)c.n_in + c.n_rec || syn->nnz < 0 || (syn->nnz > 0 && (!syn->row_ptr ||
        !syn->target || !syn->weight || !syn->delay)) || !syn->row_ptr)
        return fail(nullptr, EPROP_EINVAL, "synapse arrays inconsistent with n_in + n_rec");
    if (c.feedback == 1 && !feedback) return fail(nullptr, EPROP_EINVAL, "feedback = 1 needs a feedback matrix");

    eprop_net *net = new (std::nothrow) eprop_net();
    if (!net) return fail(nullptr, EPROP_ENOMEM, "host allocation failed");
    net->cfg = c;
    net->st = (cudaStream_t)cuda_stream;
    if (net->st == nullptr && c.launch_mode >= 1) {
        // graphs cannot be captured on the legacy default stream
        if (cudaStreamCreateWithFlags(&net->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete net;
            return fail(nullptr, EPROP_ECUDA, "cannot create a stream for graph capture");
        }
        net->own_stream = 1;
    }
    if (cudaStreamCreateWithFlags(&net->st2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&net->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&net->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        if (net->ev_fork) cudaEventDestroy(net->ev_fork);
        if (net->st2) cudaStreamDestroy(net->st2);
        if (net->own_stream) cudaStreamDestroy(net->st);
        delete net;
        return fail(nullptr, EPROP_ECUDA, "cannot create the readout stream");
    }
    Net &n = net->n;
    memset(&n, 0, sizeof(n));
    cudaGetDevice(&net->dev);
    cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, net->dev);
    const long long N = c.n_rec, K = c.n_out, B = c.batch, S = syn->n_src, nnz = syn->nnz;
    n.n_in = c.n_in; n.n_rec = c.n_rec; n.n_out = c.n_out; n.n_src = (int)S; n.B = c.batch;
    n.D = c.max_delay; n.nnz = nnz;
    n.alif = c.neuron_model == 1; n.t_ref = c.t_ref; n.loss = c.loss; n.feedback = c.feedback;
    n.has_state = (c.continuous || c.update_interval > 0) ? 1 : 0;
    n.d_out = c.d_out;
    n.d_ls = c.d_ls;
    n.trace_bf16 = c.trace_dtype != 0; n.trace_type = c.trace_dtype; n.record_grad = c.record_grad != 0;
    n.record_raster = c.record_raster != 0; n.record_psi = c.record_psi != 0; n.n_thr = c.drive_weight != 0.f ? c.n_drive_thr : 0;
    const double alpha = std::exp(-(double)c.dt / c.tau_m);
    const double kappa = std::exp(-(double)c.dt / c.tau_out);
    const double kappa_e = c.kappa_e < 0.f ? kappa : (double)c.kappa_e;
    n.alpha = (float)alpha; n.kappa = (float)kappa; n.kappa_e = (float)kappa_e;
    n.rho = n.alif ? (float)std::exp(-(double)c.dt / c.tau_a) : 0.f;
    n.alpha_lo = (float)(alpha - (double)n.alpha);
    n.kappa_e_lo = (float)(kappa_e - (double)n.kappa_e);
    n.kappa_lo = (float)(kappa - (double)n.kappa);
    n.rho_lo = n.alif ? (float)(std::exp(-(double)c.dt / c.tau_a) - (double)n.rho) : 0.f;
    n.beta_a = n.alif ? c.beta_a : 0.f;
    n.v_th = c.v_th; n.gamma = c.gamma; n.beta_sg = c.beta_sg; n.lr = c.lr;
    n.drive_weight = c.drive_weight; n.drive_seed = c.drive_seed;
    n.log2_alpha = (float)std::log2(alpha); n.log2_kappa = (float)std::log2(kappa);
    n.inv_B = (float)(1.0 / c.batch);
    n.surrogate = c.surrogate; n.reset_mode = c.reset_mode; n.v_reset = c.v_reset;
    n.c_reg = c.c_reg; n.f_target = c.f_target; n.beta_reg = c.beta_reg;
    n.sign_mask = c.sign_mask; n.adam = c.optimizer == 1;
    n.adam_b1 = c.adam_b1; n.adam_b2 = c.adam_b2; n.adam_eps = c.adam_eps;
    n.if_period = c.if_period; n.if_seed = c.if_seed;

    std::vector<DevAlloc> &o = net->fixed_allocs;
    void *p;
    eprop_status s;
#define FA(field, type, count)                                                        \
    do {                                                                              \
        cudaError_t _e = dalloc(o, &p, (size_t)(count) * sizeof(type));               \
        if (_e != cudaSuccess) { s = cuda_fail(nullptr, _e, "allocation"); goto fail_out; } \
        n.field = reinterpret_cast<decltype(n.field)>(p);                             \
    } while (0)
    {
        const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        // synapses
        long long *rp;
        FA(row_ptr, long long, S + 1);
        rp = const_cast<long long *>(n.row_ptr);
        if (cudaMemcpy(rp, syn->row_ptr, (S + 1) * sizeof(long long), kind) != cudaSuccess) {
            s = fail(nullptr, EPROP_EINVAL, "cannot read row_ptr");
            goto fail_out;
        }
        {
            std::vector<long long> hp(S + 1);
            cudaMemcpy(hp.data(), rp, (S + 1) * sizeof(long long), cudaMemcpyDeviceToHost);
            if (hp[0] != 0 || hp[S] != nnz) { s = fail(nullptr, EPROP_EINVAL, "row_ptr must run from 0 to nnz"); goto fail_out; }
            for (long long i = 0; i < S; ++i)
                if (hp[i + 1] < hp[i]) { s = fail(nullptr, EPROP_EINVAL, "row_ptr must be non-decreasing"); goto fail_out; }
            net->nnz_in = hp[c.n_in];
            n.nnz_in = hp[c.n_in];
            long long mx = 0;
            for (long long i = 0; i < S; ++i) mx = std::max(mx, hp[i + 1] - hp[i]);
            n.segs = (int)std::max(1LL, (mx + eprop::kSeg - 1) / eprop::kSeg);
        }
        uint32_t *td;
        FA(tgt_d, uint32_t, nnz + 16);
        td = const_cast<uint32_t *>(n.tgt_d);
        FA(w, float, nnz + 16);
        if (nnz > 0) {
            const int32_t *tg = syn->target;
            const uint8_t *dl = syn->delay;
            const float *wt = syn->weight;
            void *t_tg = nullptr, *t_dl = nullptr, *t_w = nullptr;
            std::vector<DevAlloc> tmp;
            if (!is_device) {
                if (dalloc(tmp, &t_tg, nnz * 4) != cudaSuccess || dalloc(tmp, &t_dl, nnz) != cudaSuccess ||
                    dalloc(tmp, &t_w, nnz * 4) != cudaSuccess) {
                    free_all(tmp);
                    s = fail(nullptr, EPROP_ENOMEM, "staging allocation failed");
                    goto fail_out;
                }
                cudaMemcpy(t_tg, tg, nnz * 4, cudaMemcpyHostToDevice);
                cudaMemcpy(t_dl, dl, nnz, cudaMemcpyHostToDevice);
                cudaMemcpy(t_w, wt, nnz * 4, cudaMemcpyHostToDevice);
                tg = (const int32_t *)t_tg; dl = (const uint8_t *)t_dl; wt = (const float *)t_w;
            }
            unsigned int *flag;
            cudaMalloc(&flag, 4);
            cudaMemset(flag, 0, 4);
            check_synapses_kernel<<<1024, 256>>>(tg, dl, nnz, c.n_rec, c.max_delay, flag);
            pack_synapses_kernel<<<1024, 256>>>(tg, dl, wt, nnz, td, n.w);
            unsigned int hflag = 0;
            cudaError_t e = cudaMemcpy(&hflag, flag, 4, cudaMemcpyDeviceToHost);
            cudaFree(flag);
            free_all(tmp);
            if (e != cudaSuccess) { s = cuda_fail(nullptr, e, "synapse packing"); goto fail_out; }
            if (hflag & 1u) { s = fail(nullptr, EPROP_EINVAL, "synapse target out of [0, n_rec)"); goto fail_out; }
            if (hflag & 2u) { s = fail(nullptr, EPROP_EINVAL, "synapse delay out of [1, max_delay]"); goto fail_out; }
        }
        if (c.trace_kernel == 4) {
            s = build_band(net);
            if (s != EPROP_OK) goto fail_out;
        }
        {
            // band-major records include the padding of whole tiles
            const long long nnz_t = n.band ? n.nnz_b : nnz;
            if (n.has_state) {              // one trace per sample and synapse ([B][nnz])
                FA(ebar, uint16_t, (B * nnz_t + 16) * (n.trace_bf16 ? 1 : 2));
                if (n.alif) FA(epsa, uint16_t, (B * nnz_t + 16) * (n.trace_bf16 ? 1 : 2));
            }
            if (n.record_grad) FA(grad, float, nnz_t + 16);
        }
        // neurons
        FA(v, float, B * N);
        FA(a, float, B * N);
        FA(v_lo, float, B * N);
        FA(a_lo, float, B * N);
        FA(ref, int, B * N);
        FA(z_prev, uint8_t, B * N);
        FA(ring, long long, B * (c.max_delay + 1) * N);
        FA(anchor_t, int, B * S);
        FA(anchor_z, float, B * S);
        eprop::launch_fill_int(n.anchor_t, B * S, eprop::kNoSpike, 0);
        // readout
        FA(w_out, float, N * K);
        cudaMemcpy(n.w_out, w_out, N * K * 4, kind);
        {
            uint8_t *m;
            FA(out_mask, uint8_t, N * K);
            m = const_cast<uint8_t *>(n.out_mask);
            if (out_mask) cudaMemcpy(m, out_mask, N * K, kind);
            else cudaMemset(m, 1, N * K);
        }
        if (c.feedback == 1) {
            float *f;
            FA(fb, float, N * K);
            f = const_cast<float *>(n.fb);
            cudaMemcpy(f, feedback, N * K * 4, kind);
        } else {
            n.fb = n.w_out;
        }
        if (n.record_grad) FA(grad_out, float, N * K);
        FA(y, float, B * K);
        FA(y_acc, long long, B * K);
        FA(Cwin, float, B * K);
        FA(zk, float, 2 * B * N);
        FA(loss_acc, float, B);
        FA(ro_done, int, B);
        if (c.c_reg != 0.f) FA(rate, float, B * N);
        if (n.adam) {
            FA(gwin, float, nnz + 16);
            FA(adam_m, float, nnz + 16);
            FA(adam_v, float, nnz + 16);
            FA(gwin_out, float, N * K);
            FA(adam_m_out, float, N * K);
            FA(adam_v_out, float, N * K);
        }
        if (c.launch_mode == 2) {
            if (dalloc(o, &p, sizeof(eprop::GridBar)) != cudaSuccess) { s = fail(nullptr, EPROP_ENOMEM, "allocation"); goto fail_out; }
            net->gridbar = static_cast<eprop::GridBar *>(p);
            net->pers_blocks = eprop::persistent_blocks(net->sm_count);
            if (net->pers_blocks < 1) { s = fail(nullptr, EPROP_ECUDA, "persistent step loop cannot be resident"); goto fail_out; }
        }
        FA(events, unsigned long long, 1);
        FA(err_flags, unsigned int, 1);
        FA(clock, eprop::Clock, 1);
        {
            uint32_t *thr;
            FA(drive_thr, uint32_t, EPROP_MAX_DRIVE_THR);
            thr = const_cast<uint32_t *>(n.drive_thr);
            cudaMemcpy(thr, c.drive_thr, sizeof(c.drive_thr), cudaMemcpyHostToDevice);
        }
        eprop::prepare_kernel_attributes();
        eprop::prepare_step_kernel_attributes();
        eprop::prepare_learning_signal_attributes();
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { s = cuda_fail(nullptr, e, "network set-up"); goto fail_out; }
        if (c.update_interval > 0) {
            s = alloc_window(net, c.update_interval, c.update_interval);
            if (s != EPROP_OK) { g_create_err = net->err; goto fail_out; }
        }
    }
#undef FA
    *out = net;
    return EPROP_OK;
fail_out:
    free_all(net->fixed_allocs);
    free_all(net->win_allocs);
    cudaEventDestroy(net->ev_fork);
    cudaEventDestroy(net->ev_join);
    cudaStreamDestroy(net->st2);
    if (net->own_stream) cudaStreamDestroy(net->st);
    delete net;
    return s;
}

extern "C" eprop_status eprop_set_inputs_targets(eprop_net *net, const int64_t *in_step_ptr,
                                                 const int32_t *in_ids, int64_t n_in_ids,
                                                 const float *targets, const uint8_t *window,
                                                 const int32_t *lengths, int32_t T, int32_t is_device) {
    if (!net) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    const eprop_config &c = net->cfg;
    Net &n = net->n;
    if (T < 1 || !in_step_ptr || !targets || n_in_ids < 0 || (n_in_ids > 0 && !in_ids))
        return fail(net, EPROP_EINVAL, "T >= 1, in_step_ptr and targets are required");
    if (c.update_interval > 0 && T % c.update_interval)
        return fail(net, EPROP_EINVAL, "T must be a multiple of update_interval");
    if (c.continuous && c.update_interval == 0 && net->U_fixed && T != net->U_fixed)
        return fail(net, EPROP_EINVAL, "continuous networks with update_interval 0 keep the first T");
    const long long B = c.batch, K = c.n_out, N = c.n_rec;
    const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // host-side validation
    if (!is_device) {
        if (in_step_ptr[0] != 0 || in_step_ptr[B * T] != n_in_ids)
            return fail(net, EPROP_EINVAL, "in_step_ptr must run from 0 to n_in_ids");
        long long mx = 0;
        for (long long q = 0; q < B * T; ++q) {
            const long long d = in_step_ptr[q + 1] - in_step_ptr[q];
            if (d < 0) return fail(net, EPROP_EINVAL, "in_step_ptr must be non-decreasing");
            if (d > mx) mx = d;
        }
        for (long long q = 0; q < n_in_ids; ++q)
            if (in_ids[q] < 0 || in_ids[q] >= c.n_in) return fail(net, EPROP_EINVAL, "input id out of [0, n_in)");
        if (lengths)
            for (long long b = 0; b < B; ++b)
                if (lengths[b] < 1 || lengths[b] > T) return fail(net, EPROP_EINVAL, "lengths must be in [1, T]");
        net->max_in_per_step = mx;
    } else {
        net->max_in_per_step = 1 << 14;
    }
    // (re)allocate per-T buffers
    if (net->in_allocs.empty() || T != net->T_in || n_in_ids > net->x_cap) {
        cudaStreamSynchronize(net->st);
        free_all(net->in_allocs);
        if (net->gexec) {
            cudaGraphExecDestroy(net->gexec);
            net->gexec = nullptr;
            net->g_T = -1;
        }
        void *p;
        std::vector<DevAlloc> &o = net->in_allocs;
#define IA(field, type, count)                                                     \
        do {                                                                       \
            cudaError_t _e = dalloc(o, &p, (size_t)(count) * sizeof(type));        \
            if (_e != cudaSuccess) return cuda_fail(net, _e, "input allocation");  \
            n.field = reinterpret_cast<decltype(n.field)>(p);                      \
        } while (0)
        const long long cap = n_in_ids > 0 ? n_in_ids : 1;
        IA(x_ptr, long long, B * T + 1);
        IA(x_ids, int, cap);
        IA(targets, float, B * T * K);
        IA(window, uint8_t, B * T);
        IA(lengths, int, B);
        IA(y_rec, float, B * T * K);
        if (n.record_raster) IA(rec_raster, uint32_t, B * ((T + 31) / 32) * N);
        if (n.record_psi) IA(rec_psi, float, B * T * N);
        if (net->pred && (n.pred_mode & 2)) IA(pred_rec, float, B * T * n.pred_in);
#undef IA
        net->x_cap = cap;
    }
    n.T = T;
    cudaStream_t st = net->st;
    CK(net, cudaMemcpyAsync(const_cast<long long *>(n.x_ptr), in_step_ptr, (B * T + 1) * 8, kind, st));
    if (n_in_ids > 0) CK(net, cudaMemcpyAsync(const_cast<int *>(n.x_ids), in_ids, n_in_ids * 4, kind, st));
    CK(net, cudaMemcpyAsync(const_cast<float *>(n.targets), targets, B * T * K * 4, kind, st));
    if (window) CK(net, cudaMemcpyAsync(const_cast<uint8_t *>(n.window), window, B * T, kind, st));
    else CK(net, cudaMemsetAsync(const_cast<uint8_t *>(n.window), 1, B * T, st));
    if (lengths) {
        CK(net, cudaMemcpyAsync(const_cast<int *>(n.lengths), lengths, B * 4, kind, st));
    } else {
        std::vector<int> l(B, T);
        CK(net, cudaMemcpyAsync(const_cast<int *>(n.lengths), l.data(), B * 4, cudaMemcpyHostToDevice, st));
        CK(net, cudaStreamSynchronize(st));
    }
    if (is_device) {
        unsigned int *flag;
        CK(net, cudaMalloc(&flag, 4));
        cudaMemsetAsync(flag, 0, 4, st);
        check_inputs_kernel<<<256, 256, 0, st>>>(n.x_ptr, B * T + 1, n.x_ids, n_in_ids, n.lengths, (int)B, T,
                                                 c.n_in, flag);
        unsigned int h = 0;
        cudaMemcpyAsync(&h, flag, 4, cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        cudaFree(flag);
        if (e != cudaSuccess) return cuda_fail(net, e, "input validation");
        if (h & 1u) return fail(net, EPROP_EINVAL, "input id out of [0, n_in)");
        if (h & 2u) return fail(net, EPROP_EINVAL, "in_step_ptr must be non-decreasing from 0 to n_in_ids");
        if (h & 4u) return fail(net, EPROP_EINVAL, "lengths must be in [1, T]");
    }
    const int U = c.update_interval > 0 ? c.update_interval : T;
    eprop_status s = alloc_window(net, U, T);
    if (s != EPROP_OK) return s;
    net->T_in = T;
    net->have_inputs = 1;
    net->have_sim = 0;                  // the recorded outputs no longer match these inputs
    return EPROP_OK;
}

// ------------------------------------------------------------ simulate

static void issue_call(eprop_net *net, int T, const uint8_t *forced) {
    Net n = net->n;
    const eprop_config &c = net->cfg;
    cudaStream_t st = net->st;
    n.T = T;
    n.forced = forced;
    const long long B = c.batch, N = c.n_rec, K = c.n_out, S = n.n_src;
    const int U = n.U;
    if (!c.continuous) {
        cudaMemsetAsync(n.v, 0, B * N * 4, st);
        cudaMemsetAsync(n.a, 0, B * N * 4, st);
        cudaMemsetAsync(n.v_lo, 0, B * N * 4, st);
        cudaMemsetAsync(n.a_lo, 0, B * N * 4, st);
        cudaMemsetAsync(n.ref, 0, B * N * 4, st);
        cudaMemsetAsync(n.z_prev, 0, B * N, st);
        cudaMemsetAsync(n.ring, 0, B * (n.D + 1) * N * 8, st);
        cudaMemsetAsync(n.bits, 0, B * S * n.RW * 4, st);
        cudaMemsetAsync(n.list_cnt, 0, B * n.RS * eprop::kBkt * 4, st);
        cudaMemsetAsync(n.y, 0, B * K * 4, st);
        cudaMemsetAsync(n.y_acc, 0, B * K * 8, st);
        cudaMemsetAsync(n.zk, 0, 2 * B * N * 4, st);
        cudaMemsetAsync(n.psi_hist, 0, B * (U + 1) * N * 4, st);
        cudaMemsetAsync(n.anchor_z, 0, B * S * 4, st);
        if (n.rate) cudaMemsetAsync(n.rate, 0, B * N * 4, st);
        eprop::launch_fill_int(n.anchor_t, B * S, eprop::kNoSpike, st);
        if (n.has_state) {
            const size_t tb = n.trace_bf16 ? 2 : 4;
            const long long nt = n.band ? n.nnz_b : n.nnz;
            cudaMemsetAsync(n.ebar, 0, B * nt * tb, st);
            if (n.alif) cudaMemsetAsync(n.epsa, 0, B * nt * tb, st);
        }
    }
    if (n.record_raster) cudaMemsetAsync(n.rec_raster, 0, B * ((T + 31) / 32) * N * 4, st);
    if (n.pred_mode && !c.continuous) {
        cudaMemsetAsync(n.pop_rate, 0, B * eprop::kPopGroups * 4, st);
        cudaMemsetAsync(n.pop_cnt, 0, B * eprop::kPopGroups * 4, st);
    }
    long long L = 0, LT = 0, nwin = 0;
    if (!c.continuous) L += 1;                       // anchor fill
    eprop::launch_begin_call(n, c.continuous, st);
    L += 1;
    // the delivery and trace kernels hold two 256-thread blocks per SM (launch
    // bounds); their work queues are drained by whichever blocks are resident
    const int grid_rows = (c.blocks_per_sm > 0 ? c.blocks_per_sm : 2) * net->sm_count;
    // delivery without carried state holds four blocks per SM; with several
    // samples the grid's x dimension is shared among them (each sample's
    // step has a few spiking rows, not enough for a full grid of its own)
    int deliver_rows = (c.blocks_per_sm > 0 ? c.blocks_per_sm : (n.has_state && !n.dense ? 2 : 4)) *
                       net->sm_count;
    if (B > 1) deliver_rows = std::max(1, (int)((deliver_rows + B - 1) / B));
    // window pass: two blocks per SM by default (a third fits, but the
    // smaller L1 that leaves for the table lookups measured slower)
    const int pass_rows = (c.blocks_per_sm > 0 ? c.blocks_per_sm : 2) * net->sm_count;
    const int idle_rows = (c.blocks_per_sm > 0 ? c.blocks_per_sm : 3) * net->sm_count;
    const int nw = T / U;
    if (c.profile && (int)net->ev.size() < 2 * nw) {
        for (int q = (int)net->ev.size(); q < 2 * nw; ++q) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            net->ev.push_back(e);
        }
    }
    // Readout work (the per-step readout sum and error, the window's readout
    // weight update) reads the step's spike list and W_out and feeds only the
    // window-end kernels, so it runs on the second stream beside delivery and
    // the next neuron updates; the weight update is forked after the tables
    // kernel, which reads W_out as the feedback matrix when B is symmetric,
    // and overlaps the window pass.  Joins: before the error filter and tables
    // of a window (they read its errors), before the rollover (it clears the
    // spike bits the weight update reads), and at the end of the call.  With
    // a predictor attached everything stays on one stream (the prediction
    // feeds the step's learning signal), and so it does when the spike-list
    // ring is not longer than the update window (batched form, RS = 2).
    // Otherwise a readout trails the neuron updates by fewer than U steps
    // (the joins at window ends), and the ring's RS > U slots keep its
    // step's list until it has run (with a readout delay d_out it reads the
    // list of the step d_out back, and RS >= d_out + 2 keeps that one too).
    // (the persistent step loop does the readout itself: one stream)
    const bool fork = n.pred_mode == 0 && n.RS > n.U && c.launch_mode != 2;
    cudaStream_t sr = fork ? net->st2 : st;
    auto fork_readout = [&]() {
        if (!fork) return;
        cudaEventRecord(net->ev_fork, st);
        cudaStreamWaitEvent(net->st2, net->ev_fork, 0);
    };
    auto join_readout = [&]() {
        if (!fork) return;
        cudaEventRecord(net->ev_join, net->st2);
        cudaStreamWaitEvent(st, net->ev_join, 0);
    };
    const bool persistent = c.launch_mode == 2;
    if (persistent) {
        // form (2): every step of the call in one cooperative launch
        cudaError_t le = eprop::launch_persistent_steps(n, T, net->gridbar, net->pers_blocks, st);
        if (le != cudaSuccess && net->launch_err == cudaSuccess) net->launch_err = le;
        L += 1;
    }
    for (int i = 1; i <= T; ++i) {
        if (persistent) {
            if (i % U != 0) continue;
        } else {
        if (c.n_in > 0) { eprop::launch_inject(n, i, (int)net->max_in_per_step, st); L += 1; }
        eprop::launch_neuron(n, i, net->sm_count, st);
        fork_readout();
        eprop::launch_readout(n, i, net->sm_count, sr);
        if (n.pred_mode) {
            eprop::launch_pred_input(n, i, st);
            L += 1;
            if (n.pred_mode & 1) {
                n.pred_y = predictor_issue_forward(net->pred, n.pred_x, (int)B, st);
                eprop::launch_pred_apply(n, i, st);
                L += 5;
            }
        }
        if (n.band) eprop::launch_deliver_band(n, i, deliver_rows, st);
        else eprop::launch_deliver(n, i, deliver_rows, st);
        L += 3;
        }
        if (i % U == 0) {
            join_readout();
            eprop::launch_filter_error(n, i, st);
            // L[b][u][j] = sum_k B[j][k] E[b][u][k] of the whole window
            // (Eq. final-gradient), tensor cores with split TF32 operands
            eprop::launch_learning_signals(n.fb, n.E_win, n.L_win, c.n_rec, U, c.n_out, (int)B, n.err_flags, st);
            eprop::launch_tables(n, i, st);
            // after the tables: with symmetric feedback B is W_out itself
            fork_readout();
            eprop::launch_readout_weights(n, i, sr);
            L += 4;
            if (c.profile) cudaEventRecordWithFlags(net->ev[2 * nwin], st, cudaEventRecordExternal);
            if (net->trace_mode == 1) {
                eprop::launch_trace_batched(n, net->sm_count, st);
                LT += 1;
            } else if (net->trace_mode == 2 && B > 1) {
                eprop::launch_window_batched(n, i, net->sm_count, st);
                LT += 1;
            } else if (net->trace_mode == 2) {
                eprop::launch_window_pass(n, i, pass_rows, idle_rows, st);
                LT += 3;
            } else if (net->trace_mode == 3) {
                eprop::launch_window_band(n, i, net->sm_count, st);
                LT += 2;
            } else {
                eprop::launch_trace_window(n, i, grid_rows, st);
                LT += 2;
            }
            if (c.profile) cudaEventRecordWithFlags(net->ev[2 * nwin + 1], st, cudaEventRecordExternal);
            join_readout();
            if (n.adam) {                // after the readout gradient has landed
                eprop::launch_adam(n, net->sm_count, st);
                L += 2;
            }
            if (i < T || n.has_state) { eprop::launch_rollover(n, i, st); L += 1; }
            nwin += 1;
        }
    }
    join_readout();
    if (!c.continuous && n.has_state && !n.dense) {
        eprop::launch_flush(n, T, nullptr, nullptr, 0, n.nnz, 1, net->sm_count, st);
        L += 1;
    }
    eprop::launch_end_call(n, T, st);
    L += 1;
    net->launches = L + LT;
    net->trace_launches = LT;
    net->windows = nwin;
}

extern "C" eprop_status eprop_simulate(eprop_net *net, int32_t T, const uint8_t *forced_raster) {
    if (!net) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    const eprop_config &c = net->cfg;
    if (!net->have_inputs) return fail(net, EPROP_ESTATE, "eprop_set_inputs_targets must come first");
    if (T != net->T_in) return fail(net, EPROP_EINVAL, "T differs from the T of the inputs");
    if (c.continuous && c.update_interval == 0) {
        if (net->U_fixed == 0) net->U_fixed = T;
        else if (T != net->U_fixed) return fail(net, EPROP_EINVAL, "continuous network: T must stay fixed");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(net, e, "pending error before simulate");
    const bool use_graph = c.launch_mode >= 1 && forced_raster == nullptr;
    net->launch_err = cudaSuccess;
    if (use_graph) {
        if (!net->gexec || net->g_T != T) {
            if (net->gexec) {
                cudaGraphExecDestroy(net->gexec);
                net->gexec = nullptr;
            }
            cudaGraph_t g;
            CK(net, cudaStreamBeginCapture(net->st, cudaStreamCaptureModeThreadLocal));
            issue_call(net, T, nullptr);
            CK(net, cudaStreamEndCapture(net->st, &g));
            if (net->launch_err != cudaSuccess) {
                cudaGraphDestroy(g);
                return cuda_fail(net, net->launch_err, "persistent step loop capture");
            }
            e = cudaGraphInstantiate(&net->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(net, e, "cudaGraphInstantiate");
            net->g_T = T;
        }
        CK(net, cudaGraphLaunch(net->gexec, net->st));
    } else {
        issue_call(net, T, forced_raster);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(net, e, "kernel launch");
    if (net->launch_err != cudaSuccess) return cuda_fail(net, net->launch_err, "persistent step loop launch");
    net->t_abs += T;
    net->r_base = c.continuous ? net->r_base + T : T;
    net->have_sim = 1;
    return EPROP_OK;
}

// -------------------------------------------------------------- readback

static eprop_status ensure_tmp(eprop_net *net, long long count) {
    if (net->tmp_w) return EPROP_OK;
    void *p;
    if (dalloc(net->fixed_allocs, &p, count * 4) != cudaSuccess) return fail(net, EPROP_ENOMEM, "tmp alloc");
    net->tmp_w = (float *)p;
    if (dalloc(net->fixed_allocs, &p, count * 4) != cudaSuccess) return fail(net, EPROP_ENOMEM, "tmp alloc");
    net->tmp_g = (float *)p;
    return EPROP_OK;
}

extern "C" eprop_status eprop_read_weights_grads(eprop_net *net, int32_t proj, float *w, float *grad,
                                                 int32_t is_device) {
    if (!net) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    Net &n = net->n;
    const eprop_config &c = net->cfg;
    if (grad && !n.record_grad) return fail(net, EPROP_EINVAL, "gradients need record_grad = 1");
    const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t st = net->st;
    if (proj == 2) {
        const long long cnt = (long long)c.n_rec * c.n_out;
        if (w) CK(net, cudaMemcpyAsync(w, n.w_out, cnt * 4, kind, st));
        if (grad) CK(net, cudaMemcpyAsync(grad, n.grad_out, cnt * 4, kind, st));
        CK(net, cudaStreamSynchronize(st));
        return EPROP_OK;
    }
    if (proj != 0 && proj != 1) return fail(net, EPROP_EINVAL, "proj must be 0, 1 or 2");
    const long long q0 = proj == 0 ? 0 : net->nnz_in;
    const long long q1 = proj == 0 ? net->nnz_in : n.nnz;
    const long long cnt = q1 - q0;
    if (cnt == 0) return EPROP_OK;
    if (n.band) {
        eprop_status s = ensure_tmp(net, n.nnz);
        if (s != EPROP_OK) return s;
        const int r0 = proj == 0 ? 0 : c.n_in, r1 = proj == 0 ? c.n_in : c.n_in + c.n_rec;
        eprop::launch_band_gather(n, r0, r1, q0, w ? net->tmp_w : nullptr, grad ? net->tmp_g : nullptr, st);
        CK(net, cudaGetLastError());
        if (w) CK(net, cudaMemcpyAsync(w, net->tmp_w, cnt * 4, kind, st));
        if (grad) CK(net, cudaMemcpyAsync(grad, net->tmp_g, cnt * 4, kind, st));
    } else if (n.has_state && !n.dense && c.continuous && net->r_base > 0 && net->U_alloc > 0) {
        eprop_status s = ensure_tmp(net, n.nnz);
        if (s != EPROP_OK) return s;
        eprop::launch_flush(n, 0, net->tmp_w, net->tmp_g, q0, q1, 0, net->sm_count, st);
        if (w) CK(net, cudaMemcpyAsync(w, net->tmp_w, cnt * 4, kind, st));
        if (grad) CK(net, cudaMemcpyAsync(grad, net->tmp_g, cnt * 4, kind, st));
    } else {
        if (w) CK(net, cudaMemcpyAsync(w, n.w + q0, cnt * 4, kind, st));
        if (grad) CK(net, cudaMemcpyAsync(grad, n.grad + q0, cnt * 4, kind, st));
    }
    CK(net, cudaStreamSynchronize(st));
    return EPROP_OK;
}

extern "C" eprop_status eprop_readout(eprop_net *net, float *y, float *loss_per_sample, uint8_t *raster,
                                      int32_t is_device) {
    if (!net) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    if (!net->have_sim) return fail(net, EPROP_ESTATE, "no simulate call since the last set_inputs");
    Net &n = net->n;
    const eprop_config &c = net->cfg;
    const long long B = c.batch, T = net->T_in, K = c.n_out, N = c.n_rec;
    const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t st = net->st;
    if (y) CK(net, cudaMemcpyAsync(y, n.y_rec, B * T * K * 4, kind, st));
    if (loss_per_sample) CK(net, cudaMemcpyAsync(loss_per_sample, n.loss_acc, B * 4, kind, st));
    if (raster) {
        if (!n.record_raster) return fail(net, EPROP_EINVAL, "raster needs record_raster = 1");
        const long long bytes = B * T * N;
        if (net->tmp_raster_bytes < bytes) {
            void *p;
            if (dalloc(net->fixed_allocs, &p, bytes) != cudaSuccess) return fail(net, EPROP_ENOMEM, "raster alloc");
            net->tmp_raster = (unsigned char *)p;
            net->tmp_raster_bytes = bytes;
        }
        Net nn = n;
        nn.T = (int)T;
        eprop::launch_unpack_raster(nn, net->tmp_raster, st);
        CK(net, cudaMemcpyAsync(raster, net->tmp_raster, bytes, kind, st));
    }
    CK(net, cudaStreamSynchronize(st));
    return EPROP_OK;
}

// ---- autotuner of the launch shapes

static void invalidate_graph(eprop_net *net) {
    if (net->gexec) {
        cudaGraphExecDestroy(net->gexec);
        net->gexec = nullptr;
        net->g_T = -1;
    }
}

static long long alloc_bytes(const std::vector<DevAlloc> &v) {
    long long b = 0;
    for (const DevAlloc &a : v) b += (long long)a.bytes;
    return b;
}

// copies every allocation of v to (dir 0) or from (dir 1) scratch + offset
static cudaError_t copy_allocs(const std::vector<DevAlloc> &v, unsigned char *scratch, long long &off, int dir,
                               cudaStream_t st) {
    for (const DevAlloc &a : v) {
        cudaError_t e = dir == 0 ? cudaMemcpyAsync(scratch + off, a.p, a.bytes, cudaMemcpyDeviceToDevice, st)
                                 : cudaMemcpyAsync(a.p, scratch + off, a.bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        off += (long long)a.bytes;
    }
    return cudaSuccess;
}

static bool same_layout(const std::vector<DevAlloc> &a, const std::vector<size_t> &sizes) {
    if (a.size() != sizes.size()) return false;
    for (size_t q = 0; q < a.size(); ++q)
        if (a[q].bytes != sizes[q]) return false;
    return true;
}

extern "C" eprop_status eprop_autotune(eprop_net *net, eprop_tune_result *out) {
    if (!net || !out) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    if (!net->have_inputs) return fail(net, EPROP_ESTATE, "eprop_set_inputs_targets must come first");
    eprop_config &c = net->cfg;
    const int T = net->T_in;
    const int U = c.update_interval > 0 ? c.update_interval : T;
    const bool pristine = net->t_abs == 0;
    const int tk0 = c.trace_kernel, bps0 = c.blocks_per_sm;
    // candidates: the trace form (only before the first call, while the
    // carried state is still zero) and the CTAs per SM of the row kernels
    std::vector<int> tks;
    if (pristine && c.batch == 1 && net->n.has_state && !net->n.adam && !(c.sign_mask & 3) && !net->n.band)
        tks = {3, 1};
    else tks = {tk0};
    const int bps_list[4] = {1, 2, 3, 4};
    std::memset(out, 0, sizeof(*out));
    CK(net, cudaStreamSynchronize(net->st));
    // snapshot of every device allocation and of the host-side clock
    const long long bytes = alloc_bytes(net->fixed_allocs) + alloc_bytes(net->win_allocs) +
                            alloc_bytes(net->in_allocs);
    void *sp = nullptr;
    cudaError_t e = cudaMalloc(&sp, (size_t)bytes);
    if (e != cudaSuccess) return cuda_fail(net, e, "autotune snapshot");
    unsigned char *scratch = static_cast<unsigned char *>(sp);
    std::vector<size_t> win_sizes;
    for (const DevAlloc &a : net->win_allocs) win_sizes.push_back(a.bytes);
    const long long h_t_abs = net->t_abs;
    const int h_r_base = net->r_base, h_U_fixed = net->U_fixed;
    long long off = 0;
    e = copy_allocs(net->fixed_allocs, scratch, off, 0, net->st);
    if (e == cudaSuccess) e = copy_allocs(net->in_allocs, scratch, off, 0, net->st);
    const long long win_off0 = off;
    if (e == cudaSuccess) e = copy_allocs(net->win_allocs, scratch, off, 0, net->st);
    auto restore = [&]() -> cudaError_t {
        long long o = 0;
        cudaError_t r = copy_allocs(net->fixed_allocs, scratch, o, 1, net->st);
        if (r == cudaSuccess) r = copy_allocs(net->in_allocs, scratch, o, 1, net->st);
        if (r == cudaSuccess && same_layout(net->win_allocs, win_sizes)) {
            o = win_off0;
            r = copy_allocs(net->win_allocs, scratch, o, 1, net->st);
        } else {
            // another trace form's layout: the form only changes before the
            // first call, when the window buffers still hold their initial
            // zeros, so that is the state to put back
            for (const DevAlloc &a : net->win_allocs) {
                if (r != cudaSuccess) break;
                r = cudaMemsetAsync(a.p, 0, a.bytes, net->st);
            }
        }
        net->t_abs = h_t_abs;
        net->r_base = h_r_base;
        net->U_fixed = h_U_fixed;
        return r == cudaSuccess ? cudaStreamSynchronize(net->st) : r;
    };
    auto set_shape = [&](int tk, int bps) -> eprop_status {
        c.blocks_per_sm = bps;
        if (tk != c.trace_kernel) {
            c.trace_kernel = tk;
            net->U_alloc = 0;                  // the trace form decides the window layout
            eprop_status st = alloc_window(net, U, T);
            if (st != EPROP_OK) return st;
        }
        invalidate_graph(net);
        return EPROP_OK;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    eprop_status status = e == cudaSuccess ? EPROP_OK : cuda_fail(net, e, "autotune setup");
    double best = 1e300;
    int best_tk = tk0, best_bps = bps0;
    for (size_t a = 0; a < tks.size() && status == EPROP_OK; ++a) {
        for (int q = 0; q < 4 && status == EPROP_OK; ++q) {
            const int tk = tks[a], bps = bps_list[q];
            status = set_shape(tk, bps);
            if (status != EPROP_OK) break;
            status = eprop_simulate(net, T, nullptr);      // warm-up (graph capture)
            if (status != EPROP_OK) break;
            if ((e = restore()) != cudaSuccess) { status = cuda_fail(net, e, "autotune restore"); break; }
            cudaEventRecord(e0, net->st);
            status = eprop_simulate(net, T, nullptr);
            if (status != EPROP_OK) break;
            cudaEventRecord(e1, net->st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { status = cuda_fail(net, e, "autotune"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const int k = out->n_candidates;
            if (k < EPROP_TUNE_MAX) {
                out->cand_trace_kernel[k] = tk;
                out->cand_blocks_per_sm[k] = bps;
                out->cand_ms[k] = ms;
                out->n_candidates = k + 1;
            }
            if (ms < best) {
                best = ms;
                best_tk = tk;
                best_bps = bps;
            }
            if ((e = restore()) != cudaSuccess) { status = cuda_fail(net, e, "autotune restore"); break; }
        }
    }
    if (status == EPROP_OK) status = set_shape(best_tk, best_bps);
    if (status == EPROP_OK && (e = restore()) != cudaSuccess) status = cuda_fail(net, e, "autotune restore");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sp);
    out->trace_kernel = c.trace_kernel;
    out->blocks_per_sm = c.blocks_per_sm;
    return status;
}

// ---- learned learning-signal predictor

extern "C" eprop_status eprop_attach_predictor(eprop_net *net, eprop_predictor *pred, int32_t mode) {
    if (!net) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    Net &n = net->n;
    const eprop_config &c = net->cfg;
    if (mode < 0 || mode > 3) return fail(net, EPROP_EINVAL, "mode must be 0..3");
    if (mode != 0 && !pred) return fail(net, EPROP_EINVAL, "a predictor is required");
    if (mode != 0 && c.launch_mode == 2)
        return fail(net, EPROP_EINVAL, "the persistent step loop (launch_mode 2) runs without a predictor");
    CK(net, cudaStreamSynchronize(net->st));
    if (net->gexec) {                       // the captured call changes
        cudaGraphExecDestroy(net->gexec);
        net->gexec = nullptr;
        net->g_T = -1;
    }
    if (mode == 0) {
        net->pred = nullptr;
        n.pred_mode = 0;
        n.pop_cnt = nullptr;
        return EPROP_OK;
    }
    int pin = 0, pout = 0, prows = 0;
    predictor_dims(pred, &pin, &pout, &prows);
    if (pout != c.n_out || pin != c.n_out + eprop::kPopGroups)
        return fail(net, EPROP_EINVAL, "predictor must map n_out + 64 inputs to n_out outputs");
    if (prows < c.batch) return fail(net, EPROP_EINVAL, "predictor max_rows must be >= batch");
    const long long B = c.batch, G = eprop::kPopGroups;
    void *p;
    std::vector<DevAlloc> &o = net->fixed_allocs;
    if (!n.pop_rate) {
        if (dalloc(o, &p, B * G * 4) != cudaSuccess) return fail(net, EPROP_ENOMEM, "predictor buffers");
        n.pop_rate = (float *)p;
        if (dalloc(o, &p, B * G * 4) != cudaSuccess) return fail(net, EPROP_ENOMEM, "predictor buffers");
        net->pop_cnt_buf = (int *)p;
        if (dalloc(o, &p, B * pin * 4) != cudaSuccess) return fail(net, EPROP_ENOMEM, "predictor buffers");
        n.pred_x = (float *)p;
        std::vector<float> inv(G, 0.f);
        for (int g = 0; g < G; ++g) {
            const int size = c.n_rec > g ? (c.n_rec - g + (int)G - 1) / (int)G : 0;
            inv[g] = size > 0 ? 1.0f / (float)size : 0.f;
        }
        if (dalloc(o, &p, G * 4) != cudaSuccess) return fail(net, EPROP_ENOMEM, "predictor buffers");
        CK(net, cudaMemcpy(p, inv.data(), G * 4, cudaMemcpyHostToDevice));
        n.pop_inv = (const float *)p;
    }
    n.pop_cnt = net->pop_cnt_buf;
    n.pred_in = pin;
    n.pop_beta = (float)std::exp(-(double)c.dt / 20.0);
    net->pred = pred;
    n.pred_mode = mode;
    if ((mode & 2) && net->have_inputs) {
        if (dalloc(net->in_allocs, &p, B * (long long)net->T_in * pin * 4) != cudaSuccess)
            return fail(net, EPROP_ENOMEM, "predictor record buffer");
        n.pred_rec = (float *)p;
    }
    return EPROP_OK;
}

extern "C" eprop_status eprop_read_predictor_inputs(eprop_net *net, float *x, int32_t is_device) {
    if (!net || !x) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    if (!(net->n.pred_mode & 2) || !net->n.pred_rec)
        return fail(net, EPROP_EINVAL, "recording needs a predictor attached with mode bit 1");
    if (!net->have_sim) return fail(net, EPROP_ESTATE, "no simulate call since the last set_inputs");
    const long long cnt = (long long)net->cfg.batch * net->T_in * net->n.pred_in;
    CK(net, cudaMemcpyAsync(x, net->n.pred_rec, cnt * 4,
                            is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, net->st));
    CK(net, cudaStreamSynchronize(net->st));
    return EPROP_OK;
}

// ---- raster readout through a fixed device scratch (no allocation)
//
// eprop_readout unpacks the recorded raster into a device buffer that it
// allocates on first use.  Some callers cannot allocate at that point: a
// monitor reading rasters beside a simulation that holds the device's
// memory at its limit, or a loop that must not trigger the device-wide
// synchronisation a first cudaMalloc can cause.  This variant unpacks into
// a scratch array that is part of the module image (file-scope, 256-byte
// aligned, EPROP_STATIC_RASTER_BYTES), so it allocates no device memory.
// Every byte of the unpacked range is written before it is copied out, so
// nothing in the scratch has to start at zero.  One scratch serves every
// network of the process on a device: calls that overlap in time (two host
// threads, or two streams whose copies have not finished) race on it.
static __device__ __align__(256) unsigned char g_raster_scratch[EPROP_STATIC_RASTER_BYTES];

static constexpr int kMaxScratchDevices = 64;
static void *g_raster_scratch_addr[kMaxScratchDevices];
static std::mutex g_raster_scratch_mu;    // guards the address table

extern "C" eprop_status eprop_readout_raster_static(eprop_net *net, uint8_t *raster, int32_t is_device) {
    if (!net || !raster) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    if (!net->have_inputs) return fail(net, EPROP_ESTATE, "eprop_set_inputs_targets must come first");
    if (!net->n.record_raster) return fail(net, EPROP_EINVAL, "raster needs record_raster = 1");
    const long long bytes = (long long)net->cfg.batch * net->T_in * net->cfg.n_rec;
    if (bytes > (long long)EPROP_STATIC_RASTER_BYTES)
        return fail(net, EPROP_EINVAL,
                    "raster (batch * T * n_rec bytes) exceeds EPROP_STATIC_RASTER_BYTES of static scratch");
    if (!net->have_sim) return fail(net, EPROP_ESTATE, "no simulate call since the last set_inputs");
    int cur = -1;
    CK(net, cudaGetDevice(&cur));
    if (cur != net->dev) return fail(net, EPROP_EINVAL, "the network's device must be the current device");
    if (cur < 0 || cur >= kMaxScratchDevices) return fail(net, EPROP_EINVAL, "device ordinal out of range");
    // the scratch address of this device, resolved once with the device
    // current (the first call may load the module: a one-time setup); the
    // table is shared by every host thread, so it is read and filled under
    // a lock.  A device reset (cudaDeviceReset) invalidates every network
    // of that device and this address with them.
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_raster_scratch_mu);
        if (!g_raster_scratch_addr[cur]) {
            void *a = nullptr;
            CK(net, cudaGetSymbolAddress(&a, g_raster_scratch));
            g_raster_scratch_addr[cur] = a;
        }
        scratch = static_cast<unsigned char *>(g_raster_scratch_addr[cur]);
    }
    Net nn = net->n;
    nn.T = net->T_in;
    eprop::launch_unpack_raster(nn, scratch, net->st);
    CK(net, cudaGetLastError());
    CK(net, cudaMemcpyAsync(raster, scratch, (size_t)bytes,
                            is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, net->st));
    CK(net, cudaStreamSynchronize(net->st));
    return EPROP_OK;
}

// ---- the window's learning-signal product on its own (tensor cores)

// status word of the stand-alone product (bit 1: a bounded wait gave up)
static __device__ unsigned int g_lsig_status;

extern "C" eprop_status eprop_learning_signals(const float *feedback, const float *E, float *L, int32_t n_rec,
                                               int32_t U, int32_t n_out, int32_t batch, void *cuda_stream) {
    if (!feedback || !E || !L) return fail(nullptr, EPROP_EINVAL, "feedback, E and L are required");
    if (n_rec < 1 || U < 1 || n_out < 1 || batch < 1 || n_out > eprop::kMaxOut || batch >= 65536)
        return fail(nullptr, EPROP_EINVAL, "sizes out of range (1 <= n_out <= 1024, 1 <= batch < 65536)");
    cudaPointerAttributes pa[3];
    const void *ptrs[3] = {feedback, E, L};
    for (int q = 0; q < 3; ++q)
        if (cudaPointerGetAttributes(&pa[q], ptrs[q]) != cudaSuccess || pa[q].type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(nullptr, EPROP_EINVAL, "feedback, E and L must be device pointers");
        }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const unsigned int zero = 0;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_lsig_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    unsigned int *flag = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&flag, g_lsig_status);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "learning-signal status");
    eprop::prepare_learning_signal_attributes();
    eprop::launch_learning_signals(feedback, E, L, n_rec, U, n_out, batch, flag, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "learning-signal kernel launch");
    unsigned int h = 0;
    e = cudaMemcpyFromSymbolAsync(&h, g_lsig_status, sizeof(h), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "learning-signal kernel");
    if (h & 2u) return fail(nullptr, EPROP_ETIMEOUT, "a bounded wait for the tensor-core products gave up");
    return EPROP_OK;
}

extern "C" eprop_status eprop_read_surrogate(eprop_net *net, float *psi, int32_t is_device) {
    if (!net || !psi) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    if (!net->n.record_psi) return fail(net, EPROP_EINVAL, "surrogate values need record_psi = 1");
    if (!net->have_sim) return fail(net, EPROP_ESTATE, "no simulate call since the last set_inputs");
    const long long cnt = (long long)net->cfg.batch * net->T_in * net->cfg.n_rec;
    CK(net, cudaMemcpyAsync(psi, net->n.rec_psi, cnt * 4,
                            is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, net->st));
    CK(net, cudaStreamSynchronize(net->st));
    return EPROP_OK;
}

extern "C" eprop_status eprop_get_stats(eprop_net *net, eprop_stats *out) {
    if (!net || !out) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    unsigned long long h = 0;
    CK(net, cudaMemcpyAsync(&h, net->n.events, 8, cudaMemcpyDeviceToHost, net->st));
    CK(net, cudaStreamSynchronize(net->st));
    out->events = (int64_t)h;
    out->kernel_launches = net->launches;
    out->trace_launches = net->trace_launches;
    out->windows = net->windows;
    out->trace_ms = 0.0;
    if (net->cfg.profile) {
        for (long long w = 0; w < net->windows && 2 * w + 1 < (long long)net->ev.size(); ++w) {
            float ms = 0.f;
            CK(net, cudaEventElapsedTime(&ms, net->ev[2 * w], net->ev[2 * w + 1]));
            out->trace_ms += ms;
        }
    }
    return EPROP_OK;
}

extern "C" eprop_status eprop_sync(eprop_net *net) {
    if (!net) return EPROP_EINVAL;
    if (net->bad) return fail(net, EPROP_ESTATE, "network is in an error state");
    CK(net, cudaStreamSynchronize(net->st));
    CK(net, cudaGetLastError());
    unsigned int f = 0;
    CK(net, cudaMemcpy(&f, net->n.err_flags, 4, cudaMemcpyDeviceToHost));
    if (f & 6u) {
        net->bad = 1;
        net->err = (f & 4u) ? "a bounded grid-barrier wait of the persistent step loop gave up"
                            : "a bounded wait for a bulk copy or the tensor cores gave up";
        return EPROP_ETIMEOUT;
    }
    if (f & 1u) net->err = "warning: a synapse skipped more update windows than the coefficient ring holds";
    return EPROP_OK;
}

extern "C" void eprop_destroy(eprop_net *net) {
    if (!net) return;
    if (net->st) cudaStreamSynchronize(net->st);
    else cudaDeviceSynchronize();
    if (net->gexec) cudaGraphExecDestroy(net->gexec);
    for (cudaEvent_t e : net->ev) cudaEventDestroy(e);
    free_all(net->in_allocs);
    free_all(net->win_allocs);
    free_all(net->fixed_allocs);
    if (net->ev_fork) cudaEventDestroy(net->ev_fork);
    if (net->ev_join) cudaEventDestroy(net->ev_join);
    if (net->st2) cudaStreamDestroy(net->st2);
    if (net->own_stream) cudaStreamDestroy(net->st);
    delete net;
}

extern "C" const char *eprop_last_error(const eprop_net *net) {
    if (!net) return g_create_err.c_str();
    return net->err.c_str();
}
