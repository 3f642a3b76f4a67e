// Band-major learning state (trace_kernel 4): the dense window pass with the
// window coefficients of the targets held in shared memory.
//
// In the dense window pass every synapse j <- i combines, once per update
// window, its state with the window coefficients of its target j (one
// 12-28 byte entry per target) and, per arrival, one table entry Q(a) of j
// (the closed form at the top of kernels_window.cu; Eq. final-gradient,
// Eq. filtered-eligibility-trace).  With the records by source row the
// coefficient lookups are random over all targets: one L2 request per
// synapse, the bound of the source-major pass.  Here the records are kept
// by target band: band b holds every synapse whose target lies in
// [b W, (b + 1) W), by source row, padded to whole tiles of kBandTile
// records.  One CTA per SM keeps the coefficients of the band it works on in
// shared memory (W = 12288 LIF, 4608 ALIF targets) and streams the band's
// tiles with bulk copies; per tile it also copies the records of the rows
// the tile spans: per source row and window, the presynaptic trace zbar at
// the window start for every delay and the row's spike steps of the window
// (computed once per window for all rows, so the per-band visits of a row
// cost a 48-64 byte copy).  A synapse then needs an L2 request only for the
// table entries of its arrivals.  Tiles are dealt round-robin in band
// order, so the CTAs work on one or two bands at a time and the table slabs
// of those bands stay in L2.
//
// Arithmetic per synapse is that of window_pass_kernel (same coefficient,
// same row summary, arrivals in ascending order), so both forms give the
// same bits.  Delivery reads a spiking row's records from its segments in
// every band (seg[row][band]); the sum into the input ring is the exact
// int64 fixed point of the source-major delivery.  Weights and gradients are
// read back in the creation order: the position of a record in its band is
// recomputed from the source-major target array (one warp per row, per-band
// running counts), the same rule that placed it.
#include "eprop_internal.cuh"
#include "eprop_launch.h"

namespace eprop {

namespace {

constexpr int kBandStagesMax = 8;      // stages of the window kernel (as many as fit)
constexpr size_t kBandSmem = 227 * 1024 - 1024;   // dynamic shared memory of the window kernel, at most
constexpr int kRowCap = 128;             // row records staged per tile
constexpr int kBandRowBits = 15;         // row - tile row0 < 2^15

__device__ __forceinline__ int run_step_b(const Net &n, int i) { return n.clock->r_base + i; }

__device__ __forceinline__ const uint32_t *words_b(const Net &n, int src) {
    return n.bits + (long long)src * n.RW;
}

// bulk copy into shared memory with the default L2 policy (row records are
// read again by the next band)
__device__ __forceinline__ void bulk_g2s_keep(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__host__ __device__ constexpr int band_coef_floats(bool alif) { return alif ? 7 : 3; }
// one stage: records, weights, trace(s) of a tile, then its staged row records
__host__ __device__ inline uint32_t band_stage_bytes(bool alif, int rr_stride) {
    return (uint32_t)((4096 * (alif ? 4 : 3) + kRowCap * rr_stride + 127) & ~127);
}

// ------------------------------------------------------------- layout build

// per row and band: number of synapses (written into seg[row][band])
__global__ void band_count_kernel(const long long *row_ptr, const uint32_t *tgt_d, int S, int W, int nb,
                                  int *seg) {
    extern __shared__ int cnt_s[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *cnt = cnt_s + warp * nb;
    for (int row = blockIdx.x * (blockDim.x >> 5) + warp; row < S; row += gridDim.x * (blockDim.x >> 5)) {
        for (int b = lane; b < nb; b += 32) cnt[b] = 0;
        __syncwarp();
        const long long rb = row_ptr[row], re = row_ptr[row + 1];
        for (long long q = rb + lane; q < re; q += 32) atomicAdd(&cnt[(int)((tgt_d[q] & 0xFFFFFFu) / W)], 1);
        __syncwarp();
        for (int b = lane; b < nb; b += 32) seg[(long long)row * nb + b] = cnt[b];
        __syncwarp();
    }
}

// per chunk of rows: the chunk's count per band
__global__ void band_chunk_sum_kernel(const int *seg, int S, int nb, int chunk, long long *part) {
    const int c = blockIdx.x;
    const int r0 = c * chunk, r1 = min(S, r0 + chunk);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        long long s = 0;
        for (int r = r0; r < r1; ++r) s += seg[(long long)r * nb + b];
        part[(long long)c * nb + b] = s;
    }
}

// counts -> first position of each row in each band (exclusive prefix over
// the rows), from each chunk's offset
__global__ void band_chunk_scan_kernel(int *seg, int S, int nb, int chunk, const long long *off) {
    const int c = blockIdx.x;
    const int r0 = c * chunk, r1 = min(S, r0 + chunk);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        long long s = off[(long long)c * nb + b];
        for (int r = r0; r < r1; ++r) {
            const long long i = (long long)r * nb + b;
            const int v = seg[i];
            seg[i] = (int)s;
            s += v;
        }
    }
}

// largest row r in [0, S] with seg[r][b] <= p
__device__ __forceinline__ int band_row_of(const int *seg, int S, int nb, int b, long long p) {
    int lo = 0, hi = S;                      // seg[0][b] = 0 <= p
    while (hi > lo) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)seg[(long long)mid * nb + b] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// per tile: its band, first row and the rows it spans
__global__ void band_tiles_kernel(const int *seg, const long long *band_tile0, int S, int nb, long long n_tiles,
                                  int4 *tiles, unsigned *flag) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles;
         t += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = nb - 1;             // band: largest b with band_tile0[b] <= t
        while (hi > lo) {
            const int mid = (lo + hi + 1) >> 1;
            if (band_tile0[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int b = lo;
        const long long total = seg[(long long)S * nb + b];
        const long long p = (t - band_tile0[b]) * kBandTile;
        const long long pl = min(p + kBandTile - 1, total - 1);
        const int r0 = band_row_of(seg, S, nb, b, p);
        const int r1 = band_row_of(seg, S, nb, b, pl);
        if (r1 - r0 >= (1 << kBandRowBits)) atomicOr(flag, 1u);
        tiles[t] = make_int4(r0, r1 - r0 + 1, b, 0);
    }
}

// Position in the band-major order of every record of one source row, in
// the creation order: records of the row in band b take the positions
// band_base[b] + seg[row][b] + 0, 1, ... in their order inside the row.
// One warp per row; cnt (nb ints of shared memory) holds the running
// counts.  f(q, q_band, band, target - band start) per record.
template <typename F>
__device__ __forceinline__ void band_walk_row(const Net &n, int row, int *cnt, F f) {
    const int lane = threadIdx.x & 31;
    for (int b = lane; b < n.nb; b += 32) cnt[b] = 0;
    __syncwarp();
    const long long rb = n.row_ptr[row], re = n.row_ptr[row + 1];
    const int *sg = n.seg + (long long)row * n.nb;
    for (long long q0 = rb; q0 < re; q0 += 32) {
        const long long q = q0 + lane;
        const bool in = q < re;
        const unsigned act = __ballot_sync(0xffffffffu, in);
        const uint32_t j = in ? (n.tgt_d[q] & 0xFFFFFFu) : 0u;
        const int b = (int)(j / (uint32_t)n.band_w);
        const unsigned grp = __match_any_sync(0xffffffffu, in ? b : -1);
        const int rank = __popc(grp & ((1u << lane) - 1u));
        const int base = in ? cnt[b] : 0;
        __syncwarp();
        if (in) {
            f(q, n.band_base[b] + sg[b] + base + rank, b, (int)(j - (uint32_t)b * n.band_w));
            if (rank == 0) cnt[b] = base + __popc(grp);
        }
        __syncwarp();
        (void)act;
    }
}

// places the creation-order records (tgt_d, w_src) into the band-major arrays
__global__ void band_scatter_kernel(Net n, const float *w_src, uint32_t *bd_td, float *w_b) {
    extern __shared__ int cnt_s[];
    const int warp = threadIdx.x >> 5;
    int *cnt = cnt_s + warp * n.nb;
    for (int row = blockIdx.x * (blockDim.x >> 5) + warp; row < n.n_src; row += gridDim.x * (blockDim.x >> 5)) {
        band_walk_row(n, row, cnt, [&](long long q, long long qb, int b, int tl) {
            const int4 ti = n.tiles[qb / kBandTile];
            const uint32_t d = n.tgt_d[q] >> 24;
            bd_td[qb] = (uint32_t)tl | ((d - 1u) << 14) | ((uint32_t)(row - ti.x) << 17);
            w_b[qb] = w_src[q];
            (void)b;
        });
    }
}

// band-major weights / gradients -> creation order, rows [r0, r1)
__global__ void band_gather_kernel(Net n, int r0, int r1, long long q_begin, float *w_dst, float *g_dst) {
    extern __shared__ int cnt_s[];
    const int warp = threadIdx.x >> 5;
    int *cnt = cnt_s + warp * n.nb;
    for (int row = r0 + blockIdx.x * (blockDim.x >> 5) + warp; row < r1; row += gridDim.x * (blockDim.x >> 5)) {
        band_walk_row(n, row, cnt, [&](long long q, long long qb, int b, int tl) {
            if (w_dst) w_dst[q - q_begin] = n.w[qb];
            if (g_dst) g_dst[q - q_begin] = n.grad[qb];
            (void)b;
            (void)tl;
        });
    }
}


// ------------------------------------------------------------ row records

// Row record of every source for the window (a0, r_end]: zbar at a0 of the
// row's delay-d synapses for d = 1..D (RowInfo.zbar_a0, the value the
// source-major pass uses); per delay d the range [c0, ce) of the row's
// spike list whose delay-d arrivals fall in the window (packed c0 | ce << 8,
// 0xFFFF when the row has more spikes than the record keeps); the steps -
// s_lo of the row's spikes in [a0 + 1 - D, r_end - 1] (at most rr_cap).
// Layout: float zb[D] | u16 range[D] | u16 steps[rr_cap].
__global__ void band_rows_kernel(Net n, int i_end) {
    const int r_end = run_step_b(n, i_end);
    const int a0 = r_end - n.U;
    const int D = n.D;
    const int s_lo = a0 + 1 - D, s_hi = r_end - 1;
    const int src = blockIdx.x * blockDim.x + threadIdx.x;
    if (src >= n.n_src) return;
    const uint32_t *words = words_b(n, src);
    unsigned char *rec = n.rrec + (long long)src * n.rr_stride;
    float *zb = reinterpret_cast<float *>(rec);
    const int at = n.anchor_t[src];
    const float az = n.anchor_z[src];
    for (int d = 1; d <= D; ++d) zb[d - 1] = row_info(n, words, at, az, a0, d, false).zbar_a0;
    unsigned short *rg = reinterpret_cast<unsigned short *>(rec + 4 * D);
    unsigned short *sp = rg + D;
    const int mask = n.RW * 32 - 1;
    int cnt = 0;
    int r = s_lo < 1 ? 1 : s_lo;
    while (r <= s_hi) {
        const int p = r & mask;
        const int bit = p & 31;
        const int span = min(31 - bit, s_hi - r);
        uint32_t m = words[p >> 5] >> bit;
        if (span < 31) m &= (2u << span) - 1u;
        while (m) {
            if (cnt < n.rr_cap) sp[cnt] = (unsigned short)(r + __ffs(m) - 1 - s_lo);
            ++cnt;
            m &= m - 1;
        }
        r += span + 1;
    }
    for (int d = 1; d <= D; ++d) {
        if (cnt > n.rr_cap) {
            rg[d - 1] = 0xFFFFu;
            continue;
        }
        // arrival s + d in (a0, r_end]  <=>  D <= step + d <= U + D - 1
        int c0 = 0, ce = 0;
        for (int c = 0; c < cnt; ++c) {
            const int v = (int)sp[c] + d;
            c0 += v < D;
            ce += v <= n.U + D - 1;
        }
        rg[d - 1] = (unsigned short)(c0 | (ce << 8));
    }
}

template <bool ALIF>
__device__ __forceinline__ float4 band_table(const Net &n, long long qi) {
    if (ALIF) return __ldg(reinterpret_cast<const float4 *>(n.qp) + qi);
    const float2 t = __ldg(reinterpret_cast<const float2 *>(n.qp) + qi);
    return make_float4(t.x, t.y, 0.f, 0.f);
}

// arrivals of emission steps [lo, hi] (from the spike bits), added to G and
// the traces in ascending order (the order of the spike-list path)
template <bool ALIF>
__device__ __noinline__ void band_scan(const Net n, const uint32_t *words, int lo, int hi, int d, long long qrow,
                                       float &G, float &ebar, float &epsa) {
    const int mask = n.RW * 32 - 1;
    int r = lo < 1 ? 1 : lo;
    while (r <= hi) {
        const int p = r & mask;
        const int bit = p & 31;
        const int span = min(31 - bit, hi - r);
        uint32_t m = words[p >> 5] >> bit;
        if (span < 31) m &= (2u << span) - 1u;
        while (m) {
            const int a = r + __ffs(m) - 1 + d;
            m &= m - 1;
            const float4 t = band_table<ALIF>(n, qrow + (long long)a * n.n_rec);
            G += t.x;
            ebar += t.y;
            if (ALIF) epsa += t.z;
        }
        r += span + 1;
    }
}

// ------------------------------------------------------------ window pass

constexpr int kBandConsumers = 16;                     // consumer warps (512 threads, two records each)
constexpr int kBandU = kBandTile / (kBandConsumers * 32);   // records per thread and tile
constexpr int kBandWLif = 12288, kBandWAlif = 4608;  // targets per band (coefficients in shared memory)

__device__ __forceinline__ void band_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// A tile's per-thread state between its two phases: the records read from
// shared memory and the table entries of the first two arrivals in flight.
// rng: the record's arrival range (c0 | ce << 8, 0xFFFF: scan the bits);
// rro: byte offset of its row record in the stage, or -1 - (row index in the
// tile) when the tile spans more rows than are staged.
template <bool ALIF>
struct BandRegs {
    uint32_t td[kBandU], rng[kBandU];
    float wv[kBandU], zr[kBandU], eb[kBandU], ep[kBandU];
    float4 t0[kBandU], t1[kBandU];
    int rro[kBandU];
    bool live[kBandU];
};

struct BandCtx {
    int a0, r_end, s_lo, D, N, rs;
    const float *qp;                             // table entries of step a0 + 1
    float step;
};

// table entry of arrival step a of target j
template <bool ALIF>
__device__ __forceinline__ float4 band_entry(const BandCtx &x, int a, int j) {
    const long long e = (long long)(a - x.a0 - 1) * x.N + j;
    if (ALIF) return __ldg(reinterpret_cast<const float4 *>(x.qp) + e);
    const float2 t = __ldg(reinterpret_cast<const float2 *>(x.qp) + e);
    return make_float4(t.x, t.y, 0.f, 0.f);
}

// phase 1 of a tile: records, weight, traces and row summary into
// registers; the table loads of the first two arrivals are issued
template <bool ALIF, int TB>
__device__ __forceinline__ void band_phase1(const Net &n, const BandCtx &x, uint32_t soff, int4 dk, int ct,
                                            BandRegs<ALIF> &r) {
    // stage pointers derived from the dynamic shared array itself, so the
    // compiler emits shared-memory loads
    extern __shared__ __align__(128) unsigned char dsm[];
    const unsigned char *s = dsm + soff;
    constexpr int W = ALIF ? kBandWAlif : kBandWLif;
    const uint32_t *s_td = reinterpret_cast<const uint32_t *>(s);
    const float *s_w = reinterpret_cast<const float *>(s + 4096);
    const unsigned char *s_rr = s + (ALIF ? 16384 : 12288);
    const int rows_st = min(dk.z, kRowCap);
    const int jb = dk.w * W;
#pragma unroll
    for (int u = 0; u < kBandU; ++u) {
        const int idx = ct + kBandConsumers * 32 * u;
        const uint32_t td = s_td[idx];
        r.td[u] = td;
        r.live[u] = false;
        if (td == kBandPad) continue;
        const int tl = (int)(td & 0x3FFFu);
        const int dl = (int)((td >> 14) & 7u) + 1;
        const int rit = (int)(td >> 17);
        uint32_t rng;
        int s1 = 0, s2 = 0;
        if (rit < rows_st) {
            const unsigned char *rec = s_rr + rit * x.rs;
            r.rro[u] = rit * x.rs;
            r.zr[u] = reinterpret_cast<const float *>(rec)[dl - 1];
            const unsigned short *rg = reinterpret_cast<const unsigned short *>(rec + 4 * x.D);
            rng = rg[dl - 1];
            const int c0 = (int)(rng & 0xFFu), ce = (int)(rng >> 8);
            if (rng != 0xFFFFu && ce > c0) s1 = rg[x.D + c0];
            if (rng != 0xFFFFu && ce > c0 + 1) s2 = rg[x.D + c0 + 1];
        } else {
            const unsigned char *rec = n.rrec + (long long)(dk.y + rit) * x.rs;
            r.rro[u] = -1 - rit;
            r.zr[u] = reinterpret_cast<const float *>(rec)[dl - 1];
            const unsigned short *rg = reinterpret_cast<const unsigned short *>(rec + 4 * x.D);
            rng = rg[dl - 1];
            const int c0 = (int)(rng & 0xFFu), ce = (int)(rng >> 8);
            if (rng != 0xFFFFu && ce > c0) s1 = rg[x.D + c0];
            if (rng != 0xFFFFu && ce > c0 + 1) s2 = rg[x.D + c0 + 1];
        }
        r.rng[u] = rng;
        r.wv[u] = s_w[idx];
        if (TB) r.eb[u] = trace16_to_float(reinterpret_cast<const uint16_t *>(s + 8192)[idx], TB);
        else r.eb[u] = reinterpret_cast<const float *>(s + 8192)[idx];
        r.ep[u] = 0.f;
        if (ALIF) {
            if (TB) r.ep[u] = trace16_to_float(reinterpret_cast<const uint16_t *>(s + 12288)[idx], TB);
            else r.ep[u] = reinterpret_cast<const float *>(s + 12288)[idx];
        }
        const int na = rng == 0xFFFFu ? 0 : (int)(rng >> 8) - (int)(rng & 0xFFu);
        r.live[u] = na > 0 || rng == 0xFFFFu || r.zr[u] != 0.f || r.eb[u] != 0.f || r.ep[u] != 0.f;
        if (na >= 1) r.t0[u] = band_entry<ALIF>(x, x.s_lo + s1 + dl, jb + tl);
        if (na >= 2) r.t1[u] = band_entry<ALIF>(x, x.s_lo + s2 + dl, jb + tl);
    }
}

// phase 2 of a tile: the window transfer with the band's coefficients, the
// arrivals in ascending order (the first two from phase 1), the stores
template <bool ALIF, int TB>
__device__ __forceinline__ void band_phase2(const Net &n, const BandCtx &x, uint32_t soff, long long q0, int4 dk, int ct,
                                            const BandRegs<ALIF> &r) {
    extern __shared__ __align__(128) unsigned char dsm[];
    const float *cf = reinterpret_cast<const float *>(dsm);
    const unsigned char *s = dsm + soff;
    constexpr int W = ALIF ? kBandWAlif : kBandWLif;
    const int jb = dk.w * W;
    const unsigned char *s_rr = s + (ALIF ? 16384 : 12288);
#pragma unroll
    for (int u = 0; u < kBandU; ++u) {
        if (!r.live[u]) continue;
        const int idx = ct + kBandConsumers * 32 * u;
        const uint32_t td = r.td[u];
        const int tl = (int)(td & 0x3FFFu);
        const int dl = (int)((td >> 14) & 7u) + 1;
        Coef co;
        if (ALIF) {
            co.c0 = make_float4(cf[tl], cf[W + tl], cf[2 * W + tl], cf[3 * W + tl]);
            co.c1 = make_float4(cf[4 * W + tl], cf[5 * W + tl], cf[6 * W + tl], 0.f);
        } else {
            co.c0 = make_float4(cf[tl], cf[W + tl], cf[2 * W + tl], 0.f);
            co.c1 = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float G = 0.f, zbar = r.zr[u], ebar = r.eb[u], epsa = r.ep[u];
        apply_coef<ALIF>(n, co, zbar, epsa, ebar, G);
        const uint32_t rng = r.rng[u];
        if (rng != 0xFFFFu) {
            const int c0 = (int)(rng & 0xFFu), ce = (int)(rng >> 8);
            if (ce > c0) {
                G += r.t0[u].x;
                ebar += r.t0[u].y;
                if (ALIF) epsa += r.t0[u].z;
            }
            if (ce > c0 + 1) {
                G += r.t1[u].x;
                ebar += r.t1[u].y;
                if (ALIF) epsa += r.t1[u].z;
            }
            if (ce > c0 + 2) {
                // further arrivals: four table loads in flight, summed in order
                const int ro = r.rro[u];
                const unsigned char *rec = ro >= 0 ? s_rr + ro : n.rrec + (long long)(dk.y - 1 - ro) * x.rs;
                const unsigned short *sp = reinterpret_cast<const unsigned short *>(rec + 4 * x.D) + x.D;
                for (int cc = c0 + 2; cc < ce; cc += 4) {
                    float4 t[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        t[q] = cc + q < ce ? band_entry<ALIF>(x, x.s_lo + (int)sp[cc + q] + dl, jb + tl)
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (cc + q < ce) {
                            G += t[q].x;
                            ebar += t[q].y;
                            if (ALIF) epsa += t[q].z;
                        }
                }
            }
        } else {
            // rows with more spikes than the record holds
            const int row = dk.y + (int)(td >> 17);
            band_scan<ALIF>(n, words_b(n, row), x.a0 + 1 - dl, x.r_end - dl, dl, (long long)(-x.a0 - 1) * x.N + jb + tl,
                            G, ebar, epsa);
        }
        const long long q = q0 + idx;
        if (G != 0.f) __stcs(n.w + q, sgd_step(r.wv[u], x.step, G));
        if (TB) __stcs(reinterpret_cast<uint16_t *>(n.ebar) + q, float_to_trace16(ebar, TB));
        else __stcs(reinterpret_cast<float *>(n.ebar) + q, ebar);
        if (ALIF) store_trace(n.epsa, q, epsa, TB);
        if (n.record_grad) n.grad[q] = grad_add(n.grad[q], n.inv_B, G);
    }
}

// Shared-memory pipeline of the window kernel, as the consumers see it.
struct BandSm {
    uint64_t *full, *empty, *bandbar;
    int4 *desc;
    uint32_t stg;                                // byte offset of stage 0 in the dynamic shared array
};

// consumers: meet at the band barrier (bounded); false when a wait gave up
__device__ __forceinline__ bool band_sync(const Net &n, const BandSm &m, int &bphase) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) band_arrive(m.bandbar);
    const bool ok = mbar_wait(m.bandbar, (uint32_t)(bphase & 1), n.err_flags);
    ++bphase;
    return ok;
}

// One consumer step: tile c is in `cur` (phase 1 done, descriptor dk);
// phase 1 of tile c + 1 into `nxt`, the band's coefficients if tile c
// starts a new band, phase 2 of tile c, release of its stage.  False when
// the pass is over (or a wait gave up).
template <bool ALIF, int TB>
__device__ __forceinline__ bool band_wstep(const Net &n, const BandCtx &x, const BandSm &m, int c, int4 &dk,
                                           int &cur_band, int &bphase, BandRegs<ALIF> &cur, BandRegs<ALIF> &nxt) {
    const int S = n.band_stages;
    const uint32_t kStage = n.band_stage_b;
    const int ct = threadIdx.x;
    const int k = c % S, k1 = (c + 1) % S;
    if (!mbar_wait(&m.full[k1], (uint32_t)(((c + 1) / S) & 1), n.err_flags)) return false;
    const int4 dn = m.desc[k1];
    if (dn.x >= 0) band_phase1<ALIF, TB>(n, x, m.stg + k1 * kStage, dn, ct, nxt);
    if (dk.w != cur_band) {
        // every consumer warp is past the previous band's tiles
        if (!band_sync(n, m, bphase)) return false;
        constexpr int W = ALIF ? kBandWAlif : kBandWLif;
        const int j0 = dk.w * W;
        const int jn = min(W, x.N - j0);
        extern __shared__ __align__(128) unsigned char dsm[];
        float *cf = reinterpret_cast<float *>(dsm);
        for (int jj = ct; jj < jn; jj += kBandConsumers * 32) {
            if (ALIF) {
                const float4 *q = reinterpret_cast<const float4 *>(n.coef) + 2LL * (j0 + jj);
                const float4 c0 = __ldg(q), c1 = __ldg(q + 1);
                cf[jj] = c0.x; cf[W + jj] = c0.y; cf[2 * W + jj] = c0.z; cf[3 * W + jj] = c0.w;
                cf[4 * W + jj] = c1.x; cf[5 * W + jj] = c1.y; cf[6 * W + jj] = c1.z;
            } else {
                const float4 c0 = __ldg(reinterpret_cast<const float4 *>(n.coef) + (j0 + jj));
                cf[jj] = c0.x; cf[W + jj] = c0.y; cf[2 * W + jj] = c0.z;
            }
        }
        if (!band_sync(n, m, bphase)) return false;
        cur_band = dk.w;
    }
    band_phase2<ALIF, TB>(n, x, m.stg + k * kStage, (long long)dk.x * kBandTile, dk, ct, cur);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) band_arrive(&m.empty[k]);
    dk = dn;
    return dn.x >= 0;
}

constexpr int kBandThreadsAll = (kBandConsumers + 1) * 32;   // consumers + one producer warp

// Warp-specialised window pass.  One CTA per SM: a producer warp streams
// the CTA's tiles (round-robin over the grid, so all CTAs move through the
// bands together) into shared-memory stages (as many as fit) with bulk copies
// (records, weights, traces and the row records of the rows a tile spans),
// 16 consumer warps process every tile, each its 64 records.  A consumer
// warp is software-pipelined by one tile (phase 1 of tile c + 1, with the
// table loads of the first two arrivals, is issued before phase 2 of tile
// c) and releases a stage on its own (empty mbarrier), so warps drift
// apart instead of meeting at a block barrier per tile; they meet only to
// swap the band's coefficients in shared memory.  Every wait is bounded.
// TB: trace storage (0 FP32, 1 BF16, 2 FP16).
template <bool ALIF, int TB>
__global__ void __launch_bounds__(kBandThreadsAll, 1) window_band_kernel(Net n, int i_end) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ uint64_t full[kBandStagesMax], empty[kBandStagesMax], bandbar;
    __shared__ int4 desc[kBandStagesMax];        // (tile, first row, rows spanned, band); tile -1: none
    constexpr int NF = band_coef_floats(ALIF);
    const int S = n.band_stages;
    const uint32_t kStage = n.band_stage_b;
    constexpr uint32_t kRecB = kBandTile * 4u;             // bytes of a tile's 4-byte stream
    constexpr uint32_t kTrB = TB ? kBandTile * 2u : kRecB;
    constexpr int W = ALIF ? kBandWAlif : kBandWLif;
    BandCtx x;
    x.D = n.D;
    x.N = n.n_rec;
    x.r_end = run_step_b(n, i_end);
    x.a0 = x.r_end - n.U;
    x.s_lo = x.a0 + 1 - x.D;
    x.qp = n.qp;
    x.step = n.lr * n.inv_B;
    x.rs = n.rr_stride;
    unsigned char *stg = dsm + (((size_t)NF * W * 4 + 127) & ~(size_t)127);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kBandConsumers);
        }
        mbar_init(&bandbar, kBandConsumers);
    }
    fence_mbar_init();
    __syncthreads();
    if (warp == kBandConsumers) {
        // ---- producer (one thread)
        if (lane != 0) return;
        long long t = blockIdx.x;
        int4 ti = t < n.n_tiles ? n.tiles[t] : make_int4(0, 0, 0, 0);
        int issued = 0;
        bool ended = false;                      // the end marker went into stage issued % S
        for (int m = 0;; ++m) {
            const int k = m % S;
            if (m >= S && !mbar_wait(&empty[k], (uint32_t)(((m / S) - 1) & 1), n.err_flags)) break;
            if (t >= n.n_tiles) {
                desc[k] = make_int4(-1, 0, 0, 0);
                band_arrive(&full[k]);
                ended = true;
                break;
            }
            const int4 cur = ti;
            const long long tn = t + gridDim.x;
            if (tn < n.n_tiles) ti = n.tiles[tn];     // descriptor of the next issue
            const uint32_t rrb = (uint32_t)min(cur.y, kRowCap) * (uint32_t)x.rs;
            unsigned char *s = stg + k * kStage;
            const long long q0 = t * kBandTile;
            desc[k] = make_int4((int)t, cur.x, cur.y, cur.z);
            mbar_expect_tx(&full[k], 2u * kRecB + kTrB * (ALIF ? 2u : 1u) + rrb);
            bulk_g2s(s, n.bd_td + q0, kRecB, &full[k]);
            bulk_g2s(s + 4096, n.w + q0, kRecB, &full[k]);
            bulk_g2s(s + 8192, reinterpret_cast<const unsigned char *>(n.ebar) + q0 * (TB ? 2 : 4), kTrB, &full[k]);
            if (ALIF)
                bulk_g2s(s + 12288, reinterpret_cast<const unsigned char *>(n.epsa) + q0 * (TB ? 2 : 4), kTrB,
                         &full[k]);
            bulk_g2s_keep(s + (ALIF ? 16384 : 12288), n.rrec + (long long)cur.x * x.rs, rrb, &full[k]);
            t = tn;
            issued = m + 1;
        }
        // the copies in flight land before the block can exit (the tile that
        // last used the end marker's stage was consumed before the marker)
        for (int m = max(0, issued - S); m < issued; ++m)
            if (!(ended && m == issued - S)) mbar_wait(&full[m % S], (uint32_t)((m / S) & 1), n.err_flags);
        return;
    }
    // ---- consumers
    BandSm m;
    m.full = full;
    m.empty = empty;
    m.bandbar = &bandbar;
    m.desc = desc;
    m.stg = (uint32_t)(stg - dsm);
    int cur_band = -1, bphase = 0;
    if (!mbar_wait(&full[0], 0u, n.err_flags)) return;
    int4 dk = desc[0];
    if (dk.x < 0) return;
    BandRegs<ALIF> X, Y;
    band_phase1<ALIF, TB>(n, x, m.stg, dk, threadIdx.x, X);
    for (int c = 0;; c += 2) {
        if (!band_wstep<ALIF, TB>(n, x, m, c, dk, cur_band, bphase, X, Y)) break;
        if (!band_wstep<ALIF, TB>(n, x, m, c + 1, dk, cur_band, bphase, Y, X)) break;
    }
}

// -------------------------------------------------------------- delivery

// One work item of the band delivery: a spiking row's segments in a group
// of 32 bands (lane l: band 32 g + l), with the inclusive prefix of their
// lengths over the lanes.
struct BandItem {
    int src, g, part, incl, cnt, total;
    long long base;
};

__device__ __forceinline__ BandItem band_item(const Net &n, const int *ids, const BucketScan &bs, int ng, int np,
                                              long long it) {
    const int lane = threadIdx.x & 31;
    BandItem m;
    const int row = (int)(it / ((long long)ng * np));
    m.g = (int)((it / np) % ng);
    m.part = (int)(it % np);
    m.src = bucket_entry(n, ids, bs, row);
    const int b = m.g * 32 + lane;
    m.cnt = 0;
    m.base = 0;
    if (b < n.nb) {
        const int s0 = n.seg[(long long)m.src * n.nb + b];
        m.cnt = n.seg[(long long)(m.src + 1) * n.nb + b] - s0;
        m.base = n.band_base[b] + s0;
    }
    return m;
}

// Spikes of call step i (batch 1) into the input ring.  Work items: (spiking
// row, group of 32 bands, part), dealt round-robin to the warps; with few
// band groups a group's records are split into parts (as the source-major
// delivery splits rows), so a step's few spiking rows still spread over the
// grid.  The next item's segment bounds are loaded while the current one
// is delivered, four records per lane in flight.
__global__ void __launch_bounds__(256, 4) deliver_band_kernel(Net n, int i) {
    __shared__ unsigned long long ev_block;
    __shared__ long long ring_off[kMaxDelay + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = run_step_b(n, i);
    // the list slot of step r + 1 is cleared here (see deliver_kernel)
    if (blockIdx.x == 0 && threadIdx.x < kBkt) n.list_cnt[list_index(n, 0, (r + 1) % n.RS) + threadIdx.x] = 0;
    if (i > n.lengths[0]) return;
    if (threadIdx.x == 0) ev_block = 0ULL;
    if (threadIdx.x <= n.D)
        ring_off[threadIdx.x] = (long long)((n.clock->ring0 + i + (int)threadIdx.x) % (n.D + 1)) * n.n_rec;
    __syncthreads();
    const long long li = list_index(n, 0, r % n.RS);
    const int *ids = n.list_ids + li * n.list_cap;
    const BucketScan bs = bucket_scan(n.list_cnt + li);
    const int ng = (n.nb + 31) >> 5;
    const int np = ng == 1 ? 4 : (ng == 2 ? 2 : 1);   // parts per band group
    const long long items = (long long)bs.total * ng * np;
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long ev = 0ULL;
    BandItem nx;
    if (gw < items) nx = band_item(n, ids, bs, ng, np, gw);
    for (long long it = gw; it < items; it += nw) {
        BandItem m = nx;
        if (it + nw < items) nx = band_item(n, ids, bs, ng, np, it + nw);
        int incl = m.cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (m.g == 0 && m.part == 0 && lane == 0)
            ev += (unsigned long long)(n.row_ptr[m.src + 1] - n.row_ptr[m.src]);
        const int excl = incl - m.cnt;
        const int k_lo = (int)((long long)total * m.part / np), k_hi = (int)((long long)total * (m.part + 1) / np);
        for (int k0 = k_lo; k0 < k_hi; k0 += 128) {
            uint32_t tdv[4];
            float wv[4];
            int bm[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + lane + 32 * u;
                // lane holding record k: number of lanes whose inclusive end is <= k
                int l = 0;
#pragma unroll
                for (int w = 16; w > 0; w >>= 1) {
                    const int v = __shfl_sync(0xffffffffu, incl, l + w - 1);
                    if (v <= k) l += w;
                }
                const long long bq = __shfl_sync(0xffffffffu, m.base, l);
                const int eq = __shfl_sync(0xffffffffu, excl, l);
                bm[u] = m.g * 32 + l;
                const bool in = k < k_hi;
                const long long q = bq + (k - eq);
                tdv[u] = in ? n.bd_td[q] : kBandPad;
                wv[u] = in ? n.w[q] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (tdv[u] == kBandPad) continue;
                const int j = bm[u] * n.band_w + (int)(tdv[u] & 0x3FFFu);
                const int dl = (int)((tdv[u] >> 14) & 7u) + 1;
                const long long fx = __float2ll_rn(wv[u] * 4294967296.0f);
                atomicAdd(reinterpret_cast<unsigned long long *>(&n.ring[ring_off[dl] + j]), (unsigned long long)fx);
            }
        }
    }
    if (lane == 0 && ev) atomicAdd(&ev_block, ev);
    __syncthreads();
    if (threadIdx.x == 0 && ev_block) atomicAdd(n.events, ev_block);
}

}  // namespace

// ------------------------------------------------------------- launchers

int band_width(bool alif) { return alif ? kBandWAlif : kBandWLif; }

// dynamic shared memory of the window kernel for n.band_stages stages
size_t band_window_smem(const Net &n) {
    const int nf = band_coef_floats(n.alif != 0);
    return (((size_t)nf * band_width(n.alif != 0) * 4 + 127) & ~(size_t)127) +
           (size_t)n.band_stages * band_stage_bytes(n.alif != 0, n.rr_stride);
}

// stages that fit beside the coefficients (kBandSmem bytes in all)
int band_stages_fit(bool alif, int rr_stride) {
    const size_t coef = ((size_t)band_coef_floats(alif) * band_width(alif) * 4 + 127) & ~(size_t)127;
    const int s = (int)((kBandSmem - coef) / band_stage_bytes(alif, rr_stride));
    return s < kBandStagesMax ? s : kBandStagesMax;
}

uint32_t band_stage_size(bool alif, int rr_stride) { return band_stage_bytes(alif, rr_stride); }

static int band_walk_blocks(long long rows) {
    long long b = (rows + 3) / 4;
    return (int)(b < 65535 ? (b > 0 ? b : 1) : 65535);
}

void launch_band_count(const long long *row_ptr, const uint32_t *tgt_d, int S, int W, int nb, int *seg) {
    band_count_kernel<<<band_walk_blocks(S), 128, (size_t)4 * nb * 4>>>(row_ptr, tgt_d, S, W, nb, seg);
}

void launch_band_chunk_sum(const int *seg, int S, int nb, int chunk, long long *part) {
    band_chunk_sum_kernel<<<(S + chunk - 1) / chunk, 128>>>(seg, S, nb, chunk, part);
}

void launch_band_chunk_scan(int *seg, int S, int nb, int chunk, const long long *off) {
    band_chunk_scan_kernel<<<(S + chunk - 1) / chunk, 128>>>(seg, S, nb, chunk, off);
}

void launch_band_tiles(const int *seg, const long long *band_tile0, int S, int nb, long long n_tiles, int4 *tiles,
                       unsigned *flag) {
    long long blocks = (n_tiles + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    band_tiles_kernel<<<(int)blocks, 256>>>(seg, band_tile0, S, nb, n_tiles, tiles, flag);
}

void launch_band_scatter(const Net &n, const float *w_src, uint32_t *bd_td, float *w_b) {
    band_scatter_kernel<<<band_walk_blocks(n.n_src), 128, (size_t)4 * n.nb * 4>>>(n, w_src, bd_td, w_b);
}

void launch_band_gather(const Net &n, int r0, int r1, long long q_begin, float *w_dst, float *g_dst, cudaStream_t st) {
    if (r1 <= r0) return;
    band_gather_kernel<<<band_walk_blocks(r1 - r0), 128, (size_t)4 * n.nb * 4, st>>>(n, r0, r1, q_begin, w_dst,
                                                                                      g_dst);
}

void launch_window_band(const Net &n, int i_end, int sm_count, cudaStream_t st) {
    band_rows_kernel<<<(n.n_src + 255) / 256, 256, 0, st>>>(n, i_end);
    const size_t sm = band_window_smem(n);
#define EPROP_BAND(A, T) window_band_kernel<A, T><<<sm_count, kBandThreadsAll, sm, st>>>(n, i_end)
    if (n.alif) {
        if (n.trace_type == 1) EPROP_BAND(true, 1);
        else if (n.trace_type == 2) EPROP_BAND(true, 2);
        else EPROP_BAND(true, 0);
    } else {
        if (n.trace_type == 1) EPROP_BAND(false, 1);
        else if (n.trace_type == 2) EPROP_BAND(false, 2);
        else EPROP_BAND(false, 0);
    }
#undef EPROP_BAND
}

void launch_deliver_band(const Net &n, int i, int grid_x, cudaStream_t st) {
    deliver_band_kernel<<<grid_x, 256, 0, st>>>(n, i);
}

void prepare_band_attributes() {
    const int big = 227 * 1024;
    cudaFuncSetAttribute(band_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(band_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(band_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    const int w = (int)kBandSmem;
    cudaFuncSetAttribute(window_band_kernel<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, w);
    cudaFuncSetAttribute(window_band_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, w);
    cudaFuncSetAttribute(window_band_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, w);
    cudaFuncSetAttribute(window_band_kernel<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, w);
    cudaFuncSetAttribute(window_band_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, w);
    cudaFuncSetAttribute(window_band_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, w);
}

}  // namespace eprop
