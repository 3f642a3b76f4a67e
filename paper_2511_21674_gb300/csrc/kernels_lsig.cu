// Learning signals of an update window on the tensor cores (Eq. replace-
// wkj-by-bjk, Eq. final-gradient):
//
//   L[b][u][j] = sum_k B[j][k] E[b][u][k]
//
// for every neuron j, step u of the window and sample b.  As a GEMM this is
// D (M = neurons, N = window steps) = A (M x K) Bop (N x K)^T with both
// operands K-major exactly as they are stored (feedback B [N_rec][K], error
// window E [batch][U][K]), so no operand is transposed in memory.
//
// Precision: the tensor cores take TF32 operands (10 explicit mantissa
// bits).  Each operand x is split into hi = tf32(x) (round to nearest) and
// lo = tf32(x - hi); x - hi is exact in FP32 and lo keeps its top 11 bits,
// so hi + lo equals x to 2^-22 |x|.  The products hi*hi go into one FP32
// TMEM accumulator and the corrections hi*lo + lo*hi into a second one, so
// the large running sum takes one rounding per K-step of 8 (not three), and
// the epilogue adds the two; the dropped lo*lo product is below 2^-22 |a||b|.
// The result matches FP32 arithmetic to a few 1e-7 of sum_k |B_jk E_k|.
//
// Kernel shape: one CTA per tile of 128 neurons and sample (grid x = tiles,
// y = samples), 256 threads.  For each chunk of 32 K-elements the threads
// load the chunk of B (128 rows) and of E (the window's steps, padded to a
// multiple of 16) with coalesced loads, split them and store hi and lo in
// the 128-byte-swizzled K-major layout of the UMMA operand descriptors; one
// thread then issues the 3 x (K-steps of 8) tcgen05.mma of the chunk into
// the TMEM accumulators and commits them to an mbarrier, which every thread
// waits on (bounded) before the chunk buffers are refilled.  The epilogue
// reads both accumulators with tcgen05.ld (warp w % 4 owns TMEM lanes
// 32 (w % 4) .. +31, i.e. neurons; the two warpgroups split the columns),
// adds them and stores L[b][u][j] with the 32 lanes of a warp on 32
// consecutive neurons (coalesced 128-byte rows).  Windows longer than 128
// steps are done in passes of at most 128 columns.  The operand regions
// take ~65 KB of shared memory; the launch requests 100 KB so that at most
// two CTAs are resident on an SM, whose TMEM allocations (two accumulators,
// <= 256 columns per CTA) then always fit the SM's 512 columns.
#include <cstdint>

#include "eprop_internal.cuh"
#include "eprop_launch.h"

namespace eprop {

constexpr int kLsM = 128;          // neurons per tile (UMMA M)
constexpr int kLsKC = 32;          // K elements per chunk: one 128-byte swizzle row
constexpr int kLsNmax = 128;       // window steps per pass (two accumulators of <= 128 columns)
constexpr int kLsThreads = 256;
constexpr int kLsAreg = kLsM * 128;        // bytes of one A region (hi or lo)
constexpr int kLsEreg = kLsNmax * 128;     // bytes of one E region
// dynamic shared memory requested per CTA (the operand regions need less):
// 100 KB caps the residency at two CTAs per SM
constexpr size_t kLsSmem = 100 * 1024;
static_assert(1024 + 2 * (size_t)kLsAreg + 2 * (size_t)kLsEreg <= kLsSmem, "operand regions exceed the request");

// ---- PTX wrappers (tcgen05, sm_100 family)

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Byte offset of element k (0..31) of row r in a 128-byte-swizzled K-major
// region: rows are 128 bytes, the 16-byte chunk index is XORed with r mod 8
// (the region starts on a 1024-byte boundary, as the swizzle atom needs).
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) << 4) | ((k & 3) << 2)));
}

// Shared-memory matrix descriptor of a K-major operand with 128-byte swizzle:
// start address >> 4 (bits 0-13), leading byte offset (unused for swizzled
// K-major layouts, 1), stride byte offset 1024 >> 4 between 8-row groups
// (bits 32-45), the fixed 0b001 at bits 46-48, base offset 0, swizzle mode 2
// (128 B) at bits 61-63.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 32 lanes x 32 bits, 16 consecutive columns per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Stores x as (hi, lo) TF32 pair at byte offset off of the two regions.
__device__ __forceinline__ void put_split(unsigned char *hi, unsigned char *lo, uint32_t off, float x) {
    const uint32_t h = tf32_rna(x);
    const uint32_t l = tf32_rna(x - __uint_as_float(h));
    *reinterpret_cast<uint32_t *>(hi + off) = h;
    *reinterpret_cast<uint32_t *>(lo + off) = l;
}

__global__ void __launch_bounds__(kLsThreads) learning_signal_kernel(const float *__restrict__ fb,
                                                                     const float *__restrict__ E,
                                                                     float *__restrict__ L, int N, int U, int K,
                                                                     unsigned *err) {
    extern __shared__ unsigned char ls_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int b = blockIdx.y;
    const int j0 = blockIdx.x * kLsM;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(ls_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *a_hi = base, *a_lo = base + kLsAreg;
    unsigned char *e_hi = base + 2 * kLsAreg, *e_lo = e_hi + kLsEreg;
    const float *Eb = E + (long long)b * U * K;
    float *Lb = L + (long long)b * U * N;
    // TMEM: two accumulators (hi*hi, corrections) of a power of two >= 32
    // columns covering the widest pass
    const int npad_max = (min(U, kLsNmax) + 15) & ~15;
    uint32_t half = 32;
    while ((int)half < npad_max) half <<= 1;
    const uint32_t ncols = 2 * half;
    if (warp == 0) tmem_alloc(&tmem_slot, ncols);
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    uint32_t phase = 0;
    int ok = 1;
    const int q = warp & 3;               // TMEM lane quadrant of this warp
    for (int u0 = 0; u0 < U && ok; u0 += kLsNmax) {
        const int nu = min(U - u0, kLsNmax);
        const int npad = (nu + 15) & ~15;
        const uint32_t idesc = idesc_tf32(kLsM, npad);
        uint32_t acc = 0;                 // 0 until the first MMA of the pass
        for (int kc = 0; kc < K; kc += kLsKC) {
            const int k = kc + lane;
            const bool kin = k < K;
            // B chunk: 16 rows per warp, lane = k (coalesced along the row)
#pragma unroll 16
            for (int r = warp; r < kLsM; r += kLsThreads / 32) {
                const int j = j0 + r;
                const float x = (kin && j < N) ? __ldg(fb + (long long)j * K + k) : 0.f;
                put_split(a_hi, a_lo, sw128_off(r, lane), x);
            }
            // E chunk: the pass's steps, zero rows up to npad
#pragma unroll 4
            for (int r = warp; r < npad; r += kLsThreads / 32) {
                const int u = u0 + r;
                const float x = (kin && r < nu) ? __ldg(Eb + (long long)u * K + k) : 0.f;
                put_split(e_hi, e_lo, sw128_off(r, lane), x);
            }
            fence_proxy_async();          // generic stores -> tensor-core (async proxy) reads
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const int nks = (min(kLsKC, K - kc) + 7) >> 3;     // K-steps of 8 with data
                const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
                const uint32_t eh = smem_u32(e_hi), el = smem_u32(e_lo);
                for (int s = 0; s < nks; ++s) {
                    const uint32_t o = 32u * s;                      // 8 TF32 = 32 bytes along K
                    umma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(eh + o), idesc, acc);
                    umma_tf32(tmem + half, sdesc_sw128(ah + o), sdesc_sw128(el + o), idesc, acc);
                    umma_tf32(tmem + half, sdesc_sw128(al + o), sdesc_sw128(eh + o), idesc, 1);
                    acc = 1;
                }
                umma_commit(&bar);
            }
            // every thread waits for the chunk's MMAs (they read the buffers
            // about to be refilled, and the last ones feed the epilogue)
            int got = mbar_wait(&bar, phase, err) ? 1 : 0;
            phase ^= 1u;
            ok = __syncthreads_and(got);
            if (!ok) break;
        }
        if (!ok) break;
        tc_fence_after();
        // epilogue: warpgroup 0 takes the first half of the 16-column
        // groups, warpgroup 1 the rest; lane = neuron j0 + 32 q + lane
        const int j = j0 + 32 * q + lane;
        const int ngrp = npad >> 4;
        const int g_lo = warp < 4 ? 0 : (ngrp + 1) / 2, g_hi = warp < 4 ? (ngrp + 1) / 2 : ngrp;
        for (int g = g_lo; g < g_hi; ++g) {
            uint32_t v[16], w[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * g);
            tmem_ld16(ta, v);
            tmem_ld16(ta + half, w);
            if (j < N) {
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int u = 16 * g + c;
                    if (u < nu) Lb[(long long)(u0 + u) * N + j] = __uint_as_float(v[c]) + __uint_as_float(w[c]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();                  // accumulator read before the next pass overwrites it
        tc_fence_after();
    }
    if (!ok) {
        // a wait gave up (error bit 1 is set): give the MMAs in flight one
        // more bounded wait before the accumulator is released
        mbar_wait(&bar, phase ^ 1u, err);
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

// Warp-specialised form for one error window (batch 1, U <= 128, K <= 128:
// the million-neuron workload's window).  One CTA per SM walks tiles of 128
// neurons; the window's E is split into TF32 hi + lo once and stays in
// shared memory.  Roles run concurrently, joined by mbarriers:
//   warps 4-7  producers: each feedback chunk (128 rows x 32) is loaded
//              (registers one chunk ahead), split and stored into one of two
//              operand stages; arrive on full[stage];
//   warp 8     one thread issues the chunk's products into one of two
//              accumulator pairs in TMEM and commits to empty[stage], and at
//              a tile's end to acc_full[pair];
//   warps 0-3  epilogue: read a finished accumulator pair (TMEM lanes 32 w ..
//              32 w + 31 = the tile's neurons), add hi*hi and the corrections
//              and store L; arrive on acc_empty[pair].
// So the loads, the products and the stores of different tiles overlap.
// The products and their order within a tile are those of
// learning_signal_kernel.  Every wait is bounded; a wait that gives up
// raises a CTA-wide abort flag that every role checks.
constexpr int kLsPKC = 4;                          // K-chunks kept resident (K <= 128)
constexpr int kLsWThreads = 288;                   // 9 warps
constexpr int kLsWStages = 2;
constexpr size_t kLsWSmem = 1024 + (size_t)kLsPKC * 2 * kLsEreg + (size_t)kLsWStages * 2 * kLsAreg;
static_assert(kLsWSmem <= 200 * 1024, "warp-specialised learning-signal buffers exceed the request");

__device__ __forceinline__ void mbar_arrive_cta(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__global__ void __launch_bounds__(kLsWThreads, 1)
    learning_signal_ws_kernel(const float *__restrict__ fb, const float *__restrict__ E, float *__restrict__ L,
                              int N, int U, int K, unsigned *err) {
    extern __shared__ unsigned char ls_raw[];
    __shared__ uint64_t full[kLsWStages], empty[kLsWStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(ls_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *e_base = base;
    unsigned char *a_base = base + (size_t)kLsPKC * 2 * kLsEreg;
    const int nkc = (K + kLsKC - 1) / kLsKC;
    const int tiles = (N + kLsM - 1) / kLsM;
    const int npad = (U + 15) & ~15;
    uint32_t half = 32;
    while ((int)half < npad) half <<= 1;
    const uint32_t ncols = 4 * half;                 // two accumulator pairs
    if (warp == 0) tmem_alloc(&tmem_slot, ncols);
    if (tid == 0) {
        for (int q2 = 0; q2 < kLsWStages; ++q2) {
            mbar_init(&full[q2], 4);                  // one arrival per producer warp
            mbar_init(&empty[q2], 1);                 // the products' commit
        }
        for (int q2 = 0; q2 < 2; ++q2) {
            mbar_init(&acc_full[q2], 1);
            mbar_init(&acc_empty[q2], 4);             // one arrival per epilogue warp
        }
        s_abort = 0;
        fence_mbar_init();
    }
    // the error window, split once (every thread)
    for (int kc = 0; kc < nkc; ++kc) {
        const int k = kc * kLsKC + lane;
        const bool kin = k < K;
        for (int r = warp; r < npad; r += kLsWThreads / 32) {
            const float x = (kin && r < U) ? __ldg(E + (long long)r * K + k) : 0.f;
            put_split(e_base + (size_t)(2 * kc) * kLsEreg, e_base + (size_t)(2 * kc + 1) * kLsEreg,
                      sw128_off(r, lane), x);
        }
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        for (unsigned it2 = 0; it2 < kWaitLimit; ++it2) {
            if (mbar_try_wait(bar, parity)) return true;
            if (s_abort) return false;
        }
        atomicOr(err, 2u);
        s_abort = 1;
        return false;
    };
    long long n_my = 0;                               // tiles of this CTA
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) ++n_my;
    long long last_commit = -1;                       // products: chunks committed
    if (warp >= 4 && warp < 8) {
        // ---- producers: 128 threads, thread (pw, lane) owns rows pw + 4 i
        const int pw = warp - 4;
        float pre[kLsM / 4];
        auto load_chunk = [&](long long c) {
            const long long tl = c / nkc;
            const int kc = (int)(c % nkc);
            const int j0 = (int)(blockIdx.x + tl * gridDim.x) * kLsM;
            const int k = kc * kLsKC + lane;
            const bool use = tl < n_my && k < K;
#pragma unroll
            for (int i = 0; i < kLsM / 4; ++i) {
                const int j = j0 + pw + 4 * i;
                pre[i] = (use && j < N) ? __ldg(fb + (long long)j * K + k) : 0.f;
            }
        };
        const long long nch = n_my * nkc;
        if (nch > 0) load_chunk(0);
        for (long long c = 0; c < nch; ++c) {
            const int st = (int)(c % kLsWStages);
            if (c >= kLsWStages && !wait(&empty[st], (uint32_t)(((c / kLsWStages) - 1) & 1))) break;
            unsigned char *ah = a_base + (size_t)(2 * st) * kLsAreg, *al = a_base + (size_t)(2 * st + 1) * kLsAreg;
#pragma unroll
            for (int i = 0; i < kLsM / 4; ++i) put_split(ah, al, sw128_off(pw + 4 * i, lane), pre[i]);
            if (c + 1 < nch) load_chunk(c + 1);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive_cta(&full[st]);
        }
    } else if (warp == 8) {
        // ---- products: the whole warp follows the barriers (it stays
        // converged), lane 0 issues
        const uint32_t idesc = idesc_tf32(kLsM, npad);
        long long c = 0;
        for (long long tl = 0; tl < n_my; ++tl) {
            const int pair = (int)(tl & 1);
            if (tl >= 2 && !wait(&acc_empty[pair], (uint32_t)(((tl / 2) - 1) & 1))) break;
            tc_fence_after();
            const uint32_t acc_hi = tmem + (uint32_t)pair * 2 * half, acc_lo = acc_hi + half;
            bool okc = true;
            for (int kc = 0; kc < nkc; ++kc, ++c) {
                const int st = (int)(c % kLsWStages);
                if (!wait(&full[st], (uint32_t)((c / kLsWStages) & 1))) { okc = false; break; }
                tc_fence_after();
                if (lane == 0) {
                    const int nks = (min(kLsKC, K - kc * kLsKC) + 7) >> 3;
                    const uint32_t ah = smem_u32(a_base + (size_t)(2 * st) * kLsAreg);
                    const uint32_t al = smem_u32(a_base + (size_t)(2 * st + 1) * kLsAreg);
                    const uint32_t eh = smem_u32(e_base + (size_t)(2 * kc) * kLsEreg);
                    const uint32_t el = smem_u32(e_base + (size_t)(2 * kc + 1) * kLsEreg);
                    uint32_t acc = kc > 0 ? 1u : 0u;
                    for (int s2 = 0; s2 < nks; ++s2) {
                        const uint32_t o = 32u * s2;
                        umma_tf32(acc_hi, sdesc_sw128(ah + o), sdesc_sw128(eh + o), idesc, acc);
                        umma_tf32(acc_lo, sdesc_sw128(ah + o), sdesc_sw128(el + o), idesc, acc);
                        umma_tf32(acc_lo, sdesc_sw128(al + o), sdesc_sw128(eh + o), idesc, 1);
                        acc = 1;
                    }
                    umma_commit(&empty[st]);
                }
                __syncwarp();
                last_commit = c;
            }
            if (!okc) break;
            if (lane == 0) umma_commit(&acc_full[pair]);
            __syncwarp();
        }
    } else if (warp < 4) {
        // ---- epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31
        const int ngrp = npad >> 4;
        for (long long tl = 0; tl < n_my; ++tl) {
            const int pair = (int)(tl & 1);
            if (!wait(&acc_full[pair], (uint32_t)((tl / 2) & 1))) break;
            tc_fence_after();
            const int j = (int)(blockIdx.x + tl * gridDim.x) * kLsM + 32 * warp + lane;
            const uint32_t ta0 = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)pair * 2 * half;
            for (int g = 0; g < ngrp; ++g) {
                uint32_t v[16], w[16];
                tmem_ld16_nowait(ta0 + (uint32_t)(16 * g), v);
                tmem_ld16_nowait(ta0 + half + (uint32_t)(16 * g), w);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (j < N) {
#pragma unroll
                    for (int c2 = 0; c2 < 16; ++c2) {
                        const int u = 16 * g + c2;
                        if (u < U) L[(long long)u * N + j] = __uint_as_float(v[c2]) + __uint_as_float(w[c2]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cta(&acc_empty[pair]);
        }
    }
    // products in flight when a wait gave up: one more bounded wait on the
    // last commit before the accumulators are released
    if (warp == 8 && lane == 0 && s_abort && last_commit >= 0) {
        const int st = (int)(last_commit % kLsWStages);
        for (unsigned it2 = 0; it2 < kWaitLimit; ++it2)
            if (mbar_try_wait(&empty[st], (uint32_t)((last_commit / kLsWStages) & 1))) break;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

void prepare_learning_signal_attributes() {
    cudaFuncSetAttribute(learning_signal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLsSmem);
    cudaFuncSetAttribute(learning_signal_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLsWSmem);
}

void launch_learning_signals(const float *fb, const float *E, float *L, int N, int U, int K, int B,
                             unsigned *err, cudaStream_t st) {
    if (N <= 0 || U <= 0 || K <= 0 || B <= 0) return;
    if (B == 1 && U <= kLsNmax && K <= kLsPKC * kLsKC) {
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int tiles = (N + kLsM - 1) / kLsM;
        learning_signal_ws_kernel<<<tiles < sms ? tiles : sms, kLsWThreads, kLsWSmem, st>>>(fb, E, L, N, U, K, err);
        return;
    }
    const dim3 grid((unsigned)((N + kLsM - 1) / kLsM), (unsigned)B);
    learning_signal_kernel<<<grid, kLsThreads, kLsSmem, st>>>(fb, E, L, N, U, K, err);
}

}  // namespace eprop
