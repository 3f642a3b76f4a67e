// Learned learning-signal predictor: BF16 MLP with FP32 accumulation on the
// tensor cores, trained by Adam, all on the GPU (forward, backward and
// update kernels below).  Semantics and layouts: include/eprop_predictor.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "eprop_predictor.h"
#include "predictor_internal.h"

using bf16 = __nv_bfloat16;

struct eprop_predictor {
    int n_in = 0, hidden = 0, n_out = 0, max_rows = 0;
    long long n_params = 0;
    long long off_W[3] = {0, 0, 0}, off_b[3] = {0, 0, 0};
    cudaStream_t st = nullptr;
    int own_stream = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    bf16 *Wh[3] = {nullptr, nullptr, nullptr};
    bf16 *Xh = nullptr, *H1h = nullptr, *H2h = nullptr, *dYh = nullptr, *dA2h = nullptr, *dA1h = nullptr;
    float *A1 = nullptr, *A2 = nullptr, *Y = nullptr, *dYf = nullptr, *dA2f = nullptr, *dA1f = nullptr;
    float *xin = nullptr, *ein = nullptr, *yout = nullptr, *loss = nullptr;
    float *stage = nullptr;          // FP32 widening of BF16 buffers for eprop_predictor_read
    float *in_scale = nullptr;       // [n_in] input scale (part of the model; default 1)
    long long adam_t = 0;
    int rows = 0;
    std::string err;
    std::vector<void *> allocs;
};

namespace pred {

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * erfcf(-x * 0.70710678118654752f); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * erfcf(-x * 0.70710678118654752f) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// inputs: x * scale[column], rounded to BF16
__global__ void input_bf16_kernel(const float *src, const float *scale, int cols, bf16 *dst, long long n) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x)
        dst[q] = __float2bfloat16_rn(src[q] * scale[q % cols]);
}

__global__ void to_bf16_kernel(const float *src, bf16 *dst, long long n) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x)
        dst[q] = __float2bfloat16_rn(src[q]);
}

// A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn]
struct Gemm {
    const bf16 *A, *B;
    long long sam, sak, sbk, sbn;
    int M, N, K;
    const float *bias;      // [N] or null
    const float *pre;       // [M][N] pre-activation for the GELU derivative
    float *outF;            // [M][N]
    bf16 *outH;             // [M][N]
};

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_DGELU = 3 };

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M][N] = op(A) op(B) with the epilogue EPI.  CTA tile 64 x 32, four warps
// of 16 rows each; K in steps of 16 staged through shared memory (zero
// padded at the edges).  Fragment layouts of m16n8k16 (row.col): lane =
// 4 g + t; A regs (g, 2t..2t+1), (g+8, ..), (g, 2t+8..), (g+8, 2t+8..);
// B regs (2t..2t+1, g), (2t+8.., g); C (g, 2t..2t+1), (g+8, 2t..2t+1).
template <int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(Gemm g) {
    __shared__ bf16 As[64][16 + 8];
    __shared__ bf16 Bs[16][32 + 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 32;
    const int gid = lane >> 2, tig = lane & 3;
    const int rb = warp * 16;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
    const bf16 zero = __float2bfloat16_rn(0.f);
    for (int k0 = 0; k0 < g.K; k0 += 16) {
        for (int q = threadIdx.x; q < 64 * 16; q += 128) {
            const int r = q >> 4, c = q & 15;
            const int m = m0 + r, k = k0 + c;
            As[r][c] = (m < g.M && k < g.K) ? g.A[(long long)m * g.sam + (long long)k * g.sak] : zero;
        }
        for (int q = threadIdx.x; q < 16 * 32; q += 128) {
            const int r = q >> 5, c = q & 31;
            const int k = k0 + r, nn = n0 + c;
            Bs[r][c] = (k < g.K && nn < g.N) ? g.B[(long long)k * g.sbk + (long long)nn * g.sbn] : zero;
        }
        __syncthreads();
        uint32_t a[4];
        a[0] = pack2(As[rb + gid][2 * tig], As[rb + gid][2 * tig + 1]);
        a[1] = pack2(As[rb + gid + 8][2 * tig], As[rb + gid + 8][2 * tig + 1]);
        a[2] = pack2(As[rb + gid][2 * tig + 8], As[rb + gid][2 * tig + 9]);
        a[3] = pack2(As[rb + gid + 8][2 * tig + 8], As[rb + gid + 8][2 * tig + 9]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t b[2];
            b[0] = pack2(Bs[2 * tig][j * 8 + gid], Bs[2 * tig + 1][j * 8 + gid]);
            b[1] = pack2(Bs[2 * tig + 8][j * 8 + gid], Bs[2 * tig + 9][j * 8 + gid]);
            mma_bf16(acc[j], a, b);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int m = m0 + rb + gid + (e >= 2 ? 8 : 0);
            const int nn = n0 + j * 8 + 2 * tig + (e & 1);
            if (m >= g.M || nn >= g.N) continue;
            const long long o = (long long)m * g.N + nn;
            float x = acc[j][e];
            if (EPI == EPI_BIAS || EPI == EPI_BIAS_GELU) x += g.bias[nn];
            if (EPI == EPI_DGELU) x *= gelu_grad(g.pre[o]);
            g.outF[o] = x;
            if (EPI == EPI_BIAS_GELU) g.outH[o] = __float2bfloat16_rn(gelu(x));
            if (EPI == EPI_DGELU) g.outH[o] = __float2bfloat16_rn(x);
        }
}

// dY = (Y - E) / R (FP32 and BF16) and the batch loss (1 / (2 R)) sum (Y -
// E)^2, one block, fixed summation order
__global__ void loss_grad_kernel(const float *Y, const float *E, long long count, int R, float *dYf,
                                 bf16 *dYh, float *loss) {
    __shared__ float part[256];
    const float inv = 1.0f / (float)R;
    float s = 0.f;
    for (long long q = threadIdx.x; q < count; q += blockDim.x) {
        const float d = Y[q] - E[q];
        s = fmaf(d, d, s);
        dYf[q] = d * inv;
        dYh[q] = __float2bfloat16_rn(d * inv);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = 0.5f * part[0] * inv;
}

// out[n] = sum over rows of D[r][n] in row order (deterministic)
__global__ void colsum_kernel(const float *D, int R, int N, float *out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int r = 0; r < R; ++r) s += D[(long long)r * N + n];
    out[n] = s;
}

// Adam (Eq. adam1, Eq. adam2, Eq. adam) on the FP32 masters
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, long long n, float lr, float c1,
                            float c2) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = 0.9f * m[q] + 0.1f * gq;
        const float vq = 0.999f * v[q] + 0.001f * gq * gq;
        m[q] = mq;
        v[q] = vq;
        w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + 1e-8f);
    }
}

__global__ void bf16_to_float_kernel(const bf16 *src, float *dst, long long n) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x)
        dst[q] = __bfloat162float(src[q]);
}

// ------------------------------------------------------------------ host

template <int EPI>
static void gemm(cudaStream_t st, const Gemm &g) {
    const dim3 grid((g.M + 63) / 64, (g.N + 31) / 32);
    gemm_kernel<EPI><<<grid, 128, 0, st>>>(g);
}

static unsigned blocks_for(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

static uint64_t splitmix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

}  // namespace pred

using namespace pred;

static eprop_status pfail(eprop_predictor *p, eprop_status s, const char *msg) {
    if (p) p->err = msg;
    return s;
}

static eprop_status pcuda(eprop_predictor *p, cudaError_t e, const char *what) {
    if (p) p->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? EPROP_ENOMEM : EPROP_ECUDA;
}

#define PCK(p, call)                                          \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return pcuda((p), _e, #call);  \
    } while (0)

template <typename T>
static cudaError_t palloc(eprop_predictor *p, T **ptr, long long count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, (size_t)(count > 0 ? count : 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    p->allocs.push_back(q);
    *ptr = static_cast<T *>(q);
    return cudaMemset(q, 0, (size_t)(count > 0 ? count : 1) * sizeof(T));
}

static thread_local std::string g_pred_create_err;

extern "C" eprop_status eprop_predictor_create(int32_t n_in, int32_t hidden, int32_t n_out, int32_t max_rows,
                                               const float *params, uint64_t seed, void *stream,
                                               eprop_predictor **out) {
    if (!out) return EPROP_EINVAL;
    *out = nullptr;
    if (n_in < 1 || n_in > 1024 || n_out < 1 || n_out > 1024 || hidden < 16 || hidden > 1024 || max_rows < 1 ||
        max_rows > 65536) {
        g_pred_create_err = "predictor sizes out of range";
        return EPROP_EINVAL;
    }
    eprop_predictor *p = new eprop_predictor();
    p->n_in = n_in;
    p->hidden = hidden;
    p->n_out = n_out;
    p->max_rows = max_rows;
    const int fan_in[3] = {n_in, hidden, hidden}, fan_out[3] = {hidden, hidden, n_out};
    long long o = 0;
    for (int l = 0; l < 3; ++l) {
        p->off_W[l] = o;
        o += (long long)fan_in[l] * fan_out[l];
        p->off_b[l] = o;
        o += fan_out[l];
    }
    p->n_params = o;
    eprop_status s = EPROP_OK;
    cudaError_t e = cudaSuccess;
    if (stream) {
        p->st = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking);
        p->own_stream = 1;
    }
    const long long R = max_rows, H = hidden;
    if (e == cudaSuccess) e = palloc(p, &p->params, o);
    if (e == cudaSuccess) e = palloc(p, &p->grads, o);
    if (e == cudaSuccess) e = palloc(p, &p->m, o);
    if (e == cudaSuccess) e = palloc(p, &p->v, o);
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) e = palloc(p, &p->Wh[l], (long long)fan_in[l] * fan_out[l]);
    if (e == cudaSuccess) e = palloc(p, &p->Xh, R * n_in);
    if (e == cudaSuccess) e = palloc(p, &p->H1h, R * H);
    if (e == cudaSuccess) e = palloc(p, &p->H2h, R * H);
    if (e == cudaSuccess) e = palloc(p, &p->dYh, R * n_out);
    if (e == cudaSuccess) e = palloc(p, &p->dA2h, R * H);
    if (e == cudaSuccess) e = palloc(p, &p->dA1h, R * H);
    if (e == cudaSuccess) e = palloc(p, &p->A1, R * H);
    if (e == cudaSuccess) e = palloc(p, &p->A2, R * H);
    if (e == cudaSuccess) e = palloc(p, &p->Y, R * n_out);
    if (e == cudaSuccess) e = palloc(p, &p->dYf, R * n_out);
    if (e == cudaSuccess) e = palloc(p, &p->dA2f, R * H);
    if (e == cudaSuccess) e = palloc(p, &p->dA1f, R * H);
    if (e == cudaSuccess) e = palloc(p, &p->xin, R * n_in);
    if (e == cudaSuccess) e = palloc(p, &p->ein, R * n_out);
    if (e == cudaSuccess) e = palloc(p, &p->yout, R * n_out);
    if (e == cudaSuccess) e = palloc(p, &p->loss, 1);
    if (e == cudaSuccess) e = palloc(p, &p->stage, R * (H > n_in ? (H > n_out ? H : n_out) : (n_in > n_out ? n_in : n_out)));
    if (e == cudaSuccess) e = palloc(p, &p->in_scale, n_in);
    if (e == cudaSuccess) {
        std::vector<float> ones((size_t)n_in, 1.0f);
        e = cudaMemcpy(p->in_scale, ones.data(), (size_t)n_in * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        g_pred_create_err = std::string("predictor allocation: ") + cudaGetErrorString(e);
        eprop_predictor_destroy(p);
        return e == cudaErrorMemoryAllocation ? EPROP_ENOMEM : EPROP_ECUDA;
    }
    std::vector<float> init;
    if (!params) {
        init.assign((size_t)o, 0.f);
        for (int l = 0; l < 3; ++l) {
            const double sd = 1.0 / std::sqrt((double)fan_in[l]);
            const long long cnt = (long long)fan_in[l] * fan_out[l];
            for (long long q = 0; q < cnt; ++q) {
                const uint64_t h1 = splitmix(seed ^ splitmix((uint64_t)(p->off_W[l] + q) * 2 + 0));
                const uint64_t h2 = splitmix(seed ^ splitmix((uint64_t)(p->off_W[l] + q) * 2 + 1));
                const double u1 = ((double)(h1 >> 11) + 1.0) * (1.0 / 9007199254740992.0);
                const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
                init[(size_t)(p->off_W[l] + q)] =
                    (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
            }
        }
        params = init.data();
    }
    s = eprop_predictor_set_params(p, params);
    if (s != EPROP_OK) {
        g_pred_create_err = p->err;
        eprop_predictor_destroy(p);
        return s;
    }
    *out = p;
    return EPROP_OK;
}

extern "C" int64_t eprop_predictor_num_params(const eprop_predictor *p) { return p ? p->n_params : 0; }

static void refresh_weights(eprop_predictor *p) {
    const long long cnt[3] = {(long long)p->n_in * p->hidden, (long long)p->hidden * p->hidden,
                              (long long)p->hidden * p->n_out};
    for (int l = 0; l < 3; ++l)
        to_bf16_kernel<<<blocks_for(cnt[l]), 256, 0, p->st>>>(p->params + p->off_W[l], p->Wh[l], cnt[l]);
}

extern "C" eprop_status eprop_predictor_set_params(eprop_predictor *p, const float *params) {
    if (!p || !params) return EPROP_EINVAL;
    PCK(p, cudaMemcpyAsync(p->params, params, (size_t)p->n_params * 4, cudaMemcpyHostToDevice, p->st));
    PCK(p, cudaMemsetAsync(p->m, 0, (size_t)p->n_params * 4, p->st));
    PCK(p, cudaMemsetAsync(p->v, 0, (size_t)p->n_params * 4, p->st));
    p->adam_t = 0;
    refresh_weights(p);
    PCK(p, cudaGetLastError());
    PCK(p, cudaStreamSynchronize(p->st));
    return EPROP_OK;
}

// forward on x already on the device (FP32 [rows][n_in]); leaves Y in p->Y
static void issue_forward(eprop_predictor *p, const float *x, int rows, cudaStream_t st) {
    const int H = p->hidden;
    input_bf16_kernel<<<blocks_for((long long)rows * p->n_in), 256, 0, st>>>(x, p->in_scale, p->n_in, p->Xh,
                                                                            (long long)rows * p->n_in);
    Gemm g{};
    g.A = p->Xh; g.sam = p->n_in; g.sak = 1;
    g.B = p->Wh[0]; g.sbk = H; g.sbn = 1;
    g.M = rows; g.N = H; g.K = p->n_in;
    g.bias = p->params + p->off_b[0]; g.outF = p->A1; g.outH = p->H1h;
    gemm<EPI_BIAS_GELU>(st, g);
    g = Gemm{};
    g.A = p->H1h; g.sam = H; g.sak = 1;
    g.B = p->Wh[1]; g.sbk = H; g.sbn = 1;
    g.M = rows; g.N = H; g.K = H;
    g.bias = p->params + p->off_b[1]; g.outF = p->A2; g.outH = p->H2h;
    gemm<EPI_BIAS_GELU>(st, g);
    g = Gemm{};
    g.A = p->H2h; g.sam = H; g.sak = 1;
    g.B = p->Wh[2]; g.sbk = p->n_out; g.sbn = 1;
    g.M = rows; g.N = p->n_out; g.K = H;
    g.bias = p->params + p->off_b[2]; g.outF = p->Y;
    gemm<EPI_BIAS>(st, g);
    p->rows = rows;
}

const float *predictor_issue_forward(eprop_predictor *p, const float *x_dev, int rows, cudaStream_t st) {
    issue_forward(p, x_dev, rows, st);
    return p->Y;
}

void predictor_dims(const eprop_predictor *p, int *n_in, int *n_out, int *max_rows) {
    *n_in = p->n_in;
    *n_out = p->n_out;
    *max_rows = p->max_rows;
}

extern "C" eprop_status eprop_predictor_forward(eprop_predictor *p, const float *x, int32_t rows, float *y,
                                                int32_t is_device) {
    if (!p || !x || !y) return EPROP_EINVAL;
    if (rows < 1 || rows > p->max_rows) return pfail(p, EPROP_EINVAL, "rows out of range");
    const float *xd = x;
    if (!is_device) {
        PCK(p, cudaMemcpyAsync(p->xin, x, (size_t)rows * p->n_in * 4, cudaMemcpyHostToDevice, p->st));
        xd = p->xin;
    }
    issue_forward(p, xd, rows, p->st);
    PCK(p, cudaGetLastError());
    PCK(p, cudaMemcpyAsync(y, p->Y, (size_t)rows * p->n_out * 4,
                           is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->st));
    if (!is_device) PCK(p, cudaStreamSynchronize(p->st));
    return EPROP_OK;
}

extern "C" eprop_status eprop_predictor_train_step(eprop_predictor *p, const float *x, const float *e,
                                                   int32_t rows, float lr, float *loss_out, int32_t is_device) {
    if (!p || !x || !e) return EPROP_EINVAL;
    if (rows < 1 || rows > p->max_rows) return pfail(p, EPROP_EINVAL, "rows out of range");
    const int H = p->hidden, K = p->n_out, I = p->n_in;
    const float *xd = x, *ed = e;
    if (!is_device) {
        PCK(p, cudaMemcpyAsync(p->xin, x, (size_t)rows * I * 4, cudaMemcpyHostToDevice, p->st));
        PCK(p, cudaMemcpyAsync(p->ein, e, (size_t)rows * K * 4, cudaMemcpyHostToDevice, p->st));
        xd = p->xin;
        ed = p->ein;
    }
    issue_forward(p, xd, rows, p->st);
    loss_grad_kernel<<<1, 256, 0, p->st>>>(p->Y, ed, (long long)rows * K, rows, p->dYf, p->dYh, p->loss);
    Gemm g{};
    // dW3 = H2^T dY
    g.A = p->H2h; g.sam = 1; g.sak = H;
    g.B = p->dYh; g.sbk = K; g.sbn = 1;
    g.M = H; g.N = K; g.K = rows; g.outF = p->grads + p->off_W[2];
    gemm<EPI_STORE>(p->st, g);
    colsum_kernel<<<(K + 127) / 128, 128, 0, p->st>>>(p->dYf, rows, K, p->grads + p->off_b[2]);
    // dA2 = (dY W3^T) * GELU'(A2)
    g = Gemm{};
    g.A = p->dYh; g.sam = K; g.sak = 1;
    g.B = p->Wh[2]; g.sbk = 1; g.sbn = K;
    g.M = rows; g.N = H; g.K = K; g.pre = p->A2; g.outF = p->dA2f; g.outH = p->dA2h;
    gemm<EPI_DGELU>(p->st, g);
    // dW2 = H1^T dA2
    g = Gemm{};
    g.A = p->H1h; g.sam = 1; g.sak = H;
    g.B = p->dA2h; g.sbk = H; g.sbn = 1;
    g.M = H; g.N = H; g.K = rows; g.outF = p->grads + p->off_W[1];
    gemm<EPI_STORE>(p->st, g);
    colsum_kernel<<<(H + 127) / 128, 128, 0, p->st>>>(p->dA2f, rows, H, p->grads + p->off_b[1]);
    // dA1 = (dA2 W2^T) * GELU'(A1)
    g = Gemm{};
    g.A = p->dA2h; g.sam = H; g.sak = 1;
    g.B = p->Wh[1]; g.sbk = 1; g.sbn = H;
    g.M = rows; g.N = H; g.K = H; g.pre = p->A1; g.outF = p->dA1f; g.outH = p->dA1h;
    gemm<EPI_DGELU>(p->st, g);
    // dW1 = X^T dA1
    g = Gemm{};
    g.A = p->Xh; g.sam = 1; g.sak = I;
    g.B = p->dA1h; g.sbk = H; g.sbn = 1;
    g.M = I; g.N = H; g.K = rows; g.outF = p->grads + p->off_W[0];
    gemm<EPI_STORE>(p->st, g);
    colsum_kernel<<<(H + 127) / 128, 128, 0, p->st>>>(p->dA1f, rows, H, p->grads + p->off_b[0]);
    // Adam step
    p->adam_t += 1;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)p->adam_t));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)p->adam_t));
    adam_kernel<<<blocks_for(p->n_params), 256, 0, p->st>>>(p->params, p->grads, p->m, p->v, p->n_params, lr, c1,
                                                             c2);
    refresh_weights(p);
    PCK(p, cudaGetLastError());
    if (loss_out) {
        PCK(p, cudaMemcpyAsync(loss_out, p->loss, 4, cudaMemcpyDeviceToHost, p->st));
        PCK(p, cudaStreamSynchronize(p->st));
    }
    return EPROP_OK;
}

extern "C" eprop_status eprop_predictor_read(eprop_predictor *p, int32_t which, float *dst, int64_t count) {
    if (!p || !dst) return EPROP_EINVAL;
    const long long R = p->rows, H = p->hidden, K = p->n_out;
    const float *srcF = nullptr;
    const bf16 *srcH = nullptr;
    long long n = 0;
    switch (which) {
        case 0: srcF = p->params; n = p->n_params; break;
        case 1: srcF = p->grads; n = p->n_params; break;
        case 2: srcF = p->A1; n = R * H; break;
        case 3: srcH = p->H1h; n = R * H; break;
        case 4: srcF = p->A2; n = R * H; break;
        case 5: srcH = p->H2h; n = R * H; break;
        case 6: srcF = p->Y; n = R * K; break;
        case 7: srcH = p->dYh; n = R * K; break;
        case 8: srcH = p->dA2h; n = R * H; break;
        case 9: srcH = p->dA1h; n = R * H; break;
        case 10: srcF = p->m; n = p->n_params; break;
        case 11: srcF = p->v; n = p->n_params; break;
        case 12: srcH = p->Xh; n = R * p->n_in; break;
        default: return pfail(p, EPROP_EINVAL, "unknown buffer");
    }
    if (count < n) return pfail(p, EPROP_EINVAL, "destination too small");
    if (srcH) {
        bf16_to_float_kernel<<<blocks_for(n), 256, 0, p->st>>>(srcH, p->stage, n);
        PCK(p, cudaGetLastError());
        PCK(p, cudaMemcpyAsync(dst, p->stage, (size_t)n * 4, cudaMemcpyDeviceToHost, p->st));
    } else {
        PCK(p, cudaMemcpyAsync(dst, srcF, (size_t)n * 4, cudaMemcpyDeviceToHost, p->st));
    }
    PCK(p, cudaStreamSynchronize(p->st));
    return EPROP_OK;
}

extern "C" eprop_status eprop_predictor_set_input_scale(eprop_predictor *p, const float *scale) {
    if (!p || !scale) return EPROP_EINVAL;
    PCK(p, cudaStreamSynchronize(p->st));
    PCK(p, cudaMemcpy(p->in_scale, scale, (size_t)p->n_in * 4, cudaMemcpyHostToDevice));
    return EPROP_OK;
}

extern "C" eprop_status eprop_predictor_sync(eprop_predictor *p) {
    if (!p) return EPROP_EINVAL;
    PCK(p, cudaStreamSynchronize(p->st));
    PCK(p, cudaGetLastError());
    return EPROP_OK;
}

extern "C" void eprop_predictor_destroy(eprop_predictor *p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    for (void *q : p->allocs) cudaFree(q);
    if (p->own_stream && p->st) cudaStreamDestroy(p->st);
    delete p;
}

extern "C" const char *eprop_predictor_last_error(const eprop_predictor *p) {
    return p ? p->err.c_str() : g_pred_create_err.c_str();
}
