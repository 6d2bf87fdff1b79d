// Small BF16 multilayer perceptron with FP32 accumulation for the learned
// warm start: hand-written inference and training kernels on the tensor
// cores (mma.sync m16n8k16 BF16 -> FP32).
//
// Network: 16 inputs (the caller's features, zero-padded) -> 3 hidden layers
// of 128 tanh units -> 16 outputs (zero-padded; linear).  Each layer keeps
// FP32 master weights (Adam state beside them) and two BF16 copies: W^T
// [n][k] for the forward product and W [k][n] for back-propagation.
//
// One CTA of 4 warps handles 64 samples; each warp owns 16 samples (the M
// dimension of the MMA).  Training is full-batch gradient descent: a CTA
// back-propagates its samples and adds its weight gradients into FP32
// accumulators with atomics; the Adam kernel then updates every weight.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <new>
#include <string>

#include "../../include/cplbm.h"
#include "cplbm_internal.h"  // dev_alloc / dev_free
#include "trace.h"

namespace cplbm_mlp {

constexpr int DIN = 16, H = 128, DOUT = 16, NL = 4;
constexpr int SAMPLES = 64, WARPS = 4, THREADS = 32 * WARPS;
__host__ __device__ constexpr int layer_k(int l) { return l == 0 ? DIN : H; }
__host__ __device__ constexpr int layer_n(int l) { return l == NL - 1 ? DOUT : H; }

// Offsets of layer l's weights [k][n] and biases in the flat parameter
// arrays (FP32 masters, gradients, Adam moments share the layout).
__host__ __device__ constexpr int w_off(int l)
{
    return l == 0 ? 0 : w_off(l - 1) + layer_k(l - 1) * layer_n(l - 1);
}
constexpr int NW = w_off(NL);
__host__ __device__ constexpr int b_off(int l)
{
    return l == 0 ? NW : b_off(l - 1) + layer_n(l - 1);
}
constexpr int NPARAM = b_off(NL);

struct Params {
    const __nv_bfloat16 *wt;  // W^T [n][k] per layer, BF16, at w_off(l)
    const __nv_bfloat16 *w;   // W [k][n] per layer, BF16, at w_off(l)
    const float *p;           // FP32 masters (biases read from here)
};

// ---------------------------------------------------------------------------
// Warp-level GEMM: acc[16 x N] += A[16 x K] * B[K x N].  A row-major in
// shared memory (lda elements per row), B given as Bt[n][k] (ldb per n).
// Fragment layouts of mma.m16n8k16 (PTX ISA): lane = 4 g + t.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_pair(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const unsigned *>(p);
}

template <int K, int N>
__device__ __forceinline__ void warp_gemm(const __nv_bfloat16 *A, int lda,
                                          const __nv_bfloat16 *Bt, int ldb,
                                          float (&acc)[N / 8][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16) {
        const unsigned a0 = ld_pair(A + g * lda + k0 + 2 * t);
        const unsigned a1 = ld_pair(A + (g + 8) * lda + k0 + 2 * t);
        const unsigned a2 = ld_pair(A + g * lda + k0 + 8 + 2 * t);
        const unsigned a3 = ld_pair(A + (g + 8) * lda + k0 + 8 + 2 * t);
#pragma unroll
        for (int j = 0; j < N / 8; ++j) {
            const __nv_bfloat16 *bp = Bt + (j * 8 + g) * ldb + k0 + 2 * t;
            const unsigned b0 = ld_pair(bp), b1 = ld_pair(bp + 8);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                "{%0, %1, %2, %3};\n"
                : "+f"(acc[j][0]), "+f"(acc[j][1]), "+f"(acc[j][2]), "+f"(acc[j][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
}

// Element (row, col) held by accumulator slot q of n-tile j.
__device__ __forceinline__ void acc_pos(int j, int q, int &row, int &col)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    row = g + (q >= 2 ? 8 : 0);
    col = j * 8 + 2 * t + (q & 1);
}

// Shared memory of one CTA.
struct Smem {
    __nv_bfloat16 wt[H * H];                // current layer's Bt operand
    __nv_bfloat16 act[NL][SAMPLES * H];     // inputs of layer l, [s][k]
    __nv_bfloat16 actT[NL][H * SAMPLES];    // the same, [k][s]
    __nv_bfloat16 dlt[SAMPLES * H];         // delta of the current layer [s][n]
    __nv_bfloat16 dltT[H * SAMPLES];        // [n][s]
    float out[SAMPLES * DOUT];
};

__device__ void load_bt(__nv_bfloat16 *dst, const __nv_bfloat16 *src, int n)
{
    for (int q = threadIdx.x; q < n; q += THREADS) dst[q] = src[q];
}

// Forward pass of the CTA's 64 samples; stores every layer's input
// (row-major and transposed) and the FP32 outputs.
__device__ void forward(const Params &P, Smem &S)
{
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        constexpr int dummy = 0;
        (void)dummy;
        const int K = layer_k(l), N = layer_n(l);
        load_bt(S.wt, P.wt + w_off(l), K * N);
        __syncthreads();
        const __nv_bfloat16 *A = S.act[l] + warp * 16 * K;
        if (N == H) {
            float acc[H / 8][4] = {};
            if (K == DIN) warp_gemm<DIN, H>(A, K, S.wt, K, acc);
            else warp_gemm<H, H>(A, K, S.wt, K, acc);
#pragma unroll
            for (int j = 0; j < H / 8; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int r, c;
                    acc_pos(j, q, r, c);
                    const float v = tanhf(acc[j][q] + P.p[b_off(l) + c]);
                    const int s = warp * 16 + r;
                    const __nv_bfloat16 bv = __float2bfloat16(v);
                    S.act[l + 1][s * H + c] = bv;
                    S.actT[l + 1][c * SAMPLES + s] = bv;
                }
        } else {
            float acc[DOUT / 8][4] = {};
            warp_gemm<H, DOUT>(A, K, S.wt, K, acc);
#pragma unroll
            for (int j = 0; j < DOUT / 8; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    int r, c;
                    acc_pos(j, q, r, c);
                    S.out[(warp * 16 + r) * DOUT + c] = acc[j][q] + P.p[b_off(l) + c];
                }
        }
        __syncthreads();
    }
}

__device__ void load_inputs(Smem &S, const float *X, int nin, int B, int s0)
{
    for (int q = threadIdx.x; q < SAMPLES * DIN; q += THREADS) {
        const int s = q / DIN, k = q % DIN, gs = s0 + s;
        const float v = (gs < B && k < nin) ? X[(long long)gs * nin + k] : 0.f;
        const __nv_bfloat16 bv = __float2bfloat16(v);
        S.act[0][s * DIN + k] = bv;
        S.actT[0][k * SAMPLES + s] = bv;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(THREADS)
    mlp_infer_kernel(Params P, const float *X, int nin, float *Y, int nout, int B)
{
    extern __shared__ __align__(16) unsigned char raw[];
    Smem &S = *reinterpret_cast<Smem *>(raw);
    const int s0 = blockIdx.x * SAMPLES;
    load_inputs(S, X, nin, B, s0);
    forward(P, S);
    for (int q = threadIdx.x; q < SAMPLES * nout; q += THREADS) {
        const int s = q / nout, c = q % nout;
        if (s0 + s < B) Y[(long long)(s0 + s) * nout + c] = S.out[s * DOUT + c];
    }
}

// Forward, mean-squared-error gradient, back-propagation and weight
// gradients of the CTA's samples; gradients are added into grad (FP32, the
// parameter layout) and the squared error into *loss.
__global__ void __launch_bounds__(THREADS)
    mlp_train_kernel(Params P, const float *X, int nin, const float *T, int nout,
                     int B, float *grad, float *loss)
{
    extern __shared__ __align__(16) unsigned char raw[];
    Smem &S = *reinterpret_cast<Smem *>(raw);
    const int s0 = blockIdx.x * SAMPLES, warp = threadIdx.x >> 5;
    load_inputs(S, X, nin, B, s0);
    forward(P, S);
    // output delta: d(mean sq error)/dy = 2 (y - t) / (B nout)
    float se = 0.f;
    for (int q = threadIdx.x; q < SAMPLES * DOUT; q += THREADS) {
        const int s = q / DOUT, c = q % DOUT, gs = s0 + s;
        float d = 0.f;
        if (gs < B && c < nout) {
            const float e = S.out[q] - T[(long long)gs * nout + c];
            se += e * e;
            d = 2.f * e / (float)(B * nout);
        }
        const __nv_bfloat16 bd = __float2bfloat16(d);
        S.dlt[s * DOUT + c] = bd;
        S.dltT[c * SAMPLES + s] = bd;
        if (c < DOUT) atomicAdd(&grad[b_off(NL - 1) + c], d);
    }
    for (int o = 16; o > 0; o >>= 1) se += __shfl_down_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, se);
    __syncthreads();
    for (int l = NL - 1; l >= 0; --l) {
        const int K = layer_k(l), N = layer_n(l);
        // weight gradient dW[k][n] = sum_s act_l[s][k] dlt[s][n]:
        // rows k (16 per warp-pass), contraction over the 64 samples
        for (int kb = warp * 16; kb < K; kb += WARPS * 16) {
            const __nv_bfloat16 *A = S.actT[l] + kb * SAMPLES;
            if (N == H) {
                float acc[H / 8][4] = {};
                warp_gemm<SAMPLES, H>(A, SAMPLES, S.dltT, SAMPLES, acc);
#pragma unroll
                for (int j = 0; j < H / 8; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        int r, c;
                        acc_pos(j, q, r, c);
                        atomicAdd(&grad[w_off(l) + (kb + r) * N + c], acc[j][q]);
                    }
            } else {
                float acc[DOUT / 8][4] = {};
                warp_gemm<SAMPLES, DOUT>(A, SAMPLES, S.dltT, SAMPLES, acc);
#pragma unroll
                for (int j = 0; j < DOUT / 8; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        int r, c;
                        acc_pos(j, q, r, c);
                        atomicAdd(&grad[w_off(l) + (kb + r) * N + c], acc[j][q]);
                    }
            }
        }
        if (l == 0) break;
        // delta of the layer below: (dlt W^T) * (1 - a^2), a = act[l]
        load_bt(S.wt, P.w + w_off(l), K * N);  // W [k][n]: Bt for this product
        __syncthreads();
        float acc[H / 8][4] = {};
        const __nv_bfloat16 *A = S.dlt + warp * 16 * N;
        if (N == H) warp_gemm<H, H>(A, N, S.wt, N, acc);
        else warp_gemm<DOUT, H>(A, N, S.wt, N, acc);
        __syncthreads();  // every warp has read dlt and wt
#pragma unroll
        for (int j = 0; j < H / 8; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int r, c;
                acc_pos(j, q, r, c);
                const int s = warp * 16 + r;
                const float a = __bfloat162float(S.act[l][s * H + c]);
                const float d = (s0 + s < B) ? acc[j][q] * (1.f - a * a) : 0.f;
                const __nv_bfloat16 bd = __float2bfloat16(d);
                S.dlt[s * H + c] = bd;
                S.dltT[c * SAMPLES + s] = bd;
            }
        __syncthreads();
        // bias gradient of layer l - 1: column sums of the new delta
        for (int c = threadIdx.x; c < H; c += THREADS) {
            float sum = 0.f;
            for (int s = 0; s < SAMPLES; ++s) sum += __bfloat162float(S.dlt[s * H + c]);
            atomicAdd(&grad[b_off(l - 1) + c], sum);
        }
        __syncthreads();
    }
}

// Adam step on the FP32 masters, then the BF16 copies; clears grad.
__global__ void mlp_adam_kernel(float *p, float *grad, float *m, float *v,
                                __nv_bfloat16 *wt, __nv_bfloat16 *w, float lr,
                                float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float g = grad[i];
    m[i] = b1 * m[i] + (1.f - b1) * g;
    v[i] = b2 * v[i] + (1.f - b2) * g * g;
    p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
    grad[i] = 0.f;
    if (i < NW) {
        int l = 0;
        while (l + 1 < NL && i >= w_off(l + 1)) ++l;
        const int K = layer_k(l), N = layer_n(l), local = i - w_off(l);
        const int k = local / N, n = local % N;
        w[i] = __float2bfloat16(p[i]);
        wt[w_off(l) + n * K + k] = __float2bfloat16(p[i]);
    }
}

}  // namespace cplbm_mlp

using namespace cplbm_mlp;
using cplbm::dev_alloc;
using cplbm::dev_free;

struct lbm_mlp {
    float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float *loss = nullptr;
    __nv_bfloat16 *wt = nullptr, *w = nullptr;
    int device = 0;
    long long steps = 0;
    std::string err;
};

namespace {
thread_local std::string g_mlp_err;

lbm_status mfail(lbm_mlp *m, lbm_status s, const char *msg, cudaError_t e)
{
    std::string t = msg;
    if (e != cudaSuccess) t += std::string(": ") + cudaGetErrorString(e);
    (m ? m->err : g_mlp_err) = t;
    return s;
}

#define MCUDA(m, call, msg)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return mfail((m), LBM_ERR_CUDA, msg, e_); \
    } while (0)

Params params_of(const lbm_mlp *m) { return Params{m->wt, m->w, m->p}; }

lbm_status smem_attr(lbm_mlp *m)
{
    static int configured = -1;
    int dev = 0;
    MCUDA(m, cudaGetDevice(&dev), "cudaGetDevice");
    if (configured == dev) return LBM_OK;
    MCUDA(m, cudaFuncSetAttribute(mlp_infer_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(Smem)), "mlp smem");
    MCUDA(m, cudaFuncSetAttribute(mlp_train_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(Smem)), "mlp smem");
    configured = dev;
    return LBM_OK;
}
}  // namespace

extern "C" {

int lbm_mlp_param_count(void) { return NPARAM; }

lbm_status lbm_mlp_create(int device, const float *init, lbm_mlp **out)
{
    if (out) *out = nullptr;
    if (!out || !init) {
        g_mlp_err = "null argument";
        return LBM_ERR_ARG;
    }
    lbm_mlp *m = new (std::nothrow) lbm_mlp();
    if (!m) return LBM_ERR_OOM;
    m->device = device;
    cudaError_t e = cudaSetDevice(device);
    const size_t fb = NPARAM * sizeof(float);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->p, fb);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->grad, fb);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->m, fb);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->v, fb);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->loss, sizeof(float));
    if (e == cudaSuccess) e = dev_alloc((void **)&m->wt, NW * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = dev_alloc((void **)&m->w, NW * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemcpy(m->p, init, fb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->grad, 0, fb);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, fb);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, fb);
    if (e == cudaSuccess) {
        // BF16 copies of the initial weights: an Adam step with lr = 0
        mlp_adam_kernel<<<(NPARAM + 255) / 256, 256>>>(m->p, m->grad, m->m, m->v,
                                                       m->wt, m->w, 0.f, 0.9f,
                                                       0.999f, 1e-8f, 1.f, 1.f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_mlp_err = std::string("mlp create: ") + cudaGetErrorString(e);
        lbm_mlp_destroy(m);
        return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    }
    *out = m;
    return LBM_OK;
}

lbm_status lbm_mlp_train(lbm_mlp *m, const float *X, int nin, const float *T,
                         int nout, int B, int iters, float lr, float *loss_out)
{
    CPLBM_TRACE("lbm_mlp_train");
    if (!m) return LBM_ERR_ARG;
    if (!X || !T || B <= 0 || nin < 1 || nin > DIN || nout < 1 || nout > DOUT ||
        iters < 0 || !(lr >= 0))
        return mfail(m, LBM_ERR_ARG, "bad training arguments", cudaSuccess);
    MCUDA(m, cudaSetDevice(m->device), "cudaSetDevice");
    lbm_status st = smem_attr(m);
    if (st != LBM_OK) return st;
    const int blocks = (B + SAMPLES - 1) / SAMPLES;
    float loss = 0.f;
    for (int it = 0; it < iters; ++it) {
        MCUDA(m, cudaMemsetAsync(m->loss, 0, sizeof(float)), "memset");
        mlp_train_kernel<<<blocks, THREADS, sizeof(Smem)>>>(params_of(m), X, nin,
                                                           T, nout, B, m->grad,
                                                           m->loss);
        MCUDA(m, cudaGetLastError(), "mlp train launch");
        ++m->steps;
        const float c1 = 1.f - std::pow(0.9f, (float)m->steps);
        const float c2 = 1.f - std::pow(0.999f, (float)m->steps);
        mlp_adam_kernel<<<(NPARAM + 255) / 256, 256>>>(m->p, m->grad, m->m, m->v,
                                                       m->wt, m->w, lr, 0.9f,
                                                       0.999f, 1e-8f, c1, c2);
        MCUDA(m, cudaGetLastError(), "mlp adam launch");
    }
    MCUDA(m, cudaMemcpy(&loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost),
          "loss copy");
    if (loss_out) *loss_out = loss / (float)(B * nout);
    return LBM_OK;
}

lbm_status lbm_mlp_gradient(lbm_mlp *m, const float *X, int nin, const float *T,
                            int nout, int B, float *grad, float *loss_out)
{
    CPLBM_TRACE("lbm_mlp_gradient");
    if (!m) return LBM_ERR_ARG;
    if (!X || !T || !grad || B <= 0 || nin < 1 || nin > DIN || nout < 1 || nout > DOUT)
        return mfail(m, LBM_ERR_ARG, "bad gradient arguments", cudaSuccess);
    MCUDA(m, cudaSetDevice(m->device), "cudaSetDevice");
    lbm_status st = smem_attr(m);
    if (st != LBM_OK) return st;
    // the training pass without the optimiser step: the accumulated full-batch
    // gradient is copied out and the accumulator cleared again
    MCUDA(m, cudaMemsetAsync(m->grad, 0, NPARAM * sizeof(float)), "memset");
    MCUDA(m, cudaMemsetAsync(m->loss, 0, sizeof(float)), "memset");
    mlp_train_kernel<<<(B + SAMPLES - 1) / SAMPLES, THREADS, sizeof(Smem)>>>(
        params_of(m), X, nin, T, nout, B, m->grad, m->loss);
    MCUDA(m, cudaGetLastError(), "mlp gradient launch");
    float loss = 0.f;
    MCUDA(m, cudaMemcpy(grad, m->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost),
          "gradient copy");
    MCUDA(m, cudaMemcpy(&loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost),
          "loss copy");
    MCUDA(m, cudaMemset(m->grad, 0, NPARAM * sizeof(float)), "memset");
    if (loss_out) *loss_out = loss / (float)(B * nout);
    return LBM_OK;
}

lbm_status lbm_mlp_predict(lbm_mlp *m, const float *X, int nin, float *Y,
                           int nout, int B)
{
    CPLBM_TRACE("lbm_mlp_predict");
    if (!m) return LBM_ERR_ARG;
    if (!X || !Y || B <= 0 || nin < 1 || nin > DIN || nout < 1 || nout > DOUT)
        return mfail(m, LBM_ERR_ARG, "bad prediction arguments", cudaSuccess);
    MCUDA(m, cudaSetDevice(m->device), "cudaSetDevice");
    lbm_status st = smem_attr(m);
    if (st != LBM_OK) return st;
    mlp_infer_kernel<<<(B + SAMPLES - 1) / SAMPLES, THREADS, sizeof(Smem)>>>(
        params_of(m), X, nin, Y, nout, B);
    MCUDA(m, cudaGetLastError(), "mlp infer launch");
    MCUDA(m, cudaDeviceSynchronize(), "mlp infer");
    return LBM_OK;
}

lbm_status lbm_mlp_get_params(lbm_mlp *m, float *out)
{
    if (!m || !out) return LBM_ERR_ARG;
    MCUDA(m, cudaMemcpy(out, m->p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost),
          "params copy");
    return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp *m)
{
    if (!m) return;
    dev_free(m->p);
    dev_free(m->grad);
    dev_free(m->m);
    dev_free(m->v);
    dev_free(m->loss);
    dev_free(m->wt);
    dev_free(m->w);
    delete m;
}

const char *lbm_mlp_last_error(const lbm_mlp *m)
{
    return m ? m->err.c_str() : g_mlp_err.c_str();
}

}  // extern "C"
