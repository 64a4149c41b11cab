// Learned cost model kernels: a 12 -> 64 -> 64 -> 1 ReLU MLP that predicts
// log2 of a loop's run time from its features.  Weights are used rounded to
// bfloat16 (round to nearest even) with FP32 accumulation; the FP32 master
// weights are what SGD updates.  Gradients are taken with respect to the
// rounded weights and summed over the batch in a fixed order (per-team
// partials, then a fixed fold), so training is bit-for-bit repeatable.
//
// Parameter block (FP32): W1[64][12], b1[64], W2[64][64], b2[64], W3[64], b3.
#include <cuda_bf16.h>

#include "device_common.cuh"
#include "runtime_internal.h"

namespace upir {

namespace {

constexpr int NI = UPIR_MLP_IN, NH = UPIR_MLP_HIDDEN, NP = UPIR_MLP_NPARAM;
constexpr int OFF_W1 = 0, OFF_B1 = NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH;
constexpr int kRowsPerTeam = 64;  // rows of the batch one backward team folds

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Weights in shared memory, rounded to bfloat16 (biases stay FP32).
struct SmemNet {
    float w1[NH * NI], b1[NH], w2[NH * NH], b2[NH], w3[NH], b3;
};

__device__ __forceinline__ void load_net(SmemNet& n, const float* __restrict__ p) {
    for (int i = threadIdx.x; i < NH * NI; i += blockDim.x) n.w1[i] = bf16r(p[OFF_W1 + i]);
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) n.w2[i] = bf16r(p[OFF_W2 + i]);
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        n.b1[i] = p[OFF_B1 + i];
        n.b2[i] = p[OFF_B2 + i];
        n.w3[i] = bf16r(p[OFF_W3 + i]);
    }
    if (threadIdx.x == 0) n.b3 = p[OFF_B3];
}

// One row through the network with 64 threads (thread j = hidden unit j).
// Leaves h1, h2 (and the pre-activations' signs) in shared memory; returns
// the prediction in every thread.
__device__ __forceinline__ float forward_row(const SmemNet& n, const float* __restrict__ x, float* h1,
                                             float* h2, float* red) {
    const int j = threadIdx.x;
    float z = n.b1[j];
#pragma unroll
    for (int i = 0; i < NI; ++i) z = __fmaf_rn(n.w1[j * NI + i], x[i], z);
    h1[j] = fmaxf(z, 0.0f);
    __syncthreads();
    float z2 = n.b2[j];
#pragma unroll 16
    for (int k = 0; k < NH; ++k) z2 = __fmaf_rn(n.w2[j * NH + k], h1[k], z2);
    h2[j] = fmaxf(z2, 0.0f);
    // y = b3 + sum_j w3_j h2_j: fixed butterfly over the two warps, then their sum
    float v = __fmul_rn(n.w3[j], h2[j]);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
    if ((j & 31) == 0) red[j >> 5] = v;
    __syncthreads();
    const float y = __fadd_rn(n.b3, __fadd_rn(red[0], red[1]));
    __syncthreads();  // red is reused
    return y;
}

__global__ void __launch_bounds__(NH) mlp_forward_kernel(const float* __restrict__ params,
                                                         const float* __restrict__ X, int batch,
                                                         float* __restrict__ pred) {
    __shared__ SmemNet net;
    __shared__ float xs[NI], h1[NH], h2[NH], red[2];
    load_net(net, params);
    __syncthreads();
    for (int r = blockIdx.x; r < batch; r += gridDim.x) {
        if (threadIdx.x < NI) xs[threadIdx.x] = X[(int64_t)r * NI + threadIdx.x];
        __syncthreads();
        const float y = forward_row(net, xs, h1, h2, red);
        if (threadIdx.x == 0) pred[r] = y;
    }
}

// Backward: team g folds rows [g * R, (g + 1) * R) in order into per-thread
// gradient accumulators (thread j owns row j of W1, W2 and b1, b2, W3[j]),
// then writes them to partial slot g.  Loss partial in the last entry.
__global__ void __launch_bounds__(NH) mlp_backward_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ X,
                                                          const float* __restrict__ T, int batch,
                                                          float* __restrict__ partials) {
    __shared__ SmemNet net;
    __shared__ float xs[NI], h1[NH], h2[NH], dz2s[NH], red[2];
    load_net(net, params);
    __syncthreads();
    const int j = threadIdx.x;
    float gw1[NI], gw2[NH], gb1 = 0.0f, gb2 = 0.0f, gw3 = 0.0f, gb3 = 0.0f, loss = 0.0f;
#pragma unroll
    for (int i = 0; i < NI; ++i) gw1[i] = 0.0f;
#pragma unroll
    for (int k = 0; k < NH; ++k) gw2[k] = 0.0f;
    const float inv_b = 1.0f / (float)batch;
    const int r0 = blockIdx.x * kRowsPerTeam, r1 = min(r0 + kRowsPerTeam, batch);
    for (int r = r0; r < r1; ++r) {
        if (j < NI) xs[j] = X[(int64_t)r * NI + j];
        __syncthreads();
        const float y = forward_row(net, xs, h1, h2, red);
        const float d = __fsub_rn(y, T[r]);
        const float dy = __fmul_rn(__fmul_rn(2.0f, d), inv_b);  // d loss / d y, loss = mean d^2
        loss = __fmaf_rn(d, d, loss);
        // layer 3
        gw3 = __fmaf_rn(dy, h2[j], gw3);
        gb3 = __fadd_rn(gb3, dy);
        const float dz2 = h2[j] > 0.0f ? __fmul_rn(dy, net.w3[j]) : 0.0f;
        dz2s[j] = dz2;
        gb2 = __fadd_rn(gb2, dz2);
#pragma unroll
        for (int k = 0; k < NH; ++k) gw2[k] = __fmaf_rn(dz2, h1[k], gw2[k]);
        __syncthreads();
        // layer 1: dh1_j = sum_k W2[k][j] dz2_k (thread j is now input unit j of layer 2)
        float dh1 = 0.0f;
#pragma unroll 16
        for (int k = 0; k < NH; ++k) dh1 = __fmaf_rn(net.w2[k * NH + j], dz2s[k], dh1);
        const float dz1 = h1[j] > 0.0f ? dh1 : 0.0f;
        gb1 = __fadd_rn(gb1, dz1);
#pragma unroll
        for (int i = 0; i < NI; ++i) gw1[i] = __fmaf_rn(dz1, xs[i], gw1[i]);
        __syncthreads();  // xs, h1, h2, dz2s are rewritten by the next row
    }
    float* out = partials + (int64_t)blockIdx.x * (NP + 1);
#pragma unroll
    for (int i = 0; i < NI; ++i) out[OFF_W1 + j * NI + i] = gw1[i];
#pragma unroll
    for (int k = 0; k < NH; ++k) out[OFF_W2 + j * NH + k] = gw2[k];
    out[OFF_B1 + j] = gb1;
    out[OFF_B2 + j] = gb2;
    out[OFF_W3 + j] = gw3;
    // the team's loss and db3 (identical in every thread) from thread 0
    if (j == 0) {
        out[OFF_B3] = gb3;
        out[NP] = loss;
    }
}

// Fold the team partials of each parameter in team order.
__global__ void mlp_fold_kernel(const float* __restrict__ partials, int teams, float* __restrict__ grad,
                                float* __restrict__ loss, int batch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > NP) return;
    float s = 0.0f;
    for (int g = 0; g < teams; ++g) s = __fadd_rn(s, partials[(int64_t)g * (NP + 1) + i]);
    if (i < NP) grad[i] = s;
    else if (loss) *loss = __fdiv_rn(s, (float)batch);
}

__global__ void mlp_sgd_kernel(float* __restrict__ params, const float* __restrict__ grad, float lr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NP) params[i] = __fsub_rn(params[i], __fmul_rn(lr, grad[i]));
}

}  // namespace

}  // namespace upir

using namespace upir;

extern "C" upir_status upir_mlp_forward(upir_ctx ctx, const float* params, const float* x, int32_t batch,
                                        float* pred) {
    if (!ctx) return UPIR_EINVAL;
    if (batch < 0 || (batch > 0 && (!params || !x || !pred)))
        return fail(ctx, UPIR_EINVAL, "upir_mlp_forward: bad arguments");
    if (batch == 0) return UPIR_OK;
    const int teams = std::min<int>(batch, kNumSMs * 16);
    mlp_forward_kernel<<<teams, UPIR_MLP_HIDDEN, 0, ctx->stream>>>(params, x, batch, pred);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? UPIR_OK : cuda_fail(ctx, e, "upir_mlp_forward");
}

extern "C" upir_status upir_mlp_backward(upir_ctx ctx, const float* params, const float* x,
                                         const float* target, int32_t batch, float* grad, float* loss) {
    if (!ctx) return UPIR_EINVAL;
    if (batch <= 0 || !params || !x || !target || !grad)
        return fail(ctx, UPIR_EINVAL, "upir_mlp_backward: bad arguments");
    const int teams = (batch + kRowsPerTeam - 1) / kRowsPerTeam;
    const size_t bytes = (size_t)teams * (NP + 1) * sizeof(float);
    if (bytes > ctx->mlp_scratch_bytes) {
        if (ctx->mlp_scratch) {
            cudaStreamSynchronize(ctx->stream);
            dev_free(ctx, ctx->mlp_scratch, ctx->mlp_scratch_bytes);
            ctx->mlp_scratch = nullptr;
            ctx->mlp_scratch_bytes = 0;
        }
        ctx->mlp_scratch = dev_alloc(ctx, bytes);
        if (!ctx->mlp_scratch) return fail(ctx, UPIR_ENOMEM, "upir_mlp_backward: scratch of %zu bytes", bytes);
        ctx->mlp_scratch_bytes = bytes;
    }
    float* partials = static_cast<float*>(ctx->mlp_scratch);
    mlp_backward_kernel<<<teams, UPIR_MLP_HIDDEN, 0, ctx->stream>>>(params, x, target, batch, partials);
    mlp_fold_kernel<<<(NP + 1 + 255) / 256, 256, 0, ctx->stream>>>(partials, teams, grad, loss, batch);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? UPIR_OK : cuda_fail(ctx, e, "upir_mlp_backward");
}

extern "C" upir_status upir_mlp_sgd(upir_ctx ctx, float* params, const float* grad, float lr) {
    if (!ctx) return UPIR_EINVAL;
    if (!params || !grad) return fail(ctx, UPIR_EINVAL, "upir_mlp_sgd: bad arguments");
    mlp_sgd_kernel<<<(NP + 255) / 256, 256, 0, ctx->stream>>>(params, grad, lr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? UPIR_OK : cuda_fail(ctx, e, "upir_mlp_sgd");
}
