// Fused L1 photometric loss of a rendered image against a target, with its
// gradient, for the training step: dL/dI = scale * sign(I - T) and the sum
// |I - T| (the caller scales it, e.g. by 1/n for the mean).  One pass, float4
// loads, block reduction and one atomic per block.
#include "lodgs_internal.cuh"

using namespace lodgs;

namespace {

constexpr int LB = 256;

__device__ __forceinline__ float sgn(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(LB) k_l1(const float *__restrict__ img, const float *__restrict__ tgt, int64_t n,
                                           float scale, float *__restrict__ dL, float *__restrict__ loss_sum) {
    __shared__ float s_w[LB / 32];
    float acc = 0.f;
    const int64_t n4 = n / 4;
    const float4 *i4 = reinterpret_cast<const float4 *>(img);
    const float4 *t4 = reinterpret_cast<const float4 *>(tgt);
    float4 *g4 = reinterpret_cast<float4 *>(dL);
    for (int64_t i = blockIdx.x * (int64_t)LB + threadIdx.x; i < n4; i += (int64_t)gridDim.x * LB) {
        const float4 a = i4[i], b = t4[i];
        const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
        acc += fabsf(d.x) + fabsf(d.y) + fabsf(d.z) + fabsf(d.w);
        g4[i] = make_float4(scale * sgn(d.x), scale * sgn(d.y), scale * sgn(d.z), scale * sgn(d.w));
    }
    for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)LB + threadIdx.x; i < n; i += (int64_t)gridDim.x * LB) {
        const float d = img[i] - tgt[i];
        acc += fabsf(d);
        dL[i] = scale * sgn(d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < LB / 32; ++w) s += s_w[w];
        atomicAdd(loss_sum, s);
    }
}

}  // namespace

extern "C" int lodgs_l1_loss_grad(const float *image, const float *target, int64_t n, float grad_scale, float *dL,
                                  float *loss_sum, void *stream) {
    if (!image || !target || !dL || !loss_sum || n < 0) { set_error("l1_loss_grad: NULL argument"); return LODGS_E_INVALID; }
    if (((uintptr_t)image | (uintptr_t)target | (uintptr_t)dL) & 15) {
        set_error("l1_loss_grad: buffers must be 16-byte aligned");
        return LODGS_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    LODGS_CUDA(cudaMemsetAsync(loss_sum, 0, sizeof(float), st));
    if (n == 0) return LODGS_OK;
    k_l1<<<148 * 8, LB, 0, st>>>(image, target, n, grad_scale, dL, loss_sum);
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}
