// Sparse Adam over the cut set and the densification criterion.
//
// Training optimises only the nodes of the view's LoD cut (appendix
// "Implementation Details"): after the backward, each listed node row takes an
// Adam step (Kingma and Ba) with its own step count, so its bias correction
// covers the steps it took part in.  One warp per row, the row's columns spread
// over the lanes (coalesced).  The screen-space mean gradient dL/d(u, v) of
// every selected Gaussian is also reduced to a per-node maximum over views, the
// quantity densification ranks nodes by.
#include <algorithm>

#include "lodgs_internal.cuh"

using namespace lodgs;

namespace {

constexpr int AB = 256;
constexpr int MAX_STRIDE = 64;

struct ColumnRates {
    float lr[MAX_STRIDE];
};

__global__ void __launch_bounds__(AB) k_adam(float *__restrict__ params, float *__restrict__ m, float *__restrict__ v,
                                             uint32_t *__restrict__ t, const uint32_t *__restrict__ rows,
                                             const float *__restrict__ grads, const uint32_t *__restrict__ d_n,
                                             uint32_t n_host, int stride, int used, ColumnRates rates, float b1,
                                             float b2, float eps) {
    const uint32_t n = d_n ? *d_n : n_host;
    const int lane = threadIdx.x & 31;
    const float omb1 = 1.0f - b1, omb2 = 1.0f - b2;
    const uint32_t warps = gridDim.x * (AB / 32);
    for (uint32_t i = blockIdx.x * (AB / 32) + (threadIdx.x >> 5); i < n; i += warps) {
        const uint32_t r = rows[i];
        uint32_t step = 0;
        if (lane == 0) {
            step = t[r] + 1;
            t[r] = step;
        }
        step = __shfl_sync(0xffffffffu, step, 0);
        // 1 - b^t as -expm1(t log1p(-(1 - b))): 1 - b is exact in float32 and nothing cancels
        const float bc1 = -expm1f((float)step * log1pf(-omb1)), bc2 = -expm1f((float)step * log1pf(-omb2));
        const float *g = grads + (size_t)i * stride;
        const size_t base = (size_t)r * stride;
        for (int c = lane; c < used; c += 32) {
            const float gc = g[c];
            const float mm = b1 * m[base + c] + omb1 * gc;
            const float vv = b2 * v[base + c] + omb2 * gc * gc;
            m[base + c] = mm;
            v[base + c] = vv;
            params[base + c] -= rates.lr[c] * (mm / bc1) / (sqrtf(vv / bc2) + eps);
        }
    }
}

// max over views of |dL/d(u, v)| per node (non-negative floats order like their bits)
__global__ void __launch_bounds__(AB) k_screen_grad_max(const uint32_t *__restrict__ sel_rows,
                                                        const float *__restrict__ g2d,
                                                        const uint32_t *__restrict__ cnt,
                                                        unsigned int *__restrict__ max_bits) {
    const uint32_t n = cnt[C_NSEL_EFF];
    for (uint32_t i = blockIdx.x * AB + threadIdx.x; i < n; i += gridDim.x * AB) {
        const float gu = g2d[(size_t)i * G2D_STRIDE], gv = g2d[(size_t)i * G2D_STRIDE + 1];
        const float norm = sqrtf(gu * gu + gv * gv);
        if (norm > 0.f) atomicMax(&max_bits[sel_rows[i]], __float_as_uint(norm));
    }
}

}  // namespace

extern "C" int lodgs_adam_step(lodgs_scene *sc, float *params, float *m, float *v, uint32_t *t, const uint32_t *rows,
                               const float *grads, const uint32_t *d_n, int64_t max_n, const float *lr, float b1,
                               float b2, float eps, void *stream) {
    if (!sc || !params || !m || !v || !t || !rows || !grads || !lr || max_n < 0) {
        set_error("adam_step: NULL argument or negative count");
        return LODGS_E_INVALID;
    }
    if (sc->stride > MAX_STRIDE) { set_error("adam_step: record stride above 64"); return LODGS_E_INVALID; }
    if (!(b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps >= 0.f)) {
        set_error("adam_step: need 0 <= b1, b2 < 1 and eps >= 0");
        return LODGS_E_INVALID;
    }
    if (max_n == 0) return LODGS_OK;
    ColumnRates rates{};
    for (int c = 0; c < sc->stride; ++c) rates.lr[c] = lr[c];
    const int used = 14 + 3 * ((sc->sh_degree + 1) * (sc->sh_degree + 1) - 1);
    const int64_t blocks = std::min<int64_t>((max_n + AB / 32 - 1) / (AB / 32), 148 * 16);
    k_adam<<<(unsigned)std::max<int64_t>(blocks, 1), AB, 0, (cudaStream_t)stream>>>(
        params, m, v, t, rows, grads, d_n, (uint32_t)max_n, sc->stride, used, rates, b1, b2, eps);
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

extern "C" int lodgs_frame_screen_grad_max(lodgs_frame *fr, float *max_per_node, void *stream) {
    if (!fr || !max_per_node) { set_error("frame_screen_grad_max: NULL argument"); return LODGS_E_INVALID; }
    if (!fr->blend_bwd_done) { set_error("frame_screen_grad_max: no backward on this frame's last render"); return LODGS_E_STATE; }
    k_screen_grad_max<<<148 * 4, AB, 0, (cudaStream_t)stream>>>(fr->f.sel_rows, fr->f.g2d, fr->f.cnt,
                                                               reinterpret_cast<unsigned int *>(max_per_node));
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

extern "C" int lodgs_frame_device_count(lodgs_frame *fr, const uint32_t **d_n_selected) {
    if (!fr || !d_n_selected) { set_error("frame_device_count: NULL argument"); return LODGS_E_INVALID; }
    *d_n_selected = fr->f.cnt + C_NSEL_EFF;
    return LODGS_OK;
}
