// Sparse Adam over the cut set and the densification criterion.
//
// Training optimises only the nodes of the view's LoD cut (appendix
// "Implementation Details"): after the backward, each listed node row takes an
// Adam step (Kingma and Ba) with its own step count, so its bias correction
// covers the steps it took part in.  Sixteen-byte quarters of a row are spread
// over threads (coalesced).  The screen-space mean gradient dL/d(u, v) of
// every selected Gaussian is also reduced to a per-node maximum over views, the
// quantity densification ranks nodes by.  After a densification renumbers the
// rows, per-row state (parameters' moments, step counts, gradient statistics)
// follows its node through a row gather.
#include <algorithm>

#include "lodgs_internal.cuh"

using namespace lodgs;

namespace {

constexpr int AB = 256;
constexpr int MAX_STRIDE = 64;

struct ColumnRates {
    float lr[MAX_STRIDE];
};

// One thread per 16-byte quarter of a row: every access of a row (its step
// count, the gradient, m, v and the parameters) is issued at once, so a row
// costs one memory round trip.  Whole rows go to one warp (32 / quads rows per
// warp, the remaining lanes idle): the quarter holding column 0 writes the new
// step count only after every quarter of its row has read the old one, which
// a __syncwarp orders.  Columns at or past `used` keep their bits.
__global__ void __launch_bounds__(AB) k_adam(float4 *__restrict__ params, float4 *__restrict__ m,
                                             float4 *__restrict__ v, uint32_t *__restrict__ t,
                                             const uint32_t *__restrict__ rows, const float4 *__restrict__ grads,
                                             const uint32_t *__restrict__ d_n, uint32_t n_host, int quads, int used,
                                             ColumnRates rates, float b1, float b2, float eps,
                                             uint32_t *__restrict__ dirty) {
    const uint32_t n = d_n ? min(*d_n, n_host) : n_host;    // never past the caller's max_n rows
    const float omb1 = 1.0f - b1, omb2 = 1.0f - b2;
    const int lane = threadIdx.x & 31;
    const int rpw = 32 / quads;                              // rows per warp (quads <= 16)
    const int slot = lane / quads, q = lane % quads;
    const uint64_t n_warps = ((uint64_t)n + rpw - 1) / rpw;
    const uint64_t grid_warps = (uint64_t)gridDim.x * (AB / 32);
    for (uint64_t w = (uint64_t)blockIdx.x * (AB / 32) + (threadIdx.x >> 5); w < n_warps; w += grid_warps) {
        const uint64_t i = w * rpw + slot;
        const bool act = slot < rpw && i < n;
        uint32_t r = 0, step = 0;
        size_t at = 0;
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f), mm = g, vv = g, pp = g;
        if (act) {
            r = rows[i];
            at = (size_t)r * quads + q;
            step = t[r] + 1;
            g = grads[(size_t)i * quads + q];
            mm = m[at];
            vv = v[at];
            pp = params[at];
        }
        __syncwarp();                                        // every quarter has read t[r]
        if (!act) continue;
        if (q == 0) {
            t[r] = step;
            if (dirty) dirty[r] = 1u;                // trained since it was loaded (cache slabs)
        }
        // 1 - b^t as -expm1(t log1p(-(1 - b))): 1 - b is exact in float32 and nothing cancels
        const float bc1 = -expm1f((float)step * log1pf(-omb1)), bc2 = -expm1f((float)step * log1pf(-omb2));
        float *mp = &mm.x, *vp = &vv.x, *pq = &pp.x;
        const float *gp = &g.x;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int col = 4 * q + c;
            if (col < used) {
                mp[c] = b1 * mp[c] + omb1 * gp[c];
                vp[c] = b2 * vp[c] + omb2 * gp[c] * gp[c];
                pq[c] -= rates.lr[col] * (mp[c] / bc1) / (sqrtf(vp[c] / bc2) + eps);
            }
        }
        m[at] = mm;
        v[at] = vv;
        params[at] = pp;
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

// dst[r] = src[src_row[r]] (row_words 32-bit words), zeros where src_row[r] is
// -1 or not below n_src.  One thread per word: consecutive threads read
// consecutive words of a row.
__global__ void __launch_bounds__(AB) k_gather_rows(const uint32_t *__restrict__ src, int64_t n_src,
                                                    uint32_t *__restrict__ dst, const int32_t *__restrict__ src_row,
                                                    int64_t n_rows, int row_words) {
    const int64_t total = n_rows * row_words;
    for (int64_t e = (int64_t)blockIdx.x * AB + threadIdx.x; e < total; e += (int64_t)gridDim.x * AB) {
        const int64_t r = e / row_words;
        const int c = (int)(e % row_words);
        const int32_t s = src_row[r];
        dst[e] = (s >= 0 && s < n_src) ? src[(int64_t)s * row_words + c] : 0u;
    }
}

}  // namespace

extern "C" int lodgs_gather_rows(const void *src, int64_t n_src, void *dst, const int32_t *src_row, int64_t n_rows,
                                 int32_t row_words, void *stream) {
    if (n_rows < 0 || n_src < 0 || row_words <= 0 || (n_rows > 0 && (!src_row || !dst || (n_src > 0 && !src)))) {
        set_error("gather_rows: NULL argument or bad size");
        return LODGS_E_INVALID;
    }
    if (src && dst && src == dst) { set_error("gather_rows: src and dst must not alias"); return LODGS_E_INVALID; }
    if (n_rows == 0) return LODGS_OK;
    const int64_t blocks = std::min<int64_t>((n_rows * row_words + AB - 1) / AB, 148 * 32);
    k_gather_rows<<<(unsigned)blocks, AB, 0, (cudaStream_t)stream>>>(
        static_cast<const uint32_t *>(src), n_src, static_cast<uint32_t *>(dst), src_row, n_rows, row_words);
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

namespace lodgs {
int launch_adam(const lodgs_scene *sc, float *params, float *m, float *v, uint32_t *t, const uint32_t *rows,
                const float *grads, const uint32_t *d_n, int64_t max_n, const float *lr, float b1, float b2,
                float eps, cudaStream_t st, uint32_t *dirty) {
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
    if (sc->stride % 4 || (uintptr_t)params % 16 || (uintptr_t)m % 16 || (uintptr_t)v % 16 || (uintptr_t)grads % 16) {
        set_error("adam_step: params, m, v and grads must be 16-byte aligned");
        return LODGS_E_INVALID;
    }
    const int quads = sc->stride / 4;
    const int64_t rpw = 32 / quads, warps = (max_n + rpw - 1) / rpw;
    const int64_t blocks = std::min<int64_t>((warps + AB / 32 - 1) / (AB / 32), 148 * 64);
    k_adam<<<(unsigned)std::max<int64_t>(blocks, 1), AB, 0, st>>>(
        reinterpret_cast<float4 *>(params), reinterpret_cast<float4 *>(m), reinterpret_cast<float4 *>(v), t, rows,
        reinterpret_cast<const float4 *>(grads), d_n, (uint32_t)max_n, quads, used, rates, b1, b2, eps, dirty);
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}
}  // namespace lodgs

extern "C" int lodgs_adam_step(lodgs_scene *sc, float *params, float *m, float *v, uint32_t *t, const uint32_t *rows,
                               const float *grads, const uint32_t *d_n, int64_t max_n, const float *lr, float b1,
                               float b2, float eps, void *stream) {
    return launch_adam(sc, params, m, v, t, rows, grads, d_n, max_n, lr, b1, b2, eps, (cudaStream_t)stream);
}

extern "C" int lodgs_frame_screen_grad_max(lodgs_frame *fr, float *max_per_node, void *stream) {
    if (!fr || !max_per_node) { set_error("frame_screen_grad_max: NULL argument"); return LODGS_E_INVALID; }
    if (int rc = check_frame(fr->scene, fr, "frame_screen_grad_max")) return rc;
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
