// a5-a8: tile x depth ordering and per-tile front-to-back compositing (Eq. 1-2)
// with its backward.
//
// Ordering is done depth-first: the selected Gaussians are stably sorted once
// by their float32 depth key (ties keep ascending selection order), the
// (tile, Gaussian) pairs are emitted in that order, and a stable radix sort on
// the tile id alone groups them by tile.  The result is the (tile, depth,
// index) order of a full-key sort at a fraction of its passes, because pairs
// outnumber Gaussians.
//
// Blending runs one 256-thread CTA per 16x16 tile; batches of the tile's
// Gaussians are staged in shared memory.  Eq. 1 is truncated once a pixel's
// transmittance falls below 1e-4 (the Gaussian that crosses the bound is still
// blended), so the neglected tail is at most 1e-4 of the colour.  The support test p >= -4.5 uses
// explicitly rounded float32 operations (it decides which pixels a Gaussian
// touches); the alpha, transmittance and colour arithmetic are ordinary fp32.
// The backward recomputes each pixel's final transmittance and last
// contributor from the sorted list (nothing per pixel is stored by the forward)
// and then walks the list back to front.
#include "lodgs_internal.cuh"

namespace lodgs {
namespace {

constexpr int RB = 256;
constexpr int RGRID = 148 * 8;

__global__ void k_gather_nt(const uint32_t *__restrict__ order, const uint32_t *__restrict__ ntiles,
                            const uint32_t *__restrict__ cnt, uint32_t *__restrict__ nt_sorted) {
    uint32_t n = cnt[C_NSEL_EFF];
    for (uint32_t r = blockIdx.x * RB + threadIdx.x; r < n; r += gridDim.x * RB) nt_sorted[r] = ntiles[order[r]];
}

__global__ void k_clamp_pairs(uint32_t *cnt, uint64_t cap_pairs) {
    uint32_t n = cnt[C_NPAIR];
    if (n > cap_pairs || (cnt[C_STATUS] & ST_CAPACITY)) { cnt[C_STATUS] |= ST_CAPACITY; n = 0; }
    cnt[C_NPAIR_EFF] = n;
}

__global__ void k_emit(const uint32_t *__restrict__ order, const uint32_t *__restrict__ ntiles,
                       const uint2 *__restrict__ rect, const uint32_t *__restrict__ pair_off,
                       const uint32_t *__restrict__ cnt, int TX, uint32_t *__restrict__ pkey,
                       uint32_t *__restrict__ pval) {
    if (cnt[C_NPAIR_EFF] == 0) return;
    uint32_t n = cnt[C_NSEL_EFF];
    for (uint32_t r = blockIdx.x * RB + threadIdx.x; r < n; r += gridDim.x * RB) {
        uint32_t g = order[r];
        if (ntiles[g] == 0) continue;
        uint2 rc = rect[g];
        uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu, y1 = rc.y >> 16;
        uint32_t o = pair_off[r];
        for (uint32_t ty = y0; ty < y1; ++ty)
            for (uint32_t tx = x0; tx < x1; ++tx) {
                pkey[o] = ty * (uint32_t)TX + tx;
                pval[o] = g;
                ++o;
            }
    }
}

__global__ void k_ranges(const uint32_t *__restrict__ pkey, const uint32_t *__restrict__ cnt, uint2 *__restrict__ ranges) {
    uint32_t n = cnt[C_NPAIR_EFF];
    for (uint32_t p = blockIdx.x * RB + threadIdx.x; p < n; p += gridDim.x * RB) {
        uint32_t t = pkey[p];
        if (p == 0 || pkey[p - 1] != t) ranges[t].x = p;
        if (p + 1 == n || pkey[p + 1] != t) ranges[t].y = p + 1;
    }
}

// support exponent p = -1/2 d^T Q d with d = mean - pixel centre; float32,
// explicitly rounded (no contraction beyond the written fmaf)
__device__ __forceinline__ float support_p(float4 a, float nhc, float xc, float yc, float &dx, float &dy) {
    dx = __fsub_rn(a.x, xc);
    dy = __fsub_rn(a.y, yc);
    return __fmaf_rn(__fmul_rn(a.w, dx), dy, __fmaf_rn(__fmul_rn(nhc, dy), dy, __fmul_rn(__fmul_rn(a.z, dx), dx)));
}

constexpr float SUPPORT_P = -4.5f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float T_MIN = 1e-4f;

__global__ void __launch_bounds__(RB) k_blend(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ pval,
                                              const float4 *__restrict__ sp_a, const float4 *__restrict__ sp_b,
                                              const float *__restrict__ sp_c, const uint32_t *__restrict__ cnt,
                                              int W, int H, int TX, float bg0, float bg1, float bg2,
                                              float *__restrict__ image) {
    __shared__ float4 s_a[RB], s_b[RB];
    __shared__ float s_c[RB];
    if (cnt[C_STATUS] & ST_CAPACITY) return;
    const int tile = blockIdx.x, tid = threadIdx.x;
    const int px = (tile % TX) * TILE + (tid & 15), py = (tile / TX) * TILE + (tid >> 4);
    const bool inside = px < W && py < H;
    const float xc = (float)px + 0.5f, yc = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    float T = 1.0f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    bool done = !inside;
    for (uint32_t base = rg.x; base < rg.y; base += RB) {
        if (__syncthreads_count(done) == RB) break;
        uint32_t idx = base + tid;
        if (idx < rg.y) {
            uint32_t g = pval[idx];
            s_a[tid] = sp_a[g];
            s_b[tid] = sp_b[g];
            s_c[tid] = sp_c[g];
        }
        __syncthreads();
        int n = min((uint32_t)RB, rg.y - base);
        if (!done) {
            for (int j = 0; j < n; ++j) {
                float4 a = s_a[j];
                float4 b = s_b[j];
                float dx, dy;
                float p = support_p(a, b.x, xc, yc, dx, dy);
                if (p < SUPPORT_P) continue;
                float alpha = fminf(ALPHA_MAX, b.y * __expf(p));
                float w = alpha * T;
                c0 += b.z * w; c1 += b.w * w; c2 += s_c[j] * w;
                T = T * (1.0f - alpha);
                if (T < T_MIN) { done = true; break; }
            }
        }
    }
    if (inside) {
        float *o = image + ((size_t)py * W + px) * 3;
        o[0] = c0 + T * bg0; o[1] = c1 + T * bg1; o[2] = c2 + T * bg2;
    }
}

__global__ void __launch_bounds__(RB) k_blend_bwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ pval,
                                                  const float4 *__restrict__ sp_a, const float4 *__restrict__ sp_b,
                                                  const float *__restrict__ sp_c, const uint32_t *__restrict__ cnt,
                                                  int W, int H, int TX, float bg0, float bg1, float bg2,
                                                  const float *__restrict__ dL_dimg, float *__restrict__ g2d) {
    __shared__ float4 s_a[RB], s_b[RB];
    __shared__ float s_c[RB];
    __shared__ uint32_t s_g[RB];
    __shared__ float s_grad[RB][9];
    __shared__ uint32_t s_maxlast;
    if (cnt[C_STATUS] & ST_CAPACITY) return;
    const int tile = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int px = (tile % TX) * TILE + (tid & 15), py = (tile / TX) * TILE + (tid >> 4);
    const bool inside = px < W && py < H;
    const float xc = (float)px + 0.5f, yc = (float)py + 0.5f;
    const uint2 rg = ranges[tile];
    if (tid == 0) s_maxlast = 0;
    // ---- pass 1: final transmittance and last contributor of each pixel ----
    float T = 1.0f;
    uint32_t last = 0;
    bool done = !inside;
    for (uint32_t base = rg.x; base < rg.y; base += RB) {
        if (__syncthreads_count(done) == RB) break;
        uint32_t idx = base + tid;
        if (idx < rg.y) {
            uint32_t g = pval[idx];
            s_a[tid] = sp_a[g];
            s_b[tid] = sp_b[g];
        }
        __syncthreads();
        int n = min((uint32_t)RB, rg.y - base);
        if (!done) {
            for (int j = 0; j < n; ++j) {
                float4 a = s_a[j];
                float4 b = s_b[j];
                float dx, dy;
                float p = support_p(a, b.x, xc, yc, dx, dy);
                if (p < SUPPORT_P) continue;
                float alpha = fminf(ALPHA_MAX, b.y * __expf(p));
                T = T * (1.0f - alpha);
                last = base - rg.x + j + 1;
                if (T < T_MIN) { done = true; break; }
            }
        }
    }
    __syncthreads();
    if (inside && last) atomicMax(&s_maxlast, last);
    __syncthreads();
    const uint32_t end = rg.x + s_maxlast;
    // ---- pass 2: back to front ----
    float G0 = 0.f, G1 = 0.f, G2 = 0.f;
    if (inside) {
        const float *gi = dL_dimg + ((size_t)py * W + px) * 3;
        G0 = gi[0]; G1 = gi[1]; G2 = gi[2];
    }
    float Q0 = bg0, Q1 = bg1, Q2 = bg2;   // colour behind, divided by the transmittance in front of it
    for (uint32_t bend = end; bend > rg.x;) {
        uint32_t bstart = bend - rg.x > (uint32_t)RB ? bend - RB : rg.x;
        int n = (int)(bend - bstart);
        __syncthreads();
        if (tid < n) {
            uint32_t g = pval[bstart + tid];
            s_g[tid] = g;
            s_a[tid] = sp_a[g];
            s_b[tid] = sp_b[g];
            s_c[tid] = sp_c[g];
        }
        for (int c = 0; c < 9; ++c) s_grad[tid][c] = 0.f;
        __syncthreads();
        for (int j = n - 1; j >= 0; --j) {
            uint32_t pos = bstart - rg.x + (uint32_t)j;
            float4 a = s_a[j];
            float4 b = s_b[j];
            float dx, dy;
            float p = support_p(a, b.x, xc, yc, dx, dy);
            bool contrib = inside && pos < last && p >= SUPPORT_P;
            float gv[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) gv[c] = 0.f;
            if (contrib) {
                float e = __expf(p);
                float raw = b.y * e;
                float alpha = fminf(ALPHA_MAX, raw);
                float Tb = T / (1.0f - alpha);
                float cb = s_c[j];
                float dA = G0 * (b.z - Q0) + G1 * (b.w - Q1) + G2 * (cb - Q2);
                dA *= Tb;
                float wgt = alpha * Tb;
                gv[6] = G0 * wgt; gv[7] = G1 * wgt; gv[8] = G2 * wgt;
                Q0 = alpha * b.z + (1.0f - alpha) * Q0;
                Q1 = alpha * b.w + (1.0f - alpha) * Q1;
                Q2 = alpha * cb + (1.0f - alpha) * Q2;
                T = Tb;
                if (raw <= ALPHA_MAX) {
                    float dp = dA * alpha;
                    gv[5] = dA * e;
                    gv[0] = dp * (2.0f * a.z * dx + a.w * dy);
                    gv[1] = dp * (2.0f * b.x * dy + a.w * dx);
                    gv[2] = -0.5f * dp * dx * dx;
                    gv[3] = -dp * dx * dy;
                    gv[4] = -0.5f * dp * dy * dy;
                }
            }
            if (__ballot_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int c = 0; c < 9; ++c) {
                    float v = gv[c];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    gv[c] = v;
                }
                if (lane == 0) {
#pragma unroll
                    for (int c = 0; c < 9; ++c) atomicAdd(&s_grad[j][c], gv[c]);
                }
            }
        }
        __syncthreads();
        if (tid < n) {
            float *o = g2d + (size_t)s_g[tid] * 9;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                float v = s_grad[tid][c];
                if (v != 0.f) atomicAdd(o + c, v);
            }
        }
        bend = bstart;
    }
}

int ceil_log2(uint64_t x) {
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

}  // namespace

int launch_raster(const CamK &k, FrameBufs &f, const float bg[3], float *image, cudaStream_t st,
                  const StageMarks &sm) {
    bool alt;
    sm.mark(LODGS_STAGE_DEPTH_SORT, 0, st);
    int rc = radix_sort_pairs(f.dkey, f.dval, f.dkey_alt, f.dval_alt, f.cnt + C_NSEL_EFF, (uint32_t)f.cap_sel, 0, 32,
                              f.sort_hist, st, &alt);
    if (rc) return rc;
    const uint32_t *order = alt ? f.dval_alt : f.dval;
    f.order = order;
    sm.mark(LODGS_STAGE_DEPTH_SORT, 1, st);
    sm.mark(LODGS_STAGE_EMIT, 0, st);
    k_gather_nt<<<RGRID, RB, 0, st>>>(order, f.ntiles, f.cnt, f.nt_sorted);
    count_launches(1);
    rc = scan_exclusive(f.nt_sorted, f.pair_off, f.cnt + C_NSEL_EFF, (uint32_t)f.cap_sel, f.scan_bsum,
                        f.cnt + C_NPAIR, st);
    if (rc) return rc;
    k_clamp_pairs<<<1, 1, 0, st>>>(f.cnt, f.cap_pairs);
    count_launches(1);
    k_emit<<<RGRID, RB, 0, st>>>(order, f.ntiles, f.rect, f.pair_off, f.cnt, k.TX, f.pkey, f.pval);
    count_launches(1);
    sm.mark(LODGS_STAGE_EMIT, 1, st);
    sm.mark(LODGS_STAGE_TILE_SORT, 0, st);
    const uint64_t n_tiles = (uint64_t)k.TX * k.TY;
    rc = radix_sort_pairs(f.pkey, f.pval, f.pkey_alt, f.pval_alt, f.cnt + C_NPAIR_EFF, (uint32_t)f.cap_pairs, 0,
                          ceil_log2(n_tiles), f.sort_hist, st, &alt);
    if (rc) return rc;
    const uint32_t *skey = alt ? f.pkey_alt : f.pkey;
    f.sorted_pval = alt ? f.pval_alt : f.pval;
    sm.mark(LODGS_STAGE_TILE_SORT, 1, st);
    sm.mark(LODGS_STAGE_BLEND, 0, st);
    LODGS_CUDA(cudaMemsetAsync(f.ranges, 0, n_tiles * sizeof(uint2), st));
    k_ranges<<<RGRID, RB, 0, st>>>(skey, f.cnt, f.ranges);
    count_launches(1);
    k_blend<<<(unsigned)n_tiles, RB, 0, st>>>(f.ranges, f.sorted_pval, f.sp_a, f.sp_b, f.sp_c, f.cnt, k.W, k.H, k.TX,
                                              bg[0], bg[1], bg[2], image);
    count_launches(1);
    sm.mark(LODGS_STAGE_BLEND, 1, st);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

int launch_raster_backward(const CamK &k, FrameBufs &f, const float bg[3], const float *dL_dimage, cudaStream_t st) {
    const uint64_t n_tiles = (uint64_t)k.TX * k.TY;
    LODGS_CUDA(cudaMemsetAsync(f.g2d, 0, f.cap_sel * 9 * sizeof(float), st));
    k_blend_bwd<<<(unsigned)n_tiles, RB, 0, st>>>(f.ranges, f.sorted_pval, f.sp_a, f.sp_b, f.sp_c, f.cnt, k.W, k.H,
                                                  k.TX, bg[0], bg[1], bg[2], dL_dimage, f.g2d);
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

}  // namespace lodgs
