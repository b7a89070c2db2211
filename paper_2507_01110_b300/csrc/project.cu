// a4: gather + EWA projection + SH colour of the selected nodes (Sec. 3, Eq. 2;
//     covariance R S S^T R^T; view-dependent colour b + SH of degrees 1..D).
// a9: its backward, from the per-Gaussian 2D gradients of the blend to the
//     stored record values, written as sparse or dense gradient rows.
//
// Compiled with -fmad=false: visibility, the tile rectangle and the depth key
// are integer decisions taken from float32 values evaluated as written.
#include <math.h>

#include "lodgs_internal.cuh"

namespace lodgs {
namespace {

constexpr int PB = 128;
// Grids: the projection runs one wave of resident blocks (resident_grid).  A
// fixed 8 blocks per SM was 1.14 waves at its 7 resident blocks per SM (70
// registers), the last 148 blocks almost alone on their SMs.  The backward (4
// resident blocks per SM at 128 registers) keeps 8 per SM: two full waves.
constexpr int PROJ_BWD_GRID = 148 * 8;

// Real spherical harmonics of degrees 1..3 (orthonormal, no Condon-Shortley
// phase), as polynomials of the unit direction (x, y, z); index l^2-1+(m+l).
// Constants: sqrt(3/4pi); sqrt(15/pi)/2; sqrt(5/pi)/4; sqrt(15/pi)/4;
// sqrt(35/2pi)/4; sqrt(105/pi)/2; sqrt(21/2pi)/4; sqrt(7/pi)/4; sqrt(105/pi)/4.
#define SH_C1 0.48860251190291992f
#define SH_C2A 1.0925484305920792f
#define SH_C20 0.31539156525252005f
#define SH_C22 0.54627421529603959f
#define SH_C33 0.59004358992664352f
#define SH_C32 2.8906114426405538f
#define SH_C31 0.45704579946446572f
#define SH_C30 0.37317633259011540f
#define SH_C32B 1.4453057213202769f

__device__ __forceinline__ void sh_basis(int degree, float x, float y, float z, float *Y) {
    if (degree >= 1) { Y[0] = SH_C1 * y; Y[1] = SH_C1 * z; Y[2] = SH_C1 * x; }
    if (degree >= 2) {
        Y[3] = SH_C2A * x * y; Y[4] = SH_C2A * y * z; Y[5] = SH_C20 * (3.0f * z * z - 1.0f);
        Y[6] = SH_C2A * x * z; Y[7] = SH_C22 * (x * x - y * y);
    }
    if (degree >= 3) {
        float z2 = 5.0f * z * z - 1.0f;
        Y[8] = SH_C33 * y * (3.0f * x * x - y * y); Y[9] = SH_C32 * x * y * z; Y[10] = SH_C31 * y * z2;
        Y[11] = SH_C30 * z * (5.0f * z * z - 3.0f); Y[12] = SH_C31 * x * z2; Y[13] = SH_C32B * z * (x * x - y * y);
        Y[14] = SH_C33 * x * (x * x - 3.0f * y * y);
    }
}

// gradient of each basis polynomial w.r.t. (x, y, z)
__device__ __forceinline__ void sh_basis_grad(int degree, float x, float y, float z, float (*dY)[3]) {
    if (degree >= 1) {
        dY[0][0] = 0; dY[0][1] = SH_C1; dY[0][2] = 0;
        dY[1][0] = 0; dY[1][1] = 0; dY[1][2] = SH_C1;
        dY[2][0] = SH_C1; dY[2][1] = 0; dY[2][2] = 0;
    }
    if (degree >= 2) {
        dY[3][0] = SH_C2A * y; dY[3][1] = SH_C2A * x; dY[3][2] = 0;
        dY[4][0] = 0; dY[4][1] = SH_C2A * z; dY[4][2] = SH_C2A * y;
        dY[5][0] = 0; dY[5][1] = 0; dY[5][2] = 6.0f * SH_C20 * z;
        dY[6][0] = SH_C2A * z; dY[6][1] = 0; dY[6][2] = SH_C2A * x;
        dY[7][0] = 2.0f * SH_C22 * x; dY[7][1] = -2.0f * SH_C22 * y; dY[7][2] = 0;
    }
    if (degree >= 3) {
        dY[8][0] = 6.0f * SH_C33 * x * y; dY[8][1] = SH_C33 * (3.0f * x * x - 3.0f * y * y); dY[8][2] = 0;
        dY[9][0] = SH_C32 * y * z; dY[9][1] = SH_C32 * x * z; dY[9][2] = SH_C32 * x * y;
        dY[10][0] = 0; dY[10][1] = SH_C31 * (5.0f * z * z - 1.0f); dY[10][2] = 10.0f * SH_C31 * y * z;
        dY[11][0] = 0; dY[11][1] = 0; dY[11][2] = SH_C30 * (15.0f * z * z - 3.0f);
        dY[12][0] = SH_C31 * (5.0f * z * z - 1.0f); dY[12][1] = 0; dY[12][2] = 10.0f * SH_C31 * x * z;
        dY[13][0] = 2.0f * SH_C32B * x * z; dY[13][1] = -2.0f * SH_C32B * y * z; dY[13][2] = SH_C32B * (x * x - y * y);
        dY[14][0] = SH_C33 * (3.0f * x * x - 3.0f * y * y); dY[14][1] = -6.0f * SH_C33 * x * y; dY[14][2] = 0;
    }
}

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[3][3]) {
    R[0][0] = 1.0f - 2.0f * (y * y + z * z);
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = 1.0f - 2.0f * (x * x + z * z);
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = 1.0f - 2.0f * (x * x + y * y);
}

// Shared forward geometry: 3D covariance, clamped Jacobian, T = J W, 2D covariance.
struct Geo {
    float t[3], dist, d[3];
    float qh[4], qn, R[3][3], M[3][3], S[3][3];
    float txc, tyc, J00, J02, J11, J12, T[2][3];
    float a, b, c, det;
    bool clx, cly;
};

__device__ __forceinline__ void geometry(const CamK &k, const float *mu, const float *s, const float *q, Geo &g) {
    g.d[0] = mu[0] - k.pos[0]; g.d[1] = mu[1] - k.pos[1]; g.d[2] = mu[2] - k.pos[2];
    cam_view(k, mu[0], mu[1], mu[2], g.t, &g.dist);
    float w = q[0], x = q[1], y = q[2], z = q[3];
    g.qn = sqrtf(((w * w + x * x) + y * y) + z * z);
    g.qh[0] = w / g.qn; g.qh[1] = x / g.qn; g.qh[2] = y / g.qn; g.qh[3] = z / g.qn;
    quat_rot(g.qh[0], g.qh[1], g.qh[2], g.qh[3], g.R);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) g.M[i][j] = g.R[i][j] * s[j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            g.S[i][j] = (g.M[i][0] * g.M[j][0] + g.M[i][1] * g.M[j][1]) + g.M[i][2] * g.M[j][2];
    float tx = g.t[0], ty = g.t[1], tz = g.t[2];
    float txtz = tx / tz, tytz = ty / tz;
    g.clx = txtz < -k.limx || txtz > k.limx;
    g.cly = tytz < -k.limy || tytz > k.limy;
    g.txc = fminf(k.limx, fmaxf(-k.limx, txtz)) * tz;
    g.tyc = fminf(k.limy, fmaxf(-k.limy, tytz)) * tz;
    g.J00 = k.fx / tz; g.J02 = -(k.fx * g.txc) / (tz * tz);
    g.J11 = k.fy / tz; g.J12 = -(k.fy * g.tyc) / (tz * tz);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        g.T[0][b] = g.J00 * k.R[0 * 3 + b] + g.J02 * k.R[2 * 3 + b];
        g.T[1][b] = g.J11 * k.R[1 * 3 + b] + g.J12 * k.R[2 * 3 + b];
    }
    float U[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) U[a][b] = (g.T[a][0] * g.S[0][b] + g.T[a][1] * g.S[1][b]) + g.T[a][2] * g.S[2][b];
    float s00 = (U[0][0] * g.T[0][0] + U[0][1] * g.T[0][1]) + U[0][2] * g.T[0][2];
    float s01 = (U[0][0] * g.T[1][0] + U[0][1] * g.T[1][1]) + U[0][2] * g.T[1][2];
    float s11 = (U[1][0] * g.T[1][0] + U[1][1] * g.T[1][1]) + U[1][2] * g.T[1][2];
    g.a = s00 + 0.3f; g.b = s01; g.c = s11 + 0.3f;
    g.det = g.a * g.c - g.b * g.b;
}

// Support half extents for the 8x8-block test of the blend.  The ellipse
// d^T Sigma^-1 d <= 2L of the 2D covariance (a, b; b, c) spans |dx| <= sqrt(2L a),
// |dy| <= sqrt(2L c); the support test p >= -4.5 is L = 4.5, raised to 4.51 +
// 1e-5 kap, kap = (a + c)^2 / det >= the condition number, to cover the float32
// rounding of the conic and of p, which grows with the conditioning.  Beyond
// kap = 1e5 the extents are infinite (no block is ever skipped).
__device__ __forceinline__ void support_extents(float a, float c, float det, float &rx, float &ry) {
    const float tr = a + c;
    const float kap = (tr * tr) / det;
    rx = INFINITY;
    ry = INFINITY;
    if (kap <= 1e5f) {
        const float l2 = 9.02f + 2e-5f * kap;
        rx = sqrtf(l2 * a);
        ry = sqrtf(l2 * c);
    }
}

// Floats per record of SH degree DEG (14 base values + 3 per SH coefficient,
// padded to a multiple of 8).
__host__ __device__ constexpr int rec_stride(int deg) { return (14 + 3 * ((deg + 1) * (deg + 1) - 1) + 7) / 8 * 8; }

template <int DEG>
__global__ void __launch_bounds__(PB) k_project(const float *__restrict__ rows, int stride,
                                                 const uint32_t *__restrict__ sel_rows, const View *__restrict__ view,
                                                 uint32_t *__restrict__ cnt, uint64_t cap_sel, float4 *__restrict__ sp_a,
                                                 float4 *__restrict__ sp_b, float4 *__restrict__ sp_c,
                                                 uint32_t *__restrict__ dkey, uint32_t *__restrict__ dval,
                                                 uint2 *__restrict__ rect, uint32_t *__restrict__ ntiles,
                                                 float4 *__restrict__ g2d) {
    pdl_wait();
    const CamK &k = view->k;
    // selections beyond the workspace are not rendered: the frame reports a capacity error
    uint32_t n = cnt[C_NSEL];
    if (n > cap_sel) n = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cnt[C_NSEL_EFF] = n;
        if (cnt[C_NSEL] > cap_sel) atomicOr(&cnt[C_STATUS], ST_CAPACITY);
    }
    constexpr int degree = DEG;
    constexpr int K = (DEG + 1) * (DEG + 1) - 1;
    uint32_t nvis = 0;
    unsigned long long npairs = 0;
    for (uint32_t i = blockIdx.x * PB + threadIdx.x; i < n; i += gridDim.x * PB) {
        const float *r = rows + (size_t)sel_rows[i] * stride;
        float4 r0 = *reinterpret_cast<const float4 *>(r);        // mu, s0
        float4 r1 = *reinterpret_cast<const float4 *>(r + 4);    // s1, s2, qw, qx
        float4 r2 = *reinterpret_cast<const float4 *>(r + 8);    // qy, qz, op, b0
        float2 r3 = *reinterpret_cast<const float2 *>(r + 12);   // b1, b2
        float mu[3] = {r0.x, r0.y, r0.z}, s[3] = {r0.w, r1.x, r1.y}, q[4] = {r1.z, r1.w, r2.x, r2.y};
        float op = r2.z;
        bool vis = false;
        uint32_t key = 0xffffffffu, nt = 0;
        uint2 rc = make_uint2(0, 0);
        float4 a = make_float4(0, 0, 0, 0), b = make_float4(0, 0, 0, 0), c4 = make_float4(0, 0, 0, 0);
        float tz;
        {
            float t[3], dist;
            cam_view(k, mu[0], mu[1], mu[2], t, &dist);
            tz = t[2];
        }
        if (tz > k.znear) {
            Geo g;
            geometry(k, mu, s, q, g);
            if (g.det > 0.0f) {
                float A = g.c / g.det, B = -g.b / g.det, C = g.a / g.det;
                float mid = 0.5f * (g.a + g.c);
                float disc = sqrtf(fmaxf(0.1f, mid * mid - g.det));
                float lam = mid + disc;
                float rad = ceilf(3.0f * sqrtf(lam));
                float u = (k.fx * g.t[0]) / tz + k.cx;
                float v = (k.fy * g.t[1]) / tz + k.cy;
                if (isfinite(u) && isfinite(v) && isfinite(rad)) {
                    float fx0 = fminf(fmaxf(floorf((u - rad) * 0.0625f), 0.0f), (float)k.TX);
                    float fx1 = fminf(fmaxf(floorf((u + rad) * 0.0625f) + 1.0f, 0.0f), (float)k.TX);
                    float fy0 = fminf(fmaxf(floorf((v - rad) * 0.0625f), 0.0f), (float)k.TY);
                    float fy1 = fminf(fmaxf(floorf((v + rad) * 0.0625f) + 1.0f, 0.0f), (float)k.TY);
                    int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
                    int area = (x1 - x0) * (y1 - y0);
                    if (area > 0) {
                        vis = true;
                        nt = (uint32_t)area;
                        rc = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
                        key = __float_as_uint(tz);
                        // view-dependent colour (value, not a decision)
                        float inv = 1.0f / g.dist;
                        float dx = g.d[0] * inv, dy = g.d[1] * inv, dz = g.d[2] * inv;
                        float col[3] = {r2.w, r3.x, r3.y};
                        if (K > 0) {
                            float Y[15];
                            sh_basis(degree, dx, dy, dz, Y);
                            // the coefficients (row floats 14 .. 14 + 3K) as float4 loads from
                            // float 12: rows are 16-byte aligned and padded to 8 floats, so the
                            // last chunk ends inside the row
                            constexpr int NCH = (2 + 3 * K + 3) / 4;
                            static_assert(12 + 4 * NCH <= rec_stride(DEG), "chunks inside the row");
                            float fl[4 * NCH];
#pragma unroll
                            for (int m = 0; m < NCH; ++m) {
                                const float4 v = *reinterpret_cast<const float4 *>(r + 12 + 4 * m);
                                fl[4 * m] = v.x; fl[4 * m + 1] = v.y; fl[4 * m + 2] = v.z; fl[4 * m + 3] = v.w;
                            }
                            const float *f = fl + (REC_F - 12);
#pragma unroll
                            for (int kk = 0; kk < K; ++kk) {
                                col[0] += Y[kk] * f[3 * kk];
                                col[1] += Y[kk] * f[3 * kk + 1];
                                col[2] += Y[kk] * f[3 * kk + 2];
                            }
                        }
                        a = make_float4(u, v, -0.5f * A, -B);
                        b = make_float4(-0.5f * C, op, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f));
                        float rx, ry;
                        support_extents(g.a, g.c, g.det, rx, ry);
                        c4 = make_float4(fmaxf(col[2], 0.f), rx, ry, 0.f);
                    }
                }
            }
        }
        sp_a[i] = a; sp_b[i] = b; sp_c[i] = c4;
        static_assert(G2D_STRIDE == 12, "three float4 per row");
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);       // the blend backward accumulates here
        g2d[3 * (size_t)i] = z; g2d[3 * (size_t)i + 1] = z; g2d[3 * (size_t)i + 2] = z;
        dkey[i] = key; dval[i] = i;
        rect[i] = rc; ntiles[i] = nt;
        nvis += vis ? 1u : 0u;
        npairs += nt;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nvis += __shfl_xor_sync(0xffffffffu, nvis, o);
    if ((threadIdx.x & 31) == 0 && nvis) atomicAdd(&cnt[C_NVIS], nvis);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) npairs += __shfl_xor_sync(0xffffffffu, npairs, o);
    if ((threadIdx.x & 31) == 0 && npairs)     // rectangle pairs as a 64-bit sum (32-bit index guard)
        atomicAdd(reinterpret_cast<unsigned long long *>(cnt + C_NPAIR64), npairs);
}

__device__ __forceinline__ void cp_async4(float *dst_smem, const float *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}


// Each warp handles 32 selected Gaussians at a time: the records of the
// visible ones are staged in shared memory row by row (whole-warp, coalesced
// asynchronous copies), each lane computes the gradient of its own Gaussian in place of its
// record there, and the warp writes the 32 gradient rows back row by row.
// Rows are padded to RS + 1 floats so that lanes reading the same field of
// their own rows hit distinct banks.
template <int DEG>
__global__ void __launch_bounds__(PB) k_project_bwd(const float *__restrict__ rows, int stride,
                                                     const uint32_t *__restrict__ sel_src,
                                                     const uint32_t *__restrict__ sel_rows,
                                                     const View *__restrict__ view, uint32_t *__restrict__ cnt,
                                                     const uint32_t *__restrict__ ntiles,
                                                     const float *__restrict__ g2d, float *__restrict__ out,
                                                     int dense, uint32_t out_cap) {
    pdl_wait();
    constexpr int RS = rec_stride(DEG), SP = RS + 1;
    __shared__ float s_rows[PB / 32][32 * SP];
    const CamK &k = view->k;
    const uint32_t n = cnt[C_NSEL_EFF];
    if (!dense && n > out_cap) {
        // sparse rows do not fit the caller's buffer: record it, write nothing,
        // and leave no rows for the consumers of the count (Adam, batch sums)
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicOr(&cnt[C_STATUS], ST_GRAD_CAPACITY);
            cnt[C_NSEL_EFF] = 0u;
        }
        return;
    }
    constexpr int degree = DEG;
    constexpr int K = (DEG + 1) * (DEG + 1) - 1;
    (void)stride;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *sw = s_rows[wib];
    float *r = sw + lane * SP;              // this lane's record, then its gradient row
    for (uint32_t t0 = (blockIdx.x * (PB / 32) + wib) * 32u; t0 < n; t0 += gridDim.x * PB) {
        const int m = (int)min(32u, n - t0);
        const uint32_t i = t0 + lane;
        const bool mine = lane < m;
        const bool vis = mine && ntiles[i] != 0;
        const uint32_t src = vis ? sel_src[i] : 0u;
        const unsigned vmask = __ballot_sync(0xffffffffu, vis);
        // asynchronous 4-byte copies straight into the padded rows: all of the
        // warp's row reads are in flight at once, without registers
        for (int e = 0; e < m; ++e) {
            if (!(vmask >> e & 1u)) continue;
            const float *g = rows + (size_t)__shfl_sync(0xffffffffu, src, e) * RS;
#pragma unroll
            for (int c = lane; c < RS; c += 32) cp_async4(sw + e * SP + c, g + c);
        }
        asm volatile("cp.async.commit_group;\n" ::);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncwarp();
        if (mine && !vis) {
            for (int c = 0; c < RS; ++c) r[c] = 0.f;
        } else if (vis) {
        const float *gg = g2d + (size_t)i * G2D_STRIDE;
        float g[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) g[c] = gg[c];
        float mu[3] = {r[0], r[1], r[2]}, s[3] = {r[3], r[4], r[5]}, q[4] = {r[6], r[7], r[8], r[9]};
        Geo G;
        geometry(k, mu, s, q, G);
        const float tz = G.t[2], tx = G.t[0], ty = G.t[1];
        float Qm00 = G.c / G.det, Qm01 = -G.b / G.det, Qm11 = G.a / G.det;
        // ---- colour ----
        float inv = 1.0f / G.dist;
        float dir[3] = {G.d[0] * inv, G.d[1] * inv, G.d[2] * inv};
        float Y[15], dY[15][3];
        if (K > 0) { sh_basis(degree, dir[0], dir[1], dir[2], Y); sh_basis_grad(degree, dir[0], dir[1], dir[2], dY); }
        float gdir[3] = {0.f, 0.f, 0.f};
        float grow_b[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float raw = r[REC_B + ch];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) raw += Y[kk] * r[REC_F + 3 * kk + ch];
            float gc = raw < 0.0f ? 0.0f : g[6 + ch];
            grow_b[ch] = gc;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const float f = r[REC_F + 3 * kk + ch];      // read before the slot is overwritten
                gdir[0] += gc * f * dY[kk][0];
                gdir[1] += gc * f * dY[kk][1];
                gdir[2] += gc * f * dY[kk][2];
                r[REC_F + 3 * kk + ch] = gc * Y[kk];
            }
        }
        float dotv = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
        float gd[3];
        for (int a = 0; a < 3; ++a) gd[a] = (gdir[a] - dir[a] * dotv) * inv;
        // ---- conic -> 2D covariance ----
        float gQ00 = g[2], gQ01 = 0.5f * g[3], gQ11 = g[4];
        float t00 = Qm00 * gQ00 + Qm01 * gQ01, t01 = Qm00 * gQ01 + Qm01 * gQ11;
        float t10 = Qm01 * gQ00 + Qm11 * gQ01, t11 = Qm01 * gQ01 + Qm11 * gQ11;
        float gS2[2][2];
        gS2[0][0] = -(t00 * Qm00 + t01 * Qm01);
        gS2[0][1] = -(t00 * Qm01 + t01 * Qm11);
        gS2[1][0] = -(t10 * Qm00 + t11 * Qm01);
        gS2[1][1] = -(t10 * Qm01 + t11 * Qm11);
        float gS[3][3], gT[2][3];
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float acc = 0.f;
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int c = 0; c < 2; ++c) acc += G.T[a][i2] * gS2[a][c] * G.T[c][j];
                gS[i2][j] = acc;
            }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                float acc = 0.f;
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int m = 0; m < 3; ++m) acc += 2.0f * gS2[a][c] * G.T[c][m] * G.S[m][b];
                gT[a][b] = acc;
            }
        float gJ[2][3];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int m = 0; m < 3; ++m)
                gJ[a][m] = gT[a][0] * k.R[m * 3 + 0] + gT[a][1] * k.R[m * 3 + 1] + gT[a][2] * k.R[m * 3 + 2];
        float tz2 = tz * tz, tz3 = tz2 * tz;
        float gt[3] = {0.f, 0.f, 0.f};
        gt[2] += -k.fx / tz2 * gJ[0][0] - k.fy / tz2 * gJ[1][1];
        if (!G.clx) { gt[0] += -k.fx / tz2 * gJ[0][2]; gt[2] += 2.0f * k.fx * tx / tz3 * gJ[0][2]; }
        else gt[2] += k.fx * G.txc / tz3 * gJ[0][2];
        if (!G.cly) { gt[1] += -k.fy / tz2 * gJ[1][2]; gt[2] += 2.0f * k.fy * ty / tz3 * gJ[1][2]; }
        else gt[2] += k.fy * G.tyc / tz3 * gJ[1][2];
        gt[0] += k.fx / tz * g[0];
        gt[2] += -k.fx * tx / tz2 * g[0];
        gt[1] += k.fy / tz * g[1];
        gt[2] += -k.fy * ty / tz2 * g[1];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            r[REC_MU + a] = gd[a] + k.R[0 * 3 + a] * gt[0] + k.R[1 * 3 + a] * gt[1] + k.R[2 * 3 + a] * gt[2];
        // ---- Sigma = M M^T, M = R diag(s) ----
        float gR[3][3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int i2 = 0; i2 < 3; ++i2) {
                float gM = 2.0f * (gS[i2][0] * G.M[0][j] + gS[i2][1] * G.M[1][j] + gS[i2][2] * G.M[2][j]);
                acc += gM * G.R[i2][j];
                gR[i2][j] = gM * s[j];
            }
            r[REC_S + j] = acc;
        }
        float w = G.qh[0], x = G.qh[1], y = G.qh[2], z = G.qh[3];
        float gq[4];
        gq[0] = 2.0f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
        gq[1] = 2.0f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - w * gR[1][2] + z * gR[2][0] + w * gR[2][1])
              - 4.0f * x * (gR[1][1] + gR[2][2]);
        gq[2] = 2.0f * (x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] - w * gR[2][0] + z * gR[2][1])
              - 4.0f * y * (gR[0][0] + gR[2][2]);
        gq[3] = 2.0f * (-w * gR[0][1] + x * gR[0][2] + w * gR[1][0] + y * gR[1][2] + x * gR[2][0] + y * gR[2][1])
              - 4.0f * z * (gR[0][0] + gR[1][1]);
        float qd = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
#pragma unroll
        for (int a = 0; a < 4; ++a) r[REC_Q + a] = (gq[a] - G.qh[a] * qd) / G.qn;
        r[REC_OP] = g[5];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) r[REC_B + ch] = grow_b[ch];
        for (int c = 14 + 3 * K; c < RS; ++c) r[c] = 0.f;
        }
        __syncwarp();
        const uint32_t dst_row = mine ? (dense ? sel_rows[i] : i) : 0u;
#pragma unroll 4
        for (int e = 0; e < m; ++e) {
            float2 *d = reinterpret_cast<float2 *>(out + (size_t)__shfl_sync(0xffffffffu, dst_row, e) * RS);
            for (int c = lane; c < RS / 2; c += 32) d[c] = make_float2(sw[e * SP + 2 * c], sw[e * SP + 2 * c + 1]);
        }
        __syncwarp();
    }
}

}  // namespace

int launch_project(const lodgs_scene *sc, const float *rows, FrameBufs &f, cudaStream_t st) {
#define LAUNCH_PROJ(D)                                                                                     \
    LODGS_CUDA(pdl_launch(k_project<D>, resident_grid(k_project<D>, PB), PB, st, rows, sc->stride, f.use_src ? f.sel_src : f.sel_rows, f.d_view, f.cnt, f.cap_sel, f.sp_a, \
                                           f.sp_b, f.sp_c, f.dkey, f.dval, f.rect, f.ntiles, \
                                           reinterpret_cast<float4 *>(f.g2d)))
    switch (sc->sh_degree) {
        case 0: LAUNCH_PROJ(0); break;
        case 1: LAUNCH_PROJ(1); break;
        case 2: LAUNCH_PROJ(2); break;
        default: LAUNCH_PROJ(3); break;
    }
#undef LAUNCH_PROJ
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

int launch_project_backward(const lodgs_scene *sc, const float *rows, FrameBufs &f, float *grad_rows,
                            int64_t grad_capacity, int dense, cudaStream_t st) {
    if (sc->sh_degree < 0 || sc->sh_degree > 3 || sc->stride != rec_stride(sc->sh_degree)) {
        set_error("render_backward: record stride does not match the SH degree");
        return LODGS_E_INVALID;
    }
    if (dense && grad_capacity < sc->n_nodes) {
        set_error("render_backward: dense gradient rows need n_nodes rows");
        return LODGS_E_INVALID;
    }
    const uint32_t cap = (uint32_t)std::min<int64_t>(std::max<int64_t>(grad_capacity, 0), UINT32_MAX);
#define LAUNCH_PBWD(D)                                                                                     \
    LODGS_CUDA(pdl_launch(k_project_bwd<D>, PROJ_BWD_GRID, PB, st, rows, sc->stride, f.use_src ? f.sel_src : f.sel_rows, f.sel_rows, f.d_view, \
                                               f.cnt, f.ntiles, f.g2d, grad_rows, dense, cap))
    switch (sc->sh_degree) {
        case 0: LAUNCH_PBWD(0); break;
        case 1: LAUNCH_PBWD(1); break;
        case 2: LAUNCH_PBWD(2); break;
        default: LAUNCH_PBWD(3); break;
    }
#undef LAUNCH_PBWD
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

}  // namespace lodgs
