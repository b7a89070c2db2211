// Scene construction on the device: Morton order of the leaves, level-wise
// pairwise merges into a binary hierarchy (Sec. 3 "Gaussian Hierarchies"), the
// HSPT split by a BFS on the volume test (Sec. 4.3), and the SPT layout with
// clamped intervals (Sec. 4.1, Eq. 4 and Eq. 6; appendix "Unreachable
// Gaussians").
//
// Compiled with -fmad=false: the float32 decisions (Morton quantisation, volume
// test, S and lo terms) and the float64 merge are evaluated exactly as written,
// operation by operation, so that they are reproducible on any IEEE machine.
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lodgs_internal.cuh"

namespace lodgs {
namespace {

constexpr int BT = 256;
inline int nblk(int64_t n, int t = BT) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// ---------------------------------------------------------------------------
// Morton codes
// ---------------------------------------------------------------------------
__global__ void k_aabb(const float *__restrict__ rec, int stride, int64_t n, float *__restrict__ out /*6*/) {
    __shared__ float s[6][BT];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x; i < n; i += (int64_t)gridDim.x * BT)
        for (int a = 0; a < 3; ++a) {
            float v = rec[i * stride + a];
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    for (int a = 0; a < 3; ++a) { s[a][threadIdx.x] = lo[a]; s[3 + a][threadIdx.x] = hi[a]; }
    __syncthreads();
    for (int o = BT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int a = 0; a < 3; ++a) {
                s[a][threadIdx.x] = fminf(s[a][threadIdx.x], s[a][threadIdx.x + o]);
                s[3 + a][threadIdx.x] = fmaxf(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            // combine blocks with compare-and-swap loops (min/max are exact,
            // so the result does not depend on the order of the blocks)
            float v = s[a][0];
            int *p = (int *)&out[a];
            int old = *p, assumed;
            do {
                assumed = old;
                if (__int_as_float(assumed) <= v) break;
                old = atomicCAS(p, assumed, __float_as_int(v));
            } while (old != assumed);
            v = s[3 + a][0];
            p = (int *)&out[3 + a];
            old = *p;
            do {
                assumed = old;
                if (__int_as_float(assumed) >= v) break;
                old = atomicCAS(p, assumed, __float_as_int(v));
            } while (old != assumed);
        }
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {    // 21 bits -> every third bit
    uint64_t x = v & 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__global__ void k_morton(const float *__restrict__ rec, int stride, int64_t n, const float *__restrict__ box,
                         uint32_t *__restrict__ code_lo, uint32_t *__restrict__ code_hi, uint32_t *__restrict__ idx) {
    int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i >= n) return;
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        float lo = box[a], ext = box[3 + a] - box[a];
        float u = ext > 0.0f ? (rec[i * stride + a] - lo) / ext : 0.0f;
        q[a] = (uint32_t)fminf(u * 2097152.0f, 2097151.0f);
    }
    uint64_t c = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    code_lo[i] = (uint32_t)c;
    code_hi[i] = (uint32_t)(c >> 32);
    idx[i] = (uint32_t)i;
}

__global__ void k_gather_u32(const uint32_t *__restrict__ src, const uint32_t *__restrict__ idx, int64_t n,
                             uint32_t *__restrict__ dst) {
    int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// ---------------------------------------------------------------------------
// Pairwise merge in float64 (moment matching; weights = opacity x surface term)
// ---------------------------------------------------------------------------
__device__ void quat_to_rot_d(const double q[4], double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

__device__ void cov_of_record(const float *rec, double C[3][3]) {
    double q[4];
    for (int k = 0; k < 4; ++k) q[k] = rec[REC_Q + k];
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) q[k] = q[k] / n;
    double R[3][3];
    quat_to_rot_d(q, R);
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = (double)rec[REC_S + k] * (double)rec[REC_S + k];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[i][j] = R[i][0] * v[0] * R[j][0] + R[i][1] * v[1] * R[j][1] + R[i][2] * v[2] * R[j][2];
}

// symmetric Schur rotations, cyclic order (0,1),(0,2),(1,2); stops when the
// off-diagonal mass vanishes relative to the diagonal
__device__ void jacobi3(double A[3][3], double V[3][3]) {
    const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 16; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0 || off <= 1e-34 * dia) break;
        for (int k = 0; k < 3; ++k) {
            int p = P[k], q = Q[k];
            double apq = A[p][q];
            if (apq == 0.0) continue;
            double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
            double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
            if (theta < 0.0) t = -t;
            double c = 1.0 / sqrt(t * t + 1.0);
            double s = t * c;
            A[p][p] = A[p][p] - t * apq;
            A[q][q] = A[q][q] + t * apq;
            A[p][q] = 0.0;
            A[q][p] = 0.0;
            int r = 3 - p - q;
            double arp = A[r][p], arq = A[r][q];
            A[r][p] = c * arp - s * arq;
            A[p][r] = A[r][p];
            A[r][q] = s * arp + c * arq;
            A[q][r] = A[r][q];
            for (int i = 0; i < 3; ++i) {
                double vip = V[i][p], viq = V[i][q];
                V[i][p] = c * vip - s * viq;
                V[i][q] = s * vip + c * viq;
            }
        }
    }
}

__device__ void cov_to_scale_rot(double A[3][3], double s[3], double qo[4]) {
    double V[3][3];
    jacobi3(A, V);
    double lam[3] = {A[0][0], A[1][1], A[2][2]};
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 2 - i; ++j)
            if (lam[ord[j]] < lam[ord[j + 1]]) { int t = ord[j]; ord[j] = ord[j + 1]; ord[j + 1] = t; }
    double R[3][3];
    for (int k = 0; k < 3; ++k) {
        s[k] = sqrt(lam[ord[k]] > 0.0 ? lam[ord[k]] : 0.0);
        for (int i = 0; i < 3; ++i) R[i][k] = V[i][ord[k]];
    }
    for (int k = 0; k < 3; ++k) {          // largest-magnitude component positive
        int m = 0;
        for (int i = 1; i < 3; ++i)
            if (fabs(R[i][k]) > fabs(R[m][k])) m = i;
        if (R[m][k] < 0.0)
            for (int i = 0; i < 3; ++i) R[i][k] = -R[i][k];
    }
    double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1])
               - R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0])
               + R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
    if (det < 0.0)
        for (int i = 0; i < 3; ++i) R[i][2] = -R[i][2];
    double tr = R[0][0] + R[1][1] + R[2][2], w, x, y, z;
    if (tr > 0.0) {
        double S = sqrt(tr + 1.0) * 2.0;
        w = 0.25 * S; x = (R[2][1] - R[1][2]) / S; y = (R[0][2] - R[2][0]) / S; z = (R[1][0] - R[0][1]) / S;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        double S = sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2.0;
        w = (R[2][1] - R[1][2]) / S; x = 0.25 * S; y = (R[0][1] + R[1][0]) / S; z = (R[0][2] + R[2][0]) / S;
    } else if (R[1][1] > R[2][2]) {
        double S = sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2.0;
        w = (R[0][2] - R[2][0]) / S; x = (R[0][1] + R[1][0]) / S; y = 0.25 * S; z = (R[1][2] + R[2][1]) / S;
    } else {
        double S = sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2.0;
        w = (R[1][0] - R[0][1]) / S; x = (R[0][2] + R[2][0]) / S; y = (R[1][2] + R[2][1]) / S; z = 0.25 * S;
    }
    if (w < 0.0) { w = -w; x = -x; y = -y; z = -z; }
    double n = sqrt(w * w + x * x + y * y + z * z);
    qo[0] = w / n; qo[1] = x / n; qo[2] = y / n; qo[3] = z / n;
}

__device__ void merge_pair(int stride, int ncol, const float *ra, const float *rb, float *out) {
    const float *rc[2] = {ra, rb};
    double A[2], w[2];
    for (int k = 0; k < 2; ++k) {
        double s0 = rc[k][REC_S], s1 = rc[k][REC_S + 1], s2 = rc[k][REC_S + 2];
        A[k] = s0 * s1 + s0 * s2 + s1 * s2;
        w[k] = (double)rc[k][REC_OP] * A[k];
    }
    if (w[0] + w[1] == 0.0) { w[0] = 0.5; w[1] = 0.5; }
    double W = w[0] + w[1];
    double mu[3];
    for (int a = 0; a < 3; ++a) mu[a] = (w[0] * rc[0][REC_MU + a] + w[1] * rc[1][REC_MU + a]) / W;
    double C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < 2; ++k) {
        double Ck[3][3], d[3];
        cov_of_record(rc[k], Ck);
        for (int a = 0; a < 3; ++a) d[a] = rc[k][REC_MU + a] - mu[a];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) C[i][j] += w[k] * (Ck[i][j] + d[i] * d[j]);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i][j] = C[i][j] / W;
    double s[3], q[4];
    cov_to_scale_rot(C, s, q);
    double Ap = s[0] * s[1] + s[0] * s[2] + s[1] * s[2];
    double num = (double)ra[REC_OP] * A[0] + (double)rb[REC_OP] * A[1];
    double op = Ap > 0.0 ? num / Ap : (double)ra[REC_OP] + (double)rb[REC_OP];
    if (op > 1.0) op = 1.0;
    for (int k = 0; k < stride; ++k) out[k] = 0.0f;
    for (int a = 0; a < 3; ++a) out[REC_MU + a] = (float)mu[a];
    for (int a = 0; a < 3; ++a) out[REC_S + a] = (float)s[a];
    for (int a = 0; a < 4; ++a) out[REC_Q + a] = (float)q[a];
    out[REC_OP] = (float)op;
    for (int k = 0; k < ncol; ++k)
        out[REC_B + k] = (float)((w[0] * rc[0][REC_B + k] + w[1] * rc[1][REC_B + k]) / W);
}

__global__ void k_merge_level(float *__restrict__ node_rec, int stride, int ncol, const uint32_t *__restrict__ cur,
                              int64_t len, int64_t next_id, uint32_t *__restrict__ nxt, int32_t *__restrict__ left,
                              int32_t *__restrict__ right, int32_t *__restrict__ parent) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t npair = len / 2;
    if (k < npair) {
        uint32_t a = cur[2 * k], b = cur[2 * k + 1];
        int64_t p = next_id + k;
        merge_pair(stride, ncol, node_rec + (int64_t)a * stride, node_rec + (int64_t)b * stride,
                   node_rec + p * stride);
        left[p] = (int32_t)a; right[p] = (int32_t)b;
        parent[a] = (int32_t)p; parent[b] = (int32_t)p;
        nxt[k] = (uint32_t)p;
    } else if (k == npair && (len & 1)) {
        nxt[k] = cur[len - 1];
    }
}

// ---------------------------------------------------------------------------
// HSPT: level-synchronous BFS on the volume test
// ---------------------------------------------------------------------------
__global__ void k_hspt_classify(const float *__restrict__ node_rec, int stride, const int32_t *__restrict__ left,
                                const int32_t *__restrict__ frontier, int64_t F, float spt_volume,
                                int32_t *__restrict__ kind_out, uint32_t *__restrict__ internal_flag) {
    int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i >= F) return;
    int32_t v = frontier[i];
    const float *r = node_rec + (int64_t)v * stride;
    float vol = (r[REC_S] * r[REC_S + 1]) * r[REC_S + 2];
    int kind = vol < spt_volume ? KIND_SPT : (left[v] < 0 ? KIND_LEAF : KIND_INTERNAL);
    kind_out[i] = kind;
    internal_flag[i] = kind == KIND_INTERNAL ? 1u : 0u;
}

__global__ void k_hspt_expand(const int32_t *__restrict__ frontier, int64_t F, int64_t u_base,
                              const int32_t *__restrict__ kind, const uint32_t *__restrict__ child_pos,
                              const int32_t *__restrict__ left, const int32_t *__restrict__ right,
                              int32_t *__restrict__ next, int32_t *__restrict__ next_parent) {
    int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i >= F || kind[i] != KIND_INTERNAL) return;
    int32_t v = frontier[i];
    uint32_t c = 2 * child_pos[i];
    next[c] = left[v]; next[c + 1] = right[v];
    next_parent[c] = (int32_t)(u_base + i); next_parent[c + 1] = (int32_t)(u_base + i);
}

// per node: upper index or -1; SPT index for SPT roots
__global__ void k_mark_upper(const int32_t *__restrict__ up_node, const int32_t *__restrict__ up_kind, int64_t U,
                             const uint32_t *__restrict__ spt_idx, const uint32_t *__restrict__ row_idx,
                             int32_t *__restrict__ node_spt_root, int32_t *__restrict__ node_upper_row,
                             int32_t *__restrict__ spt_root, int32_t *__restrict__ up_ref) {
    int64_t u = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (u >= U) return;
    int32_t v = up_node[u];
    if (up_kind[u] == KIND_SPT) {
        node_spt_root[v] = (int32_t)spt_idx[u];
        spt_root[spt_idx[u]] = v;
        up_ref[u] = (int32_t)spt_idx[u];
    } else {
        node_upper_row[v] = (int32_t)row_idx[u];
        up_ref[u] = (int32_t)row_idx[u];
    }
}

__device__ __forceinline__ float size_S(const float *r) {
    float s0 = r[REC_S], s1 = r[REC_S + 1], s2 = r[REC_S + 2];
    return sqrtf(((s0 * s1 + s0 * s2) + s1 * s2) / 3.0f);
}

__device__ __forceinline__ float lo_raw(const float *r, const float *rr, float kappa) {
    float dx = r[REC_MU] - rr[REC_MU], dy = r[REC_MU + 1] - rr[REC_MU + 1], dz = r[REC_MU + 2] - rr[REC_MU + 2];
    float e = sqrtf((dx * dx + dy * dy) + dz * dz);
    return size_S(r) + e / kappa;
}

// SPT membership and clamped interval of every node below the HSPT cut.
// key_hi = ~bits(hi) (hi descending), key_j = SPT index (n_spt for upper nodes).
__global__ void k_spt_intervals(const float *__restrict__ node_rec, int stride, int64_t M,
                                const int32_t *__restrict__ parent, const int32_t *__restrict__ left,
                                const int32_t *__restrict__ node_spt_root, const int32_t *__restrict__ node_upper_row,
                                uint32_t n_spt, float kappa, float *__restrict__ lo_node, float *__restrict__ hi_node,
                                uint32_t *__restrict__ key_hi, uint32_t *__restrict__ key_j,
                                uint32_t *__restrict__ ids) {
    int64_t v = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (v >= M) return;
    ids[v] = (uint32_t)v;
    if (node_upper_row[v] >= 0) {
        key_j[v] = n_spt; key_hi[v] = 0u;
        lo_node[v] = NAN; hi_node[v] = NAN;
        return;
    }
    int32_t r = (int32_t)v;                        // walk up to the SPT root
    while (r >= 0 && node_spt_root[r] < 0) r = parent[r];
    if (r < 0) {                                   // not below any SPT root: structure error
        key_j[v] = n_spt; key_hi[v] = 0u;
        lo_node[v] = NAN; hi_node[v] = NAN;
        return;
    }
    const float *rr = node_rec + (int64_t)r * stride;
    float hi = INFINITY;                           // min of lo_raw over strict ancestors within the SPT
    for (int32_t a = (int32_t)v; a != r;) {
        a = parent[a];
        hi = fminf(hi, lo_raw(node_rec + (int64_t)a * stride, rr, kappa));
    }
    float lo;
    if (left[v] < 0) lo = 0.0f;
    else lo = fminf(lo_raw(node_rec + v * stride, rr, kappa), hi);
    lo_node[v] = lo; hi_node[v] = hi;
    key_hi[v] = ~__float_as_uint(hi);
    key_j[v] = (uint32_t)node_spt_root[r];
}

__global__ void k_spt_rows(const uint32_t *__restrict__ sorted_node, const uint32_t *__restrict__ sorted_j, int64_t M,
                           uint32_t n_spt, int64_t row0, int32_t *__restrict__ node_of_row,
                           uint32_t *__restrict__ spt_base, const float *__restrict__ lo_node,
                           const float *__restrict__ hi_node, float *__restrict__ lo_row, float *__restrict__ hi_row) {
    int64_t p = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (p >= M) return;
    uint32_t j = sorted_j[p];
    if (j >= n_spt) return;
    int64_t row = row0 + p;
    uint32_t v = sorted_node[p];
    node_of_row[row] = (int32_t)v;
    lo_row[row] = lo_node[v];
    hi_row[row] = hi_node[v];
    if (p == 0 || sorted_j[p - 1] != j) spt_base[j] = (uint32_t)row;
}

__global__ void k_upper_rows(const int32_t *__restrict__ up_node, const int32_t *__restrict__ up_kind,
                             const int32_t *__restrict__ up_ref, int64_t U, int32_t *__restrict__ node_of_row,
                             float *__restrict__ lo_row, float *__restrict__ hi_row) {
    int64_t u = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (u >= U || up_kind[u] == KIND_SPT) return;
    node_of_row[up_ref[u]] = up_node[u];
    lo_row[up_ref[u]] = NAN;
    hi_row[up_ref[u]] = NAN;
}

// ---- densification helpers ---------------------------------------------
__global__ void k_gather_i32(const int32_t *__restrict__ src, const int32_t *__restrict__ idx, int64_t n,
                             int32_t *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i < n) out[i] = idx[i] >= 0 ? src[idx[i]] : -1;
}

__global__ void k_scatter_i32(int32_t *__restrict__ dst, const int32_t *__restrict__ idx_val, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i < n) dst[idx_val[2 * i]] = idx_val[2 * i + 1];
}

__global__ void k_parent_of(const int32_t *__restrict__ left, const int32_t *__restrict__ right, int64_t M,
                            int32_t *__restrict__ parent) {
    const int64_t u = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (u >= M || left[u] < 0) return;
    parent[left[u]] = (int32_t)u;
    parent[right[u]] = (int32_t)u;
}

__global__ void k_row_of_node(const int32_t *__restrict__ node_of_row, int64_t M, int32_t *__restrict__ row_of) {
    const int64_t r = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (r < M) row_of[node_of_row[r]] = (int32_t)r;
}

__global__ void k_mark(uint8_t *__restrict__ flag, const int32_t *__restrict__ ids, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (i < n) flag[ids[i]] = 1;
}

// old render row of each new render row, -1 for a node whose record is new
__global__ void k_row_map(const int32_t *__restrict__ node_of_row, int64_t M, int64_t M0,
                          const int32_t *__restrict__ old_row_of, const uint8_t *__restrict__ fresh,
                          int32_t *__restrict__ out) {
    const int64_t r = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (r >= M) return;
    const int32_t u = node_of_row[r];
    out[r] = (u < M0 && !fresh[u]) ? old_row_of[u] : -1;
}

// The two children of a densified leaf (Sec. 3 "Densification": the split of
// 3DGS-MCMC, whose implementation the paper reuses, with N = 2): both keep the
// target's mean, rotation and colour.  Their opacity o' = 1 - sqrt(1 - o)
// keeps the composited opacity at the centre, 1 - (1 - o')^2 = o; their scales
// are the target's times f = o / (2 o' - o'^2 / sqrt 2), the factor with which
// the pair, composited front to back, integrates along any line through the
// centre to the target's o * integral(g) (the second child adds
// o' g (1 - o' g), and the square of a unit-peak Gaussian integrates in one
// dimension to 1/sqrt 2 of the Gaussian).  float32 with IEEE sqrt and
// division, evaluated as written.  trip[3i..3i+2] = (target, child a, child b),
// canonical ids.
constexpr float SQRT2_F = 1.41421356f;   // sqrt(2) rounded to float32

__global__ void k_split_children(float *__restrict__ node_rec, int stride, const int32_t *__restrict__ trip,
                                 int64_t n_ops) {
    int64_t t = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (t >= n_ops * stride) return;
    const int64_t i = t / stride;
    const int c = (int)(t % stride);
    const int32_t T = trip[3 * i], a = trip[3 * i + 1], b = trip[3 * i + 2];
    const float *rec = node_rec + (int64_t)T * stride;
    float v = rec[c];
    const float sg = rec[REC_OP];
    if (sg > 0.0f && (c == REC_OP || (c >= REC_S && c < REC_S + 3))) {
        const float sp = 1.0f - sqrtf(1.0f - sg);
        if (c == REC_OP) {
            v = sp;
        } else {
            const float f = sg / (2.0f * sp - (sp * sp) / SQRT2_F);
            v = v * f;
        }
    }
    node_rec[(int64_t)a * stride + c] = v;
    node_rec[(int64_t)b * stride + c] = v;
}

// canonical records from render rows: node_rec[node_of_row[r]] = rows[r]
__global__ void k_unpermute_rows(const float *__restrict__ rows, const int32_t *__restrict__ node_of_row, int64_t M,
                                 int stride, float *__restrict__ node_rec) {
    int64_t t = blockIdx.x * (int64_t)BT + threadIdx.x;
    int q = stride / 4;
    if (t >= M * q) return;
    int64_t row = t / q;
    int c = (int)(t % q);
    reinterpret_cast<float4 *>(node_rec)[(int64_t)node_of_row[row] * q + c] =
        reinterpret_cast<const float4 *>(rows)[row * q + c];
}

__global__ void k_permute_rows(const float *__restrict__ node_rec, const int32_t *__restrict__ node_of_row,
                               int64_t M, int stride, float *__restrict__ rows) {
    int64_t t = blockIdx.x * (int64_t)BT + threadIdx.x;
    int q = stride / 4;
    if (t >= M * q) return;
    int64_t row = t / q;
    int c = (int)(t % q);
    reinterpret_cast<float4 *>(rows)[row * q + c] =
        reinterpret_cast<const float4 *>(node_rec)[(int64_t)node_of_row[row] * q + c];
}

__global__ void k_upper_entries(const float *__restrict__ node_rec, int stride, const int32_t *__restrict__ up_node,
                                const int32_t *__restrict__ up_kind, const int32_t *__restrict__ up_parent,
                                const int32_t *__restrict__ up_ref, int64_t U, UpperEntry *__restrict__ out) {
    int64_t u = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (u >= U) return;
    const float *r = node_rec + (int64_t)up_node[u] * stride;
    UpperEntry e;
    e.mu[0] = r[REC_MU]; e.mu[1] = r[REC_MU + 1]; e.mu[2] = r[REC_MU + 2];
    e.S = size_S(r);
    e.maxs = fmaxf(fmaxf(r[REC_S], r[REC_S + 1]), r[REC_S + 2]);
    e.parent = up_parent[u];
    e.kind = up_kind[u];
    e.ref = up_ref[u];
    out[u] = e;
}

__global__ void k_flag_eq(const int32_t *__restrict__ kind, int64_t U, int32_t want, int invert,
                          uint32_t *__restrict__ flag) {
    int64_t u = blockIdx.x * (int64_t)BT + threadIdx.x;
    if (u >= U) return;
    bool e = kind[u] == want;
    flag[u] = (invert ? !e : e) ? 1u : 0u;
}

template <typename T>
struct DevBuf {
    T *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t n) { return cudaMalloc((void **)&p, std::max<size_t>(1, n) * sizeof(T)); }
    T *release() { T *q = p; p = nullptr; return q; }
};

}  // namespace

void free_scene(lodgs_scene *sc) {
    if (!sc) return;
    cudaFree(sc->d_rows); cudaFree(sc->d_upper); cudaFree(sc->d_spt_base); cudaFree(sc->d_lo); cudaFree(sc->d_hi);
    cudaFree(sc->d_node_rec); cudaFree(sc->d_left); cudaFree(sc->d_right); cudaFree(sc->d_node_of_row);
    cudaFree(sc->d_up_node); cudaFree(sc->d_spt_root);
}

#define CK(x) LODGS_CUDA(x)

// HSPT and SPT layout of a hierarchy (canonical records node_rec, children
// left/right, parent, root): the level-synchronous BFS of Algorithm 1 (SPT roots
// where the volume drops below spt_volume), the clamped SPT intervals, the SPT
// row layout (per SPT by descending hi) and the render-row records.  Used by the
// build and by the rebuild after densification; the scene's previous layout is
// replaced only once the new one is complete.
int build_layout(lodgs_scene *sc, const float *node_rec_p, const int32_t *left_p, const int32_t *right_p,
                 const int32_t *parent_p, int64_t M, int32_t root, const lodgs_build_params &p, cudaStream_t st) {
    const int stride = sc->stride;
    struct { const float *p; } node_rec{node_rec_p};
    struct { const int32_t *p; } left{left_p}, right{right_p}, parent{parent_p};
    DevBuf<float> lo_node, hi_node, lo_row, hi_row, rows;
    DevBuf<int32_t> node_spt_root, node_upper_row, node_of_row;
    DevBuf<uint32_t> k0, k1, v0, v1, hist, dn, hi_g;
    CK(k0.alloc(M)); CK(k1.alloc(M)); CK(v0.alloc(M)); CK(v1.alloc(M)); CK(hi_g.alloc(M));
    CK(hist.alloc(SORT_HIST)); CK(dn.alloc(1));
    bool alt;
    int rc;
    uint32_t *ord, *kk, *kalt, *valt;
    // ---- HSPT BFS (level synchronous) ----
    DevBuf<int32_t> up_node, up_kind, up_parent, up_ref, fr_a, fr_b, frp_a, frp_b;
    DevBuf<uint32_t> flag, pos, bsum, total;
    CK(up_node.alloc(M)); CK(up_kind.alloc(M)); CK(up_parent.alloc(M)); CK(up_ref.alloc(M));
    CK(fr_a.alloc(M)); CK(fr_b.alloc(M)); CK(frp_a.alloc(M)); CK(frp_b.alloc(M));
    CK(flag.alloc(M)); CK(pos.alloc(M)); CK(bsum.alloc(SCAN_GRID_MAX)); CK(total.alloc(1));
    int32_t minus1 = -1;
    CK(cudaMemcpy(fr_a.p, &root, 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(frp_a.p, &minus1, 4, cudaMemcpyHostToDevice));
    int64_t F = 1, U = 0;
    int depth = 0;
    while (F > 0) {
        CK(cudaMemcpyAsync(up_node.p + U, fr_a.p, F * 4, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(up_parent.p + U, frp_a.p, F * 4, cudaMemcpyDeviceToDevice, st));
        k_hspt_classify<<<nblk(F), BT, 0, st>>>(node_rec.p, stride, left.p, fr_a.p, F, p.spt_volume,
                                                up_kind.p + U, flag.p);
        count_launches(1);
        uint32_t F32 = (uint32_t)F;
        CK(cudaMemcpyAsync(dn.p, &F32, 4, cudaMemcpyHostToDevice, st));
        rc = scan_exclusive(flag.p, pos.p, dn.p, F32, bsum.p, total.p, st);
        if (rc) return rc;
        uint32_t n_int = 0;
        CK(cudaMemcpyAsync(&n_int, total.p, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        k_hspt_expand<<<nblk(F), BT, 0, st>>>(fr_a.p, F, U, up_kind.p + U, pos.p, left.p, right.p, fr_b.p, frp_b.p);
        count_launches(1);
        U += F;
        F = 2 * (int64_t)n_int;
        std::swap(fr_a.p, fr_b.p);
        std::swap(frp_a.p, frp_b.p);
        ++depth;
    }
    CK(cudaGetLastError());
    // SPT indices and upper rows in BFS order
    DevBuf<uint32_t> spt_idx, row_idx;
    CK(spt_idx.alloc(U)); CK(row_idx.alloc(U));
    uint32_t U32 = (uint32_t)U, n_spt = 0, n_rows_up = 0;
    CK(cudaMemcpy(dn.p, &U32, 4, cudaMemcpyHostToDevice));
    k_flag_eq<<<nblk(U), BT, 0, st>>>(up_kind.p, U, KIND_SPT, 0, flag.p);
    count_launches(1);
    rc = scan_exclusive(flag.p, spt_idx.p, dn.p, U32, bsum.p, total.p, st);
    if (rc) return rc;
    CK(cudaMemcpy(&n_spt, total.p, 4, cudaMemcpyDeviceToHost));
    k_flag_eq<<<nblk(U), BT, 0, st>>>(up_kind.p, U, KIND_SPT, 1, flag.p);
    count_launches(1);
    rc = scan_exclusive(flag.p, row_idx.p, dn.p, U32, bsum.p, total.p, st);
    if (rc) return rc;
    CK(cudaMemcpy(&n_rows_up, total.p, 4, cudaMemcpyDeviceToHost));
    DevBuf<int32_t> spt_root;
    CK(spt_root.alloc(n_spt));
    CK(node_spt_root.alloc(M)); CK(node_upper_row.alloc(M));
    CK(cudaMemset(node_spt_root.p, 0xff, M * 4)); CK(cudaMemset(node_upper_row.p, 0xff, M * 4));
    k_mark_upper<<<nblk(U), BT, 0, st>>>(up_node.p, up_kind.p, U, spt_idx.p, row_idx.p, node_spt_root.p,
                                         node_upper_row.p, spt_root.p, up_ref.p);
    count_launches(1);

    // ---- SPT intervals and layout ----
    CK(lo_node.alloc(M)); CK(hi_node.alloc(M));
    k_spt_intervals<<<nblk(M), BT, 0, st>>>(node_rec.p, stride, M, parent.p, left.p, node_spt_root.p,
                                            node_upper_row.p, n_spt, p.kappa, lo_node.p, hi_node.p, k0.p, hi_g.p, v0.p);
    count_launches(1);
    uint32_t M32 = (uint32_t)M;
    CK(cudaMemcpy(dn.p, &M32, 4, cudaMemcpyHostToDevice));
    rc = radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, dn.p, M32, 0, 32, hist.p, st, &alt);     // hi descending
    if (rc) return rc;
    ord = alt ? v1.p : v0.p;
    kk = alt ? k0.p : k1.p; kalt = alt ? k1.p : k0.p; valt = alt ? v0.p : v1.p;
    k_gather_u32<<<nblk(M), BT, 0, st>>>(hi_g.p, ord, M, kk);
    count_launches(1);
    int jbits = 1;
    while ((1ull << jbits) <= (uint64_t)n_spt) ++jbits;
    rc = radix_sort_pairs(kk, ord, kalt, valt, dn.p, M32, 0, jbits, hist.p, st, &alt);      // SPT index
    if (rc) return rc;
    uint32_t *sorted_node = alt ? valt : ord, *sorted_j = alt ? kalt : kk;
    CK(node_of_row.alloc(M)); CK(lo_row.alloc(M)); CK(hi_row.alloc(M));
    DevBuf<uint32_t> spt_base;
    CK(spt_base.alloc(n_spt + 1));
    {
        uint32_t M32b = (uint32_t)M;
        CK(cudaMemcpy(spt_base.p + n_spt, &M32b, 4, cudaMemcpyHostToDevice));
    }
    k_spt_rows<<<nblk(M), BT, 0, st>>>(sorted_node, sorted_j, M, n_spt, n_rows_up, node_of_row.p, spt_base.p,
                                       lo_node.p, hi_node.p, lo_row.p, hi_row.p);
    count_launches(1);
    k_upper_rows<<<nblk(U), BT, 0, st>>>(up_node.p, up_kind.p, up_ref.p, U, node_of_row.p, lo_row.p, hi_row.p);
    count_launches(1);
    CK(rows.alloc((size_t)M * stride));
    k_permute_rows<<<nblk(M * (stride / 4)), BT, 0, st>>>(node_rec.p, node_of_row.p, M, stride, rows.p);
    count_launches(1);
    DevBuf<UpperEntry> upper;
    CK(upper.alloc(U));
    k_upper_entries<<<nblk(U), BT, 0, st>>>(node_rec.p, stride, up_node.p, up_kind.p, up_parent.p, up_ref.p, U,
                                            upper.p);
    count_launches(1);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));

    DevBuf<int32_t> left_keep, right_keep;
    CK(left_keep.alloc(M)); CK(right_keep.alloc(M));
    CK(cudaMemcpy(left_keep.p, left.p, M * 4, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(right_keep.p, right.p, M * 4, cudaMemcpyDeviceToDevice));
    free_scene(sc);                                  // the previous layout, if any
    sc->n_nodes = M;
    sc->n_leaves = (M + 1) / 2;
    sc->n_upper = U;
    sc->upper_depth = depth;
    sc->n_spt = n_spt;
    sc->n_upper_rows = n_rows_up;
    sc->spt_volume = p.spt_volume;
    sc->kappa = p.kappa;
    sc->d_rows = rows.release();
    sc->d_upper = upper.release();
    sc->d_spt_base = spt_base.release();
    sc->d_lo = lo_row.release();
    sc->d_hi = hi_row.release();
    sc->d_node_rec = nullptr;                        // the canonical copy is not kept: export rebuilds it
    sc->d_left = left_keep.release();
    sc->d_right = right_keep.release();
    sc->d_node_of_row = node_of_row.release();
    sc->d_up_node = up_node.release();
    sc->d_spt_root = spt_root.release();
    sc->root = root;
    return LODGS_OK;
}

int build_scene(const float *leaves, int64_t n, int degree, int on_device, const lodgs_build_params &p,
                lodgs_scene *sc) {
    const int stride = record_stride(degree);
    const int64_t M = 2 * n - 1;
    if (M >= (int64_t)1 << 31) { set_error("build_hierarchy: more than 2^31 nodes"); return LODGS_E_INVALID; }
    cudaStream_t st = 0;
    sc->n_leaves = n; sc->n_nodes = M; sc->sh_degree = degree; sc->stride = stride;
    sc->spt_volume = p.spt_volume; sc->kappa = p.kappa;

    DevBuf<float> node_rec, box, lo_node, hi_node, lo_row, hi_row, rows;
    DevBuf<int32_t> left, right, parent, node_spt_root, node_upper_row, node_of_row;
    CK(node_rec.alloc((size_t)M * stride));
    CK(cudaMemset(node_rec.p, 0, (size_t)M * stride * sizeof(float)));
    CK(cudaMemcpy(node_rec.p, leaves, (size_t)n * stride * sizeof(float),
                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    CK(left.alloc(M)); CK(right.alloc(M)); CK(parent.alloc(M));
    CK(cudaMemset(left.p, 0xff, M * 4)); CK(cudaMemset(right.p, 0xff, M * 4)); CK(cudaMemset(parent.p, 0xff, M * 4));

    // ---- Morton order ----
    DevBuf<uint32_t> k0, k1, v0, v1, hist, dn, hi_g;
    CK(k0.alloc(M)); CK(k1.alloc(M)); CK(v0.alloc(M)); CK(v1.alloc(M)); CK(hi_g.alloc(M));
    CK(hist.alloc(SORT_HIST)); CK(dn.alloc(1));
    CK(box.alloc(6));
    {
        float init[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
        CK(cudaMemcpy(box.p, init, sizeof(init), cudaMemcpyHostToDevice));
    }
    k_aabb<<<std::min(nblk(n), 1184), BT, 0, st>>>(node_rec.p, stride, n, box.p);
    count_launches(1);
    k_morton<<<nblk(n), BT, 0, st>>>(node_rec.p, stride, n, box.p, k0.p, hi_g.p, v0.p);
    count_launches(1);
    uint32_t n32 = (uint32_t)n;
    CK(cudaMemcpy(dn.p, &n32, 4, cudaMemcpyHostToDevice));
    bool alt;
    int rc = radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, dn.p, n32, 0, 32, hist.p, st, &alt);   // low word
    if (rc) return rc;
    uint32_t *ord = alt ? v1.p : v0.p;
    uint32_t *kk = alt ? k0.p : k1.p, *kalt = alt ? k1.p : k0.p, *valt = alt ? v0.p : v1.p;
    k_gather_u32<<<nblk(n), BT, 0, st>>>(hi_g.p, ord, n, kk);
    count_launches(1);
    rc = radix_sort_pairs(kk, ord, kalt, valt, dn.p, n32, 0, 31, hist.p, st, &alt);          // high word
    if (rc) return rc;
    uint32_t *order = alt ? valt : ord;

    // ---- level-wise merges ----
    DevBuf<uint32_t> lvl_a, lvl_b;
    CK(lvl_a.alloc(n)); CK(lvl_b.alloc(n));
    CK(cudaMemcpyAsync(lvl_a.p, order, n * 4, cudaMemcpyDeviceToDevice, st));
    const int ncol = 3 + 3 * sh_count(degree);
    int64_t len = n, next_id = n;
    uint32_t *cur = lvl_a.p, *nxt = lvl_b.p;
    while (len > 1) {
        int64_t npair = len / 2;
        k_merge_level<<<nblk(npair + 1, 128), 128, 0, st>>>(node_rec.p, stride, ncol, cur, len, next_id, nxt,
                                                            left.p, right.p, parent.p);
        count_launches(1);
        next_id += npair;
        len = npair + (len & 1);
        std::swap(cur, nxt);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));

    return build_layout(sc, node_rec.p, left.p, right.p, parent.p, M, (int32_t)(M - 1), p, st);
}

namespace {

// int32 -> int32 map with open addressing (keys >= 0), for the few nodes a
// densification touches out of millions
struct FlatMap {
    std::vector<int64_t> slot;                  // key << 32 | value, or -1
    size_t n = 0, mask = 0;
    FlatMap() { rehash(1024); }
    void rehash(size_t cap) {
        std::vector<int64_t> old;
        old.swap(slot);
        slot.assign(cap, -1);
        mask = cap - 1;
        n = 0;
        for (int64_t kv : old)
            if (kv >= 0) put((int32_t)(kv >> 32), (int32_t)(uint32_t)kv);
    }
    size_t home(int32_t k) const { return (size_t)(((uint64_t)(uint32_t)k * 0x9E3779B97F4A7C15ull) >> 20) & mask; }
    int64_t *find(int32_t k) {
        for (size_t i = home(k);; i = (i + 1) & mask) {
            if (slot[i] < 0) return nullptr;
            if ((int32_t)(slot[i] >> 32) == k) return &slot[i];
        }
    }
    void put(int32_t k, int32_t v) {
        if (2 * (n + 1) > slot.size()) rehash(2 * slot.size());
        for (size_t i = home(k);; i = (i + 1) & mask) {
            if (slot[i] < 0) { slot[i] = (int64_t)k << 32 | (uint32_t)v; ++n; return; }
            if ((int32_t)(slot[i] >> 32) == k) { slot[i] = (int64_t)k << 32 | (uint32_t)v; return; }
        }
    }
    bool get(int32_t k, int32_t *v) {
        const int64_t *p = find(k);
        if (!p) return false;
        *v = (int32_t)(uint32_t)*p;
        return true;
    }
    template <typename F> void each(F f) const {
        for (int64_t kv : slot)
            if (kv >= 0) f((int32_t)(kv >> 32), (int32_t)(uint32_t)kv);
    }
};

// The tree as the host edits it: values of the device arrays (children, parent,
// node of row) fetched for the nodes the operations touch, in batched gathers,
// with the edits kept in an overlay; only the changed entries go back, by
// scatter.  A value outside the prefetched set (a chain of edits reaching
// further) is fetched on its own.
struct TreeView {
    enum Field { LEFT = 0, RIGHT = 1, PARENT = 2, NOR = 3 };
    const int32_t *dev[4];
    FlatMap base[4], edit[3];
    cudaError_t err = cudaSuccess;

    int32_t get(int f, int32_t i) {
        int32_t v;
        if (f < 3 && edit[f].get(i, &v)) return v;
        if (base[f].get(i, &v)) return v;
        v = -1;
        if (i >= 0) {
            cudaError_t e = cudaMemcpy(&v, dev[f] + i, 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) err = e;
        }
        base[f].put(i, v);
        return v;
    }
    void set(int f, int32_t i, int32_t v) { edit[f].put(i, v); }
    // one gather of dev[f] at the given indices (-1 entries skipped) into the base cache
    int prefetch(int f, const std::vector<int32_t> &idx) {
        std::vector<int32_t> want;
        want.reserve(idx.size());
        int32_t v;
        for (int32_t i : idx)
            if (i >= 0 && !base[f].get(i, &v)) want.push_back(i);
        std::sort(want.begin(), want.end());
        want.erase(std::unique(want.begin(), want.end()), want.end());
        if (want.empty()) return LODGS_OK;
        DevBuf<int32_t> d_idx, d_out;
        CK(d_idx.alloc(want.size()));
        CK(d_out.alloc(want.size()));
        CK(cudaMemcpy(d_idx.p, want.data(), want.size() * 4, cudaMemcpyHostToDevice));
        k_gather_i32<<<nblk((int64_t)want.size()), BT>>>(dev[f], d_idx.p, (int64_t)want.size(), d_out.p);
        count_launches(1);
        std::vector<int32_t> got(want.size());
        CK(cudaMemcpy(got.data(), d_out.p, want.size() * 4, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < want.size(); ++k) base[f].put(want[k], got[k]);
        return LODGS_OK;
    }
};

}  // namespace

int densify_scene(lodgs_scene *sc, const lodgs_densify_op *ops, int64_t n_ops, int32_t *old_row_of_new_row,
                  int64_t capacity) {
    if (!sc->d_rows) {
        set_error("scene_densify: the scene's records are not on the device (released to a cache)");
        return LODGS_E_STATE;
    }
    const int stride = sc->stride;
    const int64_t M0 = sc->n_nodes;
    int64_t n_spawn = 0;
    for (int64_t i = 0; i < n_ops; ++i) {
        if (ops[i].kind == LODGS_DENSIFY_SPAWN) ++n_spawn;
        else if (ops[i].kind != LODGS_DENSIFY_RESPAWN) { set_error("scene_densify: unknown operation"); return LODGS_E_INVALID; }
        if (ops[i].target < 0 || ops[i].target >= M0 ||
            (ops[i].kind == LODGS_DENSIFY_RESPAWN && (ops[i].dead < 0 || ops[i].dead >= M0))) {
            set_error("scene_densify: row out of range");
            return LODGS_E_INVALID;
        }
    }
    const int64_t M = M0 + 2 * n_spawn;
    if (M >= (int64_t)1 << 31) { set_error("scene_densify: more than 2^31 nodes"); return LODGS_E_INVALID; }
    if (capacity < M) { set_error("scene_densify: old_row_of_new_row holds fewer than the new node count"); return LODGS_E_INVALID; }
    // parents of the current tree, on the device
    DevBuf<int32_t> d_parent0;
    CK(d_parent0.alloc(M0));
    CK(cudaMemset(d_parent0.p, 0xff, M0 * 4));
    k_parent_of<<<nblk(M0), BT>>>(sc->d_left, sc->d_right, M0, d_parent0.p);
    count_launches(1);
    TreeView tv;
    tv.dev[TreeView::LEFT] = sc->d_left;
    tv.dev[TreeView::RIGHT] = sc->d_right;
    tv.dev[TreeView::PARENT] = d_parent0.p;
    tv.dev[TreeView::NOR] = sc->d_node_of_row;
    // prefetch what the operations read: targets and dead nodes, their parents,
    // the parents' children and parents, and those nodes' children
    {
        std::vector<int32_t> rows_t, v1, v2, v3;
        for (int64_t i = 0; i < n_ops; ++i) {
            rows_t.push_back((int32_t)ops[i].target);
            if (ops[i].kind == LODGS_DENSIFY_RESPAWN) rows_t.push_back((int32_t)ops[i].dead);
        }
        if (int rc = tv.prefetch(TreeView::NOR, rows_t)) return rc;
        for (int32_t r : rows_t) v1.push_back(tv.get(TreeView::NOR, r));
        if (int rc = tv.prefetch(TreeView::LEFT, v1)) return rc;
        if (int rc = tv.prefetch(TreeView::PARENT, v1)) return rc;
        for (int32_t u : v1) v2.push_back(tv.get(TreeView::PARENT, u));
        for (int f : {TreeView::LEFT, TreeView::RIGHT, TreeView::PARENT})
            if (int rc = tv.prefetch(f, v2)) return rc;
        for (int32_t u : v2) v3.push_back(u >= 0 ? tv.get(TreeView::PARENT, u) : -1);
        for (int f : {TreeView::LEFT, TreeView::RIGHT})
            if (int rc = tv.prefetch(f, v3)) return rc;
    }
    FlatMap fresh;                                   // nodes whose record is new (value unused)
    std::vector<int32_t> fresh_ids;
    std::vector<int32_t> trip;                       // (target, child a, child b) per operation
    trip.reserve(3 * n_ops);
    int32_t root = sc->root;
    int32_t next = (int32_t)M0;
    auto L = [&](int32_t u) { return tv.get(TreeView::LEFT, u); };
    auto is_fresh = [&](int32_t u) { int32_t v; return fresh.get(u, &v); };
    for (int64_t i = 0; i < n_ops; ++i) {
        const int32_t T = tv.get(TreeView::NOR, (int32_t)ops[i].target);
        if (L(T) >= 0 || is_fresh(T)) {
            set_error("scene_densify: operation " + std::to_string(i) + ": the target is not an original leaf");
            return LODGS_E_INVALID;
        }
        int32_t a, b;
        if (ops[i].kind == LODGS_DENSIFY_SPAWN) {
            a = next++;
            b = next++;
        } else {
            const int32_t D = tv.get(TreeView::NOR, (int32_t)ops[i].dead);
            const int32_t P = tv.get(TreeView::PARENT, D);
            if (L(D) >= 0 || is_fresh(D) || D == T || P < 0) {
                set_error("scene_densify: operation " + std::to_string(i) +
                          ": the dead node must be an original leaf with a parent, other than the target");
                return LODGS_E_INVALID;
            }
            const int32_t S = tv.get(TreeView::LEFT, P) == D ? tv.get(TreeView::RIGHT, P) : tv.get(TreeView::LEFT, P);
            const int32_t G = tv.get(TreeView::PARENT, P);
            if (G >= 0) {                            // the sibling takes the parent's place
                if (tv.get(TreeView::LEFT, G) == P) tv.set(TreeView::LEFT, G, S);
                else tv.set(TreeView::RIGHT, G, S);
            } else {
                root = S;
            }
            tv.set(TreeView::PARENT, S, G);
            a = P;
            b = D;
        }
        tv.set(TreeView::LEFT, T, a);
        tv.set(TreeView::RIGHT, T, b);
        tv.set(TreeView::PARENT, a, T);
        tv.set(TreeView::PARENT, b, T);
        for (int32_t c : {a, b}) {
            tv.set(TreeView::LEFT, c, -1);
            tv.set(TreeView::RIGHT, c, -1);
        }
        fresh.put(a, 1);
        fresh.put(b, 1);
        fresh_ids.push_back(a);
        fresh_ids.push_back(b);
        trip.push_back(T); trip.push_back(a); trip.push_back(b);
    }
    if (tv.err != cudaSuccess) CK(tv.err);
    // the new topology: the old arrays grown by the spawned nodes, patched with the edits
    DevBuf<int32_t> d_left, d_right, d_parent, d_patch;
    CK(d_left.alloc(M)); CK(d_right.alloc(M)); CK(d_parent.alloc(M));
    CK(cudaMemset(d_left.p, 0xff, M * 4)); CK(cudaMemset(d_right.p, 0xff, M * 4)); CK(cudaMemset(d_parent.p, 0xff, M * 4));
    CK(cudaMemcpy(d_left.p, sc->d_left, M0 * 4, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(d_right.p, sc->d_right, M0 * 4, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(d_parent.p, d_parent0.p, M0 * 4, cudaMemcpyDeviceToDevice));
    {
        size_t most = 0;
        for (auto &e : tv.edit) most = std::max(most, e.n);
        CK(d_patch.alloc(2 * std::max<size_t>(most, 1)));
        int32_t *dst[3] = {d_left.p, d_right.p, d_parent.p};
        std::vector<int32_t> kv;
        for (int f = 0; f < 3; ++f) {
            if (!tv.edit[f].n) continue;
            kv.clear();
            tv.edit[f].each([&](int32_t k, int32_t v) { kv.push_back(k); kv.push_back(v); });
            CK(cudaMemcpy(d_patch.p, kv.data(), kv.size() * 4, cudaMemcpyHostToDevice));
            k_scatter_i32<<<nblk((int64_t)tv.edit[f].n), BT>>>(dst[f], d_patch.p, (int64_t)tv.edit[f].n);
            count_launches(1);
        }
    }
    // the records: canonical order on the device, children written by one kernel
    // (targets are original leaves, never rewritten within a batch, so the
    // operations' splits are independent)
    DevBuf<float> node_rec;
    DevBuf<int32_t> d_trip, old_row_of, d_fresh_ids;
    DevBuf<uint8_t> d_fresh;
    CK(node_rec.alloc((size_t)M * stride));
    CK(d_trip.alloc(trip.size()));
    CK(cudaMemcpy(d_trip.p, trip.data(), trip.size() * 4, cudaMemcpyHostToDevice));
    k_unpermute_rows<<<nblk(M0 * (stride / 4)), BT>>>(sc->d_rows, sc->d_node_of_row, M0, stride, node_rec.p);
    count_launches(1);
    if (n_ops > 0) {
        k_split_children<<<nblk(n_ops * stride), BT>>>(node_rec.p, stride, d_trip.p, n_ops);
        count_launches(1);
    }
    // what the row map needs from the old layout
    CK(old_row_of.alloc(M0));
    k_row_of_node<<<nblk(M0), BT>>>(sc->d_node_of_row, M0, old_row_of.p);
    CK(d_fresh.alloc(M));
    CK(cudaMemset(d_fresh.p, 0, M));
    CK(d_fresh_ids.alloc(fresh_ids.size()));
    if (!fresh_ids.empty()) {
        CK(cudaMemcpy(d_fresh_ids.p, fresh_ids.data(), fresh_ids.size() * 4, cudaMemcpyHostToDevice));
        k_mark<<<nblk((int64_t)fresh_ids.size()), BT>>>(d_fresh.p, d_fresh_ids.p, (int64_t)fresh_ids.size());
    }
    count_launches(2);
    CK(cudaGetLastError());
    lodgs_build_params p{sc->spt_volume, sc->kappa};
    if (int rc = build_layout(sc, node_rec.p, d_left.p, d_right.p, d_parent.p, M, root, p, 0)) return rc;
    sc->layout_version++;
    k_row_map<<<nblk(M), BT>>>(sc->d_node_of_row, M, M0, old_row_of.p, d_fresh.p, old_row_of_new_row);
    count_launches(1);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    return LODGS_OK;
}

// ---- checkpoint ------------------------------------------------------------
// File: "LODGSCN1", u32 version 1, u32 SH degree, u32 stride, u32 0, i64 node
// count, i64 root, f32 spt_volume, f32 kappa, the canonical node records
// (n x stride f32), left and right children (n i32 each), then the FNV-1a
// hash (u64) of everything before it.  The HSPT and SPT layout is not stored:
// the load rebuilds it, and the rebuild is deterministic.
namespace {
constexpr char CKPT_MAGIC[8] = {'L', 'O', 'D', 'G', 'S', 'C', 'N', '1'};

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
};

struct File {
    FILE *f = nullptr;
    ~File() { if (f) fclose(f); }
};
}  // namespace

int save_scene(const lodgs_scene *sc, const char *path) {
    if (!sc->d_rows) {
        set_error("scene_save: the scene's records are not on the device (released to a cache)");
        return LODGS_E_STATE;
    }
    const int64_t M = sc->n_nodes;
    const int stride = sc->stride;
    DevBuf<float> node_rec;
    CK(node_rec.alloc((size_t)M * stride));
    k_unpermute_rows<<<nblk(M * (stride / 4)), BT>>>(sc->d_rows, sc->d_node_of_row, M, stride, node_rec.p);
    count_launches(1);
    std::vector<float> rec((size_t)M * stride);
    std::vector<int32_t> left(M), right(M);
    CK(cudaMemcpy(rec.data(), node_rec.p, rec.size() * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(left.data(), sc->d_left, M * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(right.data(), sc->d_right, M * 4, cudaMemcpyDeviceToHost));
    File fh;
    fh.f = fopen(path, "wb");
    if (!fh.f) { set_error(std::string("scene_save: cannot open ") + path); return LODGS_E_INVALID; }
    Fnv h;
    const uint32_t head[4] = {1u, (uint32_t)sc->sh_degree, (uint32_t)stride, 0u};
    const int64_t nr[2] = {M, (int64_t)sc->root};
    const float pr[2] = {sc->spt_volume, sc->kappa};
    auto put = [&](const void *p, size_t n) {
        h.add(p, n);
        return fwrite(p, 1, n, fh.f) == n;
    };
    bool ok = put(CKPT_MAGIC, 8) && put(head, sizeof(head)) && put(nr, sizeof(nr)) && put(pr, sizeof(pr)) &&
              put(rec.data(), rec.size() * 4) && put(left.data(), M * 4) && put(right.data(), M * 4);
    ok = ok && fwrite(&h.h, 1, 8, fh.f) == 8;
    if (!ok) { set_error(std::string("scene_save: write failed: ") + path); return LODGS_E_INVALID; }
    return LODGS_OK;
}

int load_scene(const char *path, lodgs_scene *sc) {
    File fh;
    fh.f = fopen(path, "rb");
    if (!fh.f) { set_error(std::string("scene_load: cannot open ") + path); return LODGS_E_INVALID; }
    Fnv h;
    auto get = [&](void *p, size_t n) {
        if (fread(p, 1, n, fh.f) != n) return false;
        h.add(p, n);
        return true;
    };
    char magic[8];
    uint32_t head[4];
    int64_t nr[2];
    float pr[2];
    if (!get(magic, 8) || memcmp(magic, CKPT_MAGIC, 8) != 0 || !get(head, sizeof(head)) || head[0] != 1u ||
        !get(nr, sizeof(nr)) || !get(pr, sizeof(pr))) {
        set_error("scene_load: not a scene checkpoint (magic or version)");
        return LODGS_E_INVALID;
    }
    const int degree = (int)head[1], stride = (int)head[2];
    const int64_t M = nr[0];
    const int64_t root = nr[1];
    if (degree < 0 || degree > 3 || stride != record_stride(degree) || M < 1 || M >= ((int64_t)1 << 31) ||
        (M & 1) == 0 || root < 0 || root >= M) {
        set_error("scene_load: inconsistent header");
        return LODGS_E_INVALID;
    }
    std::vector<float> rec((size_t)M * stride);
    std::vector<int32_t> left(M), right(M);
    uint64_t want = 0;
    if (!get(rec.data(), rec.size() * 4) || !get(left.data(), M * 4) || !get(right.data(), M * 4) ||
        fread(&want, 1, 8, fh.f) != 8) {
        set_error("scene_load: truncated file");
        return LODGS_E_INVALID;
    }
    if (want != h.h) { set_error("scene_load: checksum mismatch (corrupted file)"); return LODGS_E_INVALID; }
    // the hierarchy must be a full binary tree over all nodes, rooted at `root`
    std::vector<int32_t> parent(M, -1);
    int64_t leaves = 0;
    for (int64_t u = 0; u < M; ++u) {
        const int32_t l = left[u], r = right[u];
        if ((l < 0) != (r < 0) || l >= M || r >= M || l == u || r == u) {
            set_error("scene_load: invalid children");
            return LODGS_E_INVALID;
        }
        if (l < 0) { ++leaves; continue; }
        if (parent[l] >= 0 || parent[r] >= 0 || l == r) { set_error("scene_load: a node with two parents"); return LODGS_E_INVALID; }
        parent[l] = (int32_t)u;
        parent[r] = (int32_t)u;
    }
    int64_t seen = 0;
    {
        std::vector<int32_t> stack{(int32_t)root};
        while (!stack.empty() && seen <= M) {
            const int32_t u = stack.back();
            stack.pop_back();
            ++seen;
            if (left[u] >= 0) { stack.push_back(left[u]); stack.push_back(right[u]); }
        }
    }
    if (parent[root] >= 0 || seen != M || 2 * leaves - 1 != M) {
        set_error("scene_load: the hierarchy is not one tree over all nodes");
        return LODGS_E_INVALID;
    }
    sc->sh_degree = degree;
    sc->stride = stride;
    DevBuf<float> d_rec;
    DevBuf<int32_t> d_left, d_right, d_parent;
    CK(d_rec.alloc(rec.size())); CK(d_left.alloc(M)); CK(d_right.alloc(M)); CK(d_parent.alloc(M));
    CK(cudaMemcpy(d_rec.p, rec.data(), rec.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_left.p, left.data(), M * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_right.p, right.data(), M * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_parent.p, parent.data(), M * 4, cudaMemcpyHostToDevice));
    lodgs_build_params p{pr[0], pr[1]};
    return build_layout(sc, d_rec.p, d_left.p, d_right.p, d_parent.p, M, (int32_t)root, p, 0);
}

}  // namespace lodgs
