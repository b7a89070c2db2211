/*
 * lodgs_oracle.c -- plain, slow CPU oracle for the LoD Gaussian render path of
 * "A LoD of Gaussians" (arxiv 2507.01110).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, imports or
 * calls this file; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg use it.  It shares no code, header or table with the CUDA
 * path.
 *
 * Values (merged attributes, projected means and conics, colours, alphas,
 * images, gradients) are computed in float64.  The decisions that turn floats
 * into integers -- Morton codes, the HSPT volume test, the LoD/cull tests of the
 * cut, the tile rectangle, the depth key and the per-pixel support test -- are
 * taken in float32 with the exact expressions below, so that an independent
 * implementation that evaluates the same expressions in IEEE float32 (no fused
 * multiply-add except where written as fmaf) reaches the same decisions.
 *
 * FP32 decision expressions (all operations IEEE round-to-nearest):
 *   D1 Morton   u = (mu_a - lo_a) / (hi_a - lo_a)   (0 if hi_a == lo_a)
 *               q_a = (uint32) fminf(u * 2097152.0f, 2097151.0f)
 *               code bit 3b+2 = bit b of q_x, 3b+1 of q_y, 3b of q_z
 *   D2 volume   vol = (s0 * s1) * s2 ; node is an SPT root iff vol < spt_volume
 *   D3 size     S = sqrtf(((s0*s1 + s0*s2) + s1*s2) / 3.0f)
 *   D4 spread   e = sqrtf((dx*dx + dy*dy) + dz*dz),  d = mu_i - mu_root
 *               lo_raw = S + e / kappa        (leaves: lo' = 0)
 *   D5 camera   d = mu - pos ; dist = sqrtf((dx*dx + dy*dy) + dz*dz)
 *               t_a = (R[a][0]*dx + R[a][1]*dy) + R[a][2]*dz
 *               x = dist * inv_k,  inv_k = tau / fx
 *   D6 cull     r = 3.0f * fmaxf(fmaxf(s0, s1), s2)
 *               culled iff tz + r < znear, or for a side plane n:
 *               ((n0*tx + n1*ty) + n2*tz) < -r
 *   D7 project  see project_fp32() below (visibility, rectangle, depth key)
 *   D8 support  dx = u - (px + 0.5f), dy = v - (py + 0.5f)
 *               p = fmaf(nb*dx, dy, fmaf(nhc*dy, dy, (nha*dx)*dx))
 *               nha = -0.5f*A, nhc = -0.5f*C, nb = -B ; support iff p >= -4.5f
 *   D9 tile     a (tile, Gaussian) pair is kept iff the support ellipse can
 *               reach a pixel centre of the tile: see tile_keep() below
 *   D10 block   the CUDA blend's 8x8-block skip test (support half extents
 *               rx, ry from the 2D covariance, then a box test): written here
 *               only as a standalone predicate, or_block_keep(), so that tests
 *               can check by brute force that it never skips a pixel passing
 *               D8.  The oracle's own blend and backward do not use it: they
 *               evaluate D8 on every (pixel, listed Gaussian).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 *
 * The OpenMP pragmas below take effect only in the separate -fopenmp build that
 * the benchmark times as its all-cores CPU baseline (pixel rows and Gaussians
 * in parallel, the backward's per-Gaussian sums by atomic adds).  The default
 * build, which every test uses, ignores them and runs one thread in the order
 * written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* threads of the OpenMP build (1 without OpenMP) */
int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

enum { REC_MU = 0, REC_S = 3, REC_Q = 6, REC_OP = 10, REC_B = 11, REC_F = 14 };
enum { KIND_INTERNAL = 0, KIND_LEAF = 1, KIND_SPT = 2 };
enum { TILE = 16 };
#define T_MIN 1e-4
#define ALPHA_MAX 0.99
#define DILATION 0.3
#define SUPPORT_P (-4.5f)
#define F32_N 7          /* float32 decision values per Gaussian: u, v, A, B, C, rx, ry */

int or_stride(int degree) {
    int k = 14 + 3 * ((degree + 1) * (degree + 1) - 1);
    return (k + 7) / 8 * 8;
}
static int sh_count(int degree) { return (degree + 1) * (degree + 1) - 1; }

/* ------------------------------------------------------------------------- */
/* Morton order of the leaves (pairing order of the hierarchy merge).         */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t code; int64_t idx; } morton_t;

static int cmp_morton(const void *a, const void *b) {
    const morton_t *x = a, *y = b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static uint64_t morton_interleave(uint32_t qx, uint32_t qy, uint32_t qz) {
    uint64_t code = 0;
    for (int b = 0; b < 21; ++b) {
        code |= (uint64_t)((qx >> b) & 1u) << (3 * b + 2);
        code |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
        code |= (uint64_t)((qz >> b) & 1u) << (3 * b + 0);
    }
    return code;
}

uint64_t or_morton_code(float mx, float my, float mz, const float *lo, const float *hi) {
    float m[3] = {mx, my, mz};
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        float ext = hi[a] - lo[a];
        float u = ext > 0.0f ? (m[a] - lo[a]) / ext : 0.0f;
        q[a] = (uint32_t)fminf(u * 2097152.0f, 2097151.0f);
    }
    return morton_interleave(q[0], q[1], q[2]);
}

/* order[k] = index of the k-th leaf in ascending (Morton code, index) order. */
int or_morton_order(int64_t n, int stride, const float *rec, int64_t *order) {
    if (n <= 0) return 0;
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = rec[REC_MU + a];
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float v = rec[i * stride + REC_MU + a];
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    morton_t *m = malloc(sizeof(morton_t) * (size_t)n);
    if (!m) return -1;
    for (int64_t i = 0; i < n; ++i) {
        const float *r = rec + i * stride;
        m[i].code = or_morton_code(r[0], r[1], r[2], lo, hi);
        m[i].idx = i;
    }
    qsort(m, (size_t)n, sizeof(morton_t), cmp_morton);
    for (int64_t i = 0; i < n; ++i) order[i] = m[i].idx;
    free(m);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Merge of two Gaussians into their parent (the hierarchy of Sec. 3: a parent */
/* approximates its two children).  Reading: weights w = sigma * A with A the  */
/* surface term s1s2+s1s3+s2s3; moment-matched mean and covariance; scales and */
/* rotation from the eigen-decomposition; opacity preserving sigma*A.          */
/* ------------------------------------------------------------------------- */
static void quat_to_rot_d(const double q[4], double R[3][3]) {
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

/* Sigma = R diag(s^2) R^T of a stored record, in float64. */
static void record_cov_d(const float *rec, double C[3][3]) {
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

/* Cyclic Jacobi eigenvalue iteration for a symmetric 3x3 matrix
 * (Golub & Van Loan, "Matrix Computations", Sec. 8.5, symmetric Schur rotations).
 * On return A is (numerically) diagonal and the columns of V are eigenvectors. */
void or_jacobi3(double A[3][3], double V[3][3]) {
    static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
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

/* Symmetric PSD 3x3 -> scales (descending) and unit quaternion (w >= 0).
 * Eigenvector signs: the largest-magnitude component of each column is made
 * positive, then column 3 is negated if det < 0 (a proper rotation). */
void or_cov_to_scale_rot(const double Cin[3][3], double s[3], double q[4]) {
    double A[3][3], V[3][3];
    memcpy(A, Cin, sizeof(A));
    or_jacobi3(A, V);
    double lam[3] = {A[0][0], A[1][1], A[2][2]};
    int ord[3] = {0, 1, 2};
    for (int i = 0; i < 3; ++i)          /* stable descending sort of 3 items */
        for (int j = 0; j < 2 - i; ++j)
            if (lam[ord[j]] < lam[ord[j + 1]]) { int t = ord[j]; ord[j] = ord[j + 1]; ord[j + 1] = t; }
    double R[3][3];
    for (int k = 0; k < 3; ++k) {
        s[k] = sqrt(lam[ord[k]] > 0.0 ? lam[ord[k]] : 0.0);
        for (int i = 0; i < 3; ++i) R[i][k] = V[i][ord[k]];
    }
    for (int k = 0; k < 3; ++k) {
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
    /* rotation matrix -> quaternion (Shepperd's branch on the largest diagonal term) */
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
    q[0] = w / n; q[1] = x / n; q[2] = y / n; q[3] = z / n;
}

/* parent record from two child records (float32 in, float64 math, float32 out) */
void or_merge_pair(int stride, int degree, const float *ra, const float *rb, float *out) {
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
    for (int a = 0; a < 3; ++a)
        mu[a] = (w[0] * rc[0][REC_MU + a] + w[1] * rc[1][REC_MU + a]) / W;
    double C[3][3] = {{0}};
    for (int k = 0; k < 2; ++k) {
        double Ck[3][3], d[3];
        record_cov_d(rc[k], Ck);
        for (int a = 0; a < 3; ++a) d[a] = rc[k][REC_MU + a] - mu[a];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) C[i][j] += w[k] * (Ck[i][j] + d[i] * d[j]);
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i][j] = C[i][j] / W;
    double s[3], q[4];
    or_cov_to_scale_rot(C, s, q);
    double Ap = s[0] * s[1] + s[0] * s[2] + s[1] * s[2];
    double num = (double)ra[REC_OP] * A[0] + (double)rb[REC_OP] * A[1];
    double op = Ap > 0.0 ? num / Ap : (double)ra[REC_OP] + (double)rb[REC_OP];
    if (op > 1.0) op = 1.0;
    memset(out, 0, sizeof(float) * (size_t)stride);
    for (int a = 0; a < 3; ++a) out[REC_MU + a] = (float)mu[a];
    for (int a = 0; a < 3; ++a) out[REC_S + a] = (float)s[a];
    for (int a = 0; a < 4; ++a) out[REC_Q + a] = (float)q[a];
    out[REC_OP] = (float)op;
    int nc = 3 + 3 * sh_count(degree);   /* base colour + SH coefficients */
    for (int k = 0; k < nc; ++k)
        out[REC_B + k] = (float)((w[0] * rc[0][REC_B + k] + w[1] * rc[1][REC_B + k]) / W);
}

/* Binary hierarchy by level-wise pairwise merging in Morton order.
 * Node ids: leaves 0..n-1 (input order), internal nodes n, n+1, ... in creation
 * order (level by level, pair by pair); an odd last node of a level is carried
 * up unchanged.  The root is node 2n-2 (0 when n == 1). */
int or_merge(int64_t n, int stride, int degree, const float *leaf_rec, const int64_t *order,
             float *node_rec, int64_t *left, int64_t *right, int64_t *parent) {
    if (n <= 0) return -1;
    int64_t M = 2 * n - 1;
    memcpy(node_rec, leaf_rec, sizeof(float) * (size_t)(n * stride));
    for (int64_t i = 0; i < M; ++i) { left[i] = right[i] = parent[i] = -1; }
    int64_t *cur = malloc(sizeof(int64_t) * (size_t)n), *nxt = malloc(sizeof(int64_t) * (size_t)n);
    if (!cur || !nxt) { free(cur); free(nxt); return -1; }
    memcpy(cur, order, sizeof(int64_t) * (size_t)n);
    int64_t len = n, next_id = n;
    while (len > 1) {
        int64_t nl = 0;
        for (int64_t k = 0; k + 1 < len; k += 2) {
            int64_t a = cur[k], b = cur[k + 1], p = next_id++;
            or_merge_pair(stride, degree, node_rec + a * stride, node_rec + b * stride, node_rec + p * stride);
            left[p] = a; right[p] = b; parent[a] = p; parent[b] = p;
            nxt[nl++] = p;
        }
        if (len & 1) nxt[nl++] = cur[len - 1];
        int64_t *t = cur; cur = nxt; nxt = t;
        len = nl;
    }
    free(cur); free(nxt);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* HSPT construction (Sec. 4.3): BFS cut of the hierarchy on the volume test   */
/* s1*s2*s3 < size; cut nodes root SPTs (Sec. 4.1), the rest is the upper      */
/* hierarchy.  SPT intervals follow Eq. 4 with the size metric of Eq. 6 read   */
/* as m_d = k*S, the conservative spread term e = |mu_i - mu_root| folded in   */
/* (the M_d of Sec. 4.1), and top-down clamping so that nodes whose parent     */
/* interval lies below their own are never selected (appendix "Unreachable     */
/* Gaussians").                                                                */
/* ------------------------------------------------------------------------- */
static float size_S(const float *r) {
    float s0 = r[REC_S], s1 = r[REC_S + 1], s2 = r[REC_S + 2];
    return sqrtf(((s0 * s1 + s0 * s2) + s1 * s2) / 3.0f);
}
static float max_scale(const float *r) { return fmaxf(fmaxf(r[REC_S], r[REC_S + 1]), r[REC_S + 2]); }

typedef struct { float hi; int64_t node; float lo; } sptent_t;
static int cmp_sptent(const void *a, const void *b) {
    const sptent_t *x = a, *y = b;
    if (x->hi != y->hi) return x->hi > y->hi ? -1 : 1;     /* hi descending */
    return (x->node > y->node) - (x->node < y->node);       /* node ascending */
}

/* Outputs (capacities M):
 *  counts[0] = n_upper, counts[1] = n_spt, counts[2] = n_rows_upper
 *  up_node[u], up_kind[u], up_parent[u], up_child[2u], up_child[2u+1], up_ref[u]
 *     (ref: render row for INTERNAL/LEAF, SPT index for SPT)
 *  spt_root[j], spt_base[j], spt_count[j]
 *  node_of_row[row], row_of_node[node], lo_row[row], hi_row[row], lo_raw_node[node] */
int or_hspt(int64_t M, int stride, const float *rec, const int64_t *left, const int64_t *right,
            int64_t root, float spt_volume, float kappa, int64_t *counts,
            int64_t *up_node, int32_t *up_kind, int64_t *up_parent, int64_t *up_child, int64_t *up_ref,
            int64_t *spt_root, int64_t *spt_base, int64_t *spt_count,
            int64_t *node_of_row, int64_t *row_of_node, float *lo_row, float *hi_row, float *lo_raw_node) {
    int64_t *queue = malloc(sizeof(int64_t) * (size_t)M), *qpar = malloc(sizeof(int64_t) * (size_t)M);
    int64_t *u_of_node = malloc(sizeof(int64_t) * (size_t)M);
    if (!queue || !qpar || !u_of_node) return -1;
    for (int64_t i = 0; i < M; ++i) { row_of_node[i] = -1; u_of_node[i] = -1; }
    int64_t head = 0, tail = 0, nu = 0, ns = 0, nrow = 0;
    queue[tail] = root; qpar[tail++] = -1;
    while (head < tail) {                                    /* Algorithm 1 */
        int64_t node = queue[head], pu = qpar[head++];
        const float *r = rec + node * stride;
        int64_t u = nu++;
        u_of_node[node] = u;
        up_node[u] = node; up_parent[u] = pu; up_child[2 * u] = up_child[2 * u + 1] = -1;
        if (pu >= 0) {
            if (up_child[2 * pu] < 0) up_child[2 * pu] = u; else up_child[2 * pu + 1] = u;
        }
        float vol = (r[REC_S] * r[REC_S + 1]) * r[REC_S + 2];
        if (vol < spt_volume) {
            up_kind[u] = KIND_SPT; up_ref[u] = ns; spt_root[ns++] = node;
        } else if (left[node] < 0) {
            up_kind[u] = KIND_LEAF; up_ref[u] = nrow; node_of_row[nrow] = node; row_of_node[node] = nrow; ++nrow;
        } else {
            up_kind[u] = KIND_INTERNAL; up_ref[u] = nrow; node_of_row[nrow] = node; row_of_node[node] = nrow; ++nrow;
            queue[tail] = left[node]; qpar[tail++] = u;
            queue[tail] = right[node]; qpar[tail++] = u;
        }
    }
    counts[0] = nu; counts[1] = ns; counts[2] = nrow;
    /* SPT layout: clamped intervals, sorted by hi descending (ties: node id) */
    sptent_t *ent = malloc(sizeof(sptent_t) * (size_t)M);
    int64_t *stack = malloc(sizeof(int64_t) * (size_t)M);
    float *lo_clamped = malloc(sizeof(float) * (size_t)M);
    if (!ent || !stack || !lo_clamped) return -1;
    for (int64_t j = 0; j < ns; ++j) {
        int64_t r0 = spt_root[j];
        const float *rr = rec + r0 * stride;
        int64_t cnt = 0, sp = 0;
        stack[sp++] = r0;
        while (sp > 0) {                                     /* pre-order walk: parents before children */
            int64_t node = stack[--sp];
            const float *r = rec + node * stride;
            float dx = r[REC_MU] - rr[REC_MU], dy = r[REC_MU + 1] - rr[REC_MU + 1], dz = r[REC_MU + 2] - rr[REC_MU + 2];
            float e = sqrtf((dx * dx + dy * dy) + dz * dz);
            float lraw = size_S(r) + e / kappa;
            lo_raw_node[node] = lraw;
            float hi, lo;
            if (node == r0) {
                hi = INFINITY;
                lo = lraw;
            } else {
                hi = lo_clamped[node];                        /* stashed by the parent below */
                lo = fminf(lraw, hi);
            }
            if (left[node] < 0) lo = 0.0f;
            ent[cnt].hi = hi; ent[cnt].lo = lo; ent[cnt].node = node; ++cnt;
            if (left[node] >= 0) {
                lo_clamped[left[node]] = lo;                  /* child's hi = this node's clamped lo */
                lo_clamped[right[node]] = lo;
                stack[sp++] = right[node];
                stack[sp++] = left[node];
            }
        }
        qsort(ent, (size_t)cnt, sizeof(sptent_t), cmp_sptent);
        spt_base[j] = nrow; spt_count[j] = cnt;
        for (int64_t e = 0; e < cnt; ++e) {
            node_of_row[nrow] = ent[e].node; row_of_node[ent[e].node] = nrow;
            lo_row[nrow] = ent[e].lo; hi_row[nrow] = ent[e].hi; ++nrow;
        }
    }
    for (int64_t rw = 0; rw < counts[2]; ++rw) { lo_row[rw] = NAN; hi_row[rw] = NAN; }
    free(ent); free(stack); free(lo_clamped); free(queue); free(qpar); free(u_of_node);
    return nrow == M ? 0 : -2;
}

/* ------------------------------------------------------------------------- */
/* Camera constants (float32, D5/D6/D7).                                      */
/* cam[] = R[9] (world->camera, row-major), pos[3], fx, fy, cx, cy, W, H,      */
/*         tau, znear                                                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    float R[3][3], pos[3], fx, fy, cx, cy, tau, znear, inv_k, limx, limy;
    float spt_scale;      /* factor on the SPT root distances (training LoD noise; 1 = none) */
    float plane[4][3];
    int W, H, TX, TY;
} cam_t;

static void cam_setup(const float *c, cam_t *k) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) k->R[i][j] = c[3 * i + j];
    for (int a = 0; a < 3; ++a) k->pos[a] = c[9 + a];
    k->fx = c[12]; k->fy = c[13]; k->cx = c[14]; k->cy = c[15];
    k->W = (int)c[16]; k->H = (int)c[17]; k->tau = c[18]; k->znear = c[19];
    k->TX = (k->W + TILE - 1) / TILE; k->TY = (k->H + TILE - 1) / TILE;
    k->inv_k = k->tau / k->fx;
    k->spt_scale = c[20] > 0.0f ? c[20] : 1.0f;
    float fW = (float)k->W, fH = (float)k->H;
    k->limx = 1.3f * ((0.5f * fW) / k->fx);
    k->limy = 1.3f * ((0.5f * fH) / k->fy);
    float l;
    l = sqrtf(k->fx * k->fx + k->cx * k->cx);
    k->plane[0][0] = k->fx / l; k->plane[0][1] = 0.0f; k->plane[0][2] = k->cx / l;
    float wr = fW - k->cx;
    l = sqrtf(k->fx * k->fx + wr * wr);
    k->plane[1][0] = -k->fx / l; k->plane[1][1] = 0.0f; k->plane[1][2] = wr / l;
    l = sqrtf(k->fy * k->fy + k->cy * k->cy);
    k->plane[2][0] = 0.0f; k->plane[2][1] = k->fy / l; k->plane[2][2] = k->cy / l;
    float hb = fH - k->cy;
    l = sqrtf(k->fy * k->fy + hb * hb);
    k->plane[3][0] = 0.0f; k->plane[3][1] = -k->fy / l; k->plane[3][2] = hb / l;
}

static void cam_view(const cam_t *k, const float *mu, float t[3], float *dist) {
    float dx = mu[0] - k->pos[0], dy = mu[1] - k->pos[1], dz = mu[2] - k->pos[2];
    *dist = sqrtf((dx * dx + dy * dy) + dz * dz);
    for (int a = 0; a < 3; ++a) t[a] = (k->R[a][0] * dx + k->R[a][1] * dy) + k->R[a][2] * dz;
}

static int cam_culled(const cam_t *k, const float t[3], float maxs) {
    float r = 3.0f * maxs;
    if (t[2] + r < k->znear) return 1;
    for (int p = 0; p < 4; ++p) {
        float s = (k->plane[p][0] * t[0] + k->plane[p][1] * t[1]) + k->plane[p][2] * t[2];
        if (s < -r) return 1;
    }
    return 0;
}

/* Frustum test of one sphere (centre mu, radius 3 * maxs) for camera cam[]:
 * 1 iff Sec. 4.3 "Frustum Culling" drops it (D5, D6). */
int or_cull_sphere(const float *cam, const float *mu, float maxs) {
    cam_t k;
    cam_setup(cam, &k);
    float t[3], dist;
    cam_view(&k, mu, t, &dist);
    return cam_culled(&k, t, maxs);
}

/* ------------------------------------------------------------------------- */
/* LoD cut: Algorithm 1 on the upper hierarchy (with frustum culling, Sec.     */
/* 4.3 "Frustum Culling") then Algorithm 2 per selected SPT at the shared root */
/* distance (Eq. 4).  Output rows ascending.  stats: [0] upper nodes visited,  */
/* [1] culled, [2] SPTs cut, [3] SPT entries scanned, [4] selected.           */
/* ------------------------------------------------------------------------- */
static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

typedef struct { int64_t j; float x; } sptq_t;

static int64_t upper_bfs(int64_t n_upper, const int64_t *up_node, const int32_t *up_kind,
                         const int64_t *up_child, const int64_t *up_ref, int stride, const float *node_rec,
                         const cam_t *k, int cull, int64_t *sel, int64_t *nsel, sptq_t *sq, int64_t *nsq,
                         int64_t *stats) {
    int64_t *queue = malloc(sizeof(int64_t) * (size_t)(n_upper + 1));
    int64_t head = 0, tail = 0;
    if (n_upper > 0) queue[tail++] = 0;
    while (head < tail) {
        int64_t u = queue[head++];
        const float *r = node_rec + up_node[u] * stride;
        float t[3], dist;
        cam_view(k, r + REC_MU, t, &dist);
        stats[0]++;
        if (cull && cam_culled(k, t, max_scale(r))) { stats[1]++; continue; }
        float x = dist * k->inv_k;
        /* LoD noise of training (appendix "Varying level of detail"): the distances to
         * the SPT roots are multiplied by a factor (1 + 5 r^4, drawn by the caller) */
        if (up_kind[u] == KIND_SPT) { sq[*nsq].j = up_ref[u]; sq[*nsq].x = x * k->spt_scale; (*nsq)++; }
        else if (up_kind[u] == KIND_LEAF) sel[(*nsel)++] = up_ref[u];
        else if (size_S(r) <= x) sel[(*nsel)++] = up_ref[u];
        else { queue[tail++] = up_child[2 * u]; queue[tail++] = up_child[2 * u + 1]; }
    }
    free(queue);
    return 0;
}

int or_select(int64_t n_upper, const int64_t *up_node, const int32_t *up_kind, const int64_t *up_child,
              const int64_t *up_ref, const int64_t *spt_base, const float *lo_row, const float *hi_row,
              int stride, const float *node_rec, const float *cam, int cull,
              int64_t *sel, int64_t *n_sel, int64_t *stats) {
    cam_t k;
    cam_setup(cam, &k);
    for (int i = 0; i < 5; ++i) stats[i] = 0;
    sptq_t *sq = malloc(sizeof(sptq_t) * (size_t)(n_upper + 1));
    int64_t ns = 0, nq = 0;
    upper_bfs(n_upper, up_node, up_kind, up_child, up_ref, stride, node_rec, &k, cull, sel, &ns, sq, &nq, stats);
    for (int64_t q = 0; q < nq; ++q) {                       /* Algorithm 2 */
        int64_t j = sq[q].j, base = spt_base[j];
        float x = sq[q].x;
        /* high = number of entries with hi > x (binary search on hi, descending);
         * the entry count of SPT j is spt_base[j+1] - spt_base[j] (spt_base has
         * n_spt + 1 entries, the last one being the row count M) */
        int64_t a = 0, b = spt_base[j + 1] - base;
        while (a < b) {
            int64_t m = a + (b - a) / 2;
            if (hi_row[base + m] > x) a = m + 1; else b = m;
        }
        int64_t high = a;
        stats[2]++; stats[3] += high;
        for (int64_t e = 0; e < high; ++e)
            if (lo_row[base + e] <= x) sel[ns++] = base + e;
    }
    qsort(sel, (size_t)ns, sizeof(int64_t), cmp_i64);
    *n_sel = ns;
    stats[4] = ns;
    free(sq);
    return 0;
}

/* Algorithm 1 alone (upper BFS with culling): the upper entries it selects and
 * the SPT roots it reaches, in the order it reaches them, each with its query
 * x_j (LoD noise factor applied).  The out-of-core cache model decides per SPT
 * root from these (Sec. 4.4, Eq. 7). */
int or_select_upper(int64_t n_upper, const int64_t *up_node, const int32_t *up_kind, const int64_t *up_child,
                    const int64_t *up_ref, int stride, const float *node_rec, const float *cam, int cull,
                    int64_t *sel, int64_t *n_sel, int64_t *spt_j, float *spt_x, int64_t *n_spt) {
    cam_t k;
    cam_setup(cam, &k);
    int64_t stats[5] = {0};
    sptq_t *sq = malloc(sizeof(sptq_t) * (size_t)(n_upper + 1));
    int64_t ns = 0, nq = 0;
    upper_bfs(n_upper, up_node, up_kind, up_child, up_ref, stride, node_rec, &k, cull, sel, &ns, sq, &nq, stats);
    for (int64_t q = 0; q < nq; ++q) { spt_j[q] = sq[q].j; spt_x[q] = sq[q].x; }
    *n_sel = ns;
    *n_spt = nq;
    free(sq);
    return 0;
}

/* Independent check of the SPT step: top-down recursive descent inside each SPT
 * selecting the first node on every root-to-leaf path whose unclamped lo_raw
 * satisfies lo_raw <= x (leaves always qualify).  Returns rows ascending. */
static void descend(int64_t node, float x, const int64_t *left, const int64_t *right,
                    const float *lo_raw_node, const int64_t *row_of_node, int64_t *sel, int64_t *ns) {
    if (left[node] < 0 || lo_raw_node[node] <= x) { sel[(*ns)++] = row_of_node[node]; return; }
    descend(left[node], x, left, right, lo_raw_node, row_of_node, sel, ns);
    descend(right[node], x, left, right, lo_raw_node, row_of_node, sel, ns);
}

int or_select_bruteforce(int64_t n_upper, const int64_t *up_node, const int32_t *up_kind, const int64_t *up_child,
                         const int64_t *up_ref, const int64_t *spt_root, const int64_t *left, const int64_t *right,
                         const float *lo_raw_node, const int64_t *row_of_node, int stride, const float *node_rec,
                         const float *cam, int cull, int64_t *sel, int64_t *n_sel) {
    cam_t k;
    cam_setup(cam, &k);
    int64_t stats[5] = {0};
    sptq_t *sq = malloc(sizeof(sptq_t) * (size_t)(n_upper + 1));
    int64_t ns = 0, nq = 0;
    upper_bfs(n_upper, up_node, up_kind, up_child, up_ref, stride, node_rec, &k, cull, sel, &ns, sq, &nq, stats);
    for (int64_t q = 0; q < nq; ++q)
        descend(spt_root[sq[q].j], sq[q].x, left, right, lo_raw_node, row_of_node, sel, &ns);
    qsort(sel, (size_t)ns, sizeof(int64_t), cmp_i64);
    *n_sel = ns;
    free(sq);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Spherical harmonics: real, orthonormal, no Condon-Shortley phase.           */
/* Y_lm = N_lm * (d^|m|/dz^|m| P_l)(z) * {Re (x+iy)^m  (m>0); 1 (m=0);         */
/*        Im (x+iy)^|m| (m<0)},  N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)  */
/*        times sqrt(2) for m != 0.  Index k = l^2 - 1 + (m + l), l >= 1.      */
/* Also returns dY/d(x,y,z) of this polynomial form.                           */
/* ------------------------------------------------------------------------- */
static double factorial(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }
static double binom(int n, int k) { return factorial(n) / (factorial(k) * factorial(n - k)); }

/* value of d^m/dz^m P_l at z, P_l = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) z^(l-2k) */
static double legendre_deriv(int l, int m, double z) {
    double acc = 0.0;
    for (int k = 0; 2 * k <= l; ++k) {
        int p = l - 2 * k;
        if (p < m) continue;
        double c = ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l);
        double fall = 1.0;
        for (int i = 0; i < m; ++i) fall *= (double)(p - i);
        acc += c * fall * pow(z, p - m);
    }
    return acc / pow(2.0, l);
}

void or_sh_eval(int degree, const double v[3], double *Y, double *dY /* 3 per coeff, may be NULL */) {
    const double x = v[0], y = v[1], z = v[2];
    for (int l = 1; l <= degree; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            int k = l * l - 1 + (m + l);
            double N = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            if (m != 0) N *= sqrt(2.0);
            /* (x + i y)^am and (x + i y)^(am-1) */
            double re = 1.0, im = 0.0, re1 = 1.0, im1 = 0.0;
            for (int i = 0; i < am; ++i) {
                re1 = re; im1 = im;
                double nr = re * x - im * y, ni = re * y + im * x;
                re = nr; im = ni;
            }
            double ang = (m > 0) ? re : (m < 0 ? im : 1.0);
            double D = legendre_deriv(l, am, z);
            Y[k] = N * D * ang;
            if (dY) {
                double dD = (am + 1 <= l) ? legendre_deriv(l, am + 1, z) : 0.0;
                double dax, day;
                if (m > 0) { dax = am * re1; day = -am * im1; }
                else if (m < 0) { dax = am * im1; day = am * re1; }
                else { dax = 0.0; day = 0.0; }
                dY[3 * k + 0] = N * D * dax;
                dY[3 * k + 1] = N * D * day;
                dY[3 * k + 2] = N * dD * ang;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Projection (EWA splatting, Sec. 3 / Eq. 2).  float32 decision chain (D7)   */
/* plus float64 values.                                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    int visible;
    int rect[4];          /* x0, y0, x1, y1 tile rectangle, exclusive max */
    uint32_t depth_key;
    float u, v, A, B, C;  /* float32 mean and conic (support test) */
    float rx, ry;         /* float32 support half extents (block test D10) */
} proj32_t;

/* Support half extents (D10).  For the 2D covariance (a, b; b, c) the ellipse
 * d^T Sigma^-1 d <= 2L reaches |dx| <= sqrt(2L a), |dy| <= sqrt(2L c).  The
 * support test D8 is p >= -4.5, i.e. L = 4.5; L is raised to 4.51 plus 1e-5
 * times kap = (a + c)^2 / det, an upper bound of the covariance's condition
 * number, which covers the float32 rounding of the conic and of p (both grow
 * with the conditioning).  Above kap = 1e5 the extents are infinite (no block
 * is skipped). */
void or_support_extents(float a, float c, float det, float *rx, float *ry) {
    float tr = a + c;
    float kap = (tr * tr) / det;
    *rx = INFINITY;
    *ry = INFINITY;
    if (kap <= 1e5f) {
        float l2 = 9.02f + 2e-5f * kap;
        *rx = sqrtf(l2 * a);
        *ry = sqrtf(l2 * c);
    }
}

static void project_fp32(const cam_t *k, const float *r, proj32_t *o) {
    memset(o, 0, sizeof(*o));
    float t[3], dist;
    cam_view(k, r + REC_MU, t, &dist);
    float tx = t[0], ty = t[1], tz = t[2];
    if (!(tz > k->znear)) return;
    float w = r[REC_Q], x = r[REC_Q + 1], y = r[REC_Q + 2], z = r[REC_Q + 3];
    float qn = sqrtf(((w * w + x * x) + y * y) + z * z);
    w = w / qn; x = x / qn; y = y / qn; z = z / qn;
    float R[3][3];
    R[0][0] = 1.0f - 2.0f * (y * y + z * z);
    R[0][1] = 2.0f * (x * y - w * z);
    R[0][2] = 2.0f * (x * z + w * y);
    R[1][0] = 2.0f * (x * y + w * z);
    R[1][1] = 1.0f - 2.0f * (x * x + z * z);
    R[1][2] = 2.0f * (y * z - w * x);
    R[2][0] = 2.0f * (x * z - w * y);
    R[2][1] = 2.0f * (y * z + w * x);
    R[2][2] = 1.0f - 2.0f * (x * x + y * y);
    float M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * r[REC_S + j];
    float S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i][j] = (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2];
    float txc = fminf(k->limx, fmaxf(-k->limx, tx / tz)) * tz;
    float tyc = fminf(k->limy, fmaxf(-k->limy, ty / tz)) * tz;
    float J00 = k->fx / tz, J02 = -(k->fx * txc) / (tz * tz);
    float J11 = k->fy / tz, J12 = -(k->fy * tyc) / (tz * tz);
    float T[2][3];
    for (int b = 0; b < 3; ++b) {
        T[0][b] = J00 * k->R[0][b] + J02 * k->R[2][b];
        T[1][b] = J11 * k->R[1][b] + J12 * k->R[2][b];
    }
    float U[2][3];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) U[a][b] = (T[a][0] * S[0][b] + T[a][1] * S[1][b]) + T[a][2] * S[2][b];
    float s00 = (U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2];
    float s01 = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2];
    float s11 = (U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2];
    float a = s00 + 0.3f, b = s01, c = s11 + 0.3f;
    float det = a * c - b * b;
    if (!(det > 0.0f)) return;
    o->A = c / det; o->B = -b / det; o->C = a / det;
    float mid = 0.5f * (a + c);
    float disc = sqrtf(fmaxf(0.1f, mid * mid - det));
    float lam = mid + disc;
    float rad = ceilf(3.0f * sqrtf(lam));
    float u = (k->fx * tx) / tz + k->cx;
    float v = (k->fy * ty) / tz + k->cy;
    if (!isfinite(u) || !isfinite(v) || !isfinite(rad)) return;
    float fx0 = fminf(fmaxf(floorf((u - rad) * 0.0625f), 0.0f), (float)k->TX);
    float fx1 = fminf(fmaxf(floorf((u + rad) * 0.0625f) + 1.0f, 0.0f), (float)k->TX);
    float fy0 = fminf(fmaxf(floorf((v - rad) * 0.0625f), 0.0f), (float)k->TY);
    float fy1 = fminf(fmaxf(floorf((v + rad) * 0.0625f) + 1.0f, 0.0f), (float)k->TY);
    o->rect[0] = (int)fx0; o->rect[1] = (int)fy0; o->rect[2] = (int)fx1; o->rect[3] = (int)fy1;
    if ((o->rect[2] - o->rect[0]) * (o->rect[3] - o->rect[1]) <= 0) return;
    o->u = u; o->v = v;
    or_support_extents(a, c, det, &o->rx, &o->ry);
    uint32_t bits;
    memcpy(&bits, &tz, 4);
    o->depth_key = bits;
    o->visible = 1;
}

/* float64 forward values of one Gaussian (any camera-visible record). */
typedef struct {
    double u, v, A, B, C, opacity, rgb[3], raw_rgb[3], depth;
} proj64_t;

static void project_fp64(const cam_t *k, int degree, const float *r, proj64_t *o) {
    double d[3], t[3];
    for (int a = 0; a < 3; ++a) d[a] = (double)r[REC_MU + a] - (double)k->pos[a];
    for (int a = 0; a < 3; ++a) t[a] = k->R[a][0] * d[0] + k->R[a][1] * d[1] + k->R[a][2] * d[2];
    double q[4];
    for (int a = 0; a < 4; ++a) q[a] = r[REC_Q + a];
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; ++a) q[a] /= qn;
    double R[3][3], S[3][3];
    quat_to_rot_d(q, R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            S[i][j] = 0.0;
            for (int m = 0; m < 3; ++m) S[i][j] += R[i][m] * r[REC_S + m] * r[REC_S + m] * R[j][m];
        }
    double tz = t[2];
    double limx = k->limx, limy = k->limy;
    double txtz = t[0] / tz, tytz = t[1] / tz;
    double txc = (txtz < -limx ? -limx : (txtz > limx ? limx : txtz)) * tz;
    double tyc = (tytz < -limy ? -limy : (tytz > limy ? limy : tytz)) * tz;
    double J[2][3] = {{k->fx / tz, 0.0, -k->fx * txc / (tz * tz)}, {0.0, k->fy / tz, -k->fy * tyc / (tz * tz)}};
    double T[2][3];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) {
            T[a][b] = 0.0;
            for (int m = 0; m < 3; ++m) T[a][b] += J[a][m] * k->R[m][b];
        }
    double S2[2][2];
    for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
            S2[a][c] = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) S2[a][c] += T[a][i] * S[i][j] * T[c][j];
        }
    double a = S2[0][0] + DILATION, b = S2[0][1], c = S2[1][1] + DILATION;
    double det = a * c - b * b;
    o->A = c / det; o->B = -b / det; o->C = a / det;
    o->u = k->fx * t[0] / tz + k->cx;
    o->v = k->fy * t[1] / tz + k->cy;
    o->depth = tz;
    o->opacity = r[REC_OP];
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double dir[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
    int K = sh_count(degree);
    double Y[64];
    if (K > 0) or_sh_eval(degree, dir, Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double c0 = r[REC_B + ch];
        for (int kk = 0; kk < K; ++kk) c0 += Y[kk] * r[REC_F + 3 * kk + ch];
        o->raw_rgb[ch] = c0;
        o->rgb[ch] = c0 > 0.0 ? c0 : 0.0;
    }
}

/* Per selected Gaussian i (rows sel[i] of row_rec): decisions (float32) and
 * values (float64).  vis/rect/key/u32.. are outputs of length n, rect 4n,
 * f32 7n (u, v, A, B, C, rx, ry), f64 12n (u, v, A, B, C, opacity, rgb[3], depth, -, -). */
int or_project(int64_t n, const int64_t *sel, int stride, int degree, const float *row_rec, const float *cam,
               int32_t *vis, int32_t *rect, uint32_t *key, float *f32, double *f64) {
    cam_t k;
    cam_setup(cam, &k);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        const float *r = row_rec + sel[i] * stride;
        proj32_t p;
        project_fp32(&k, r, &p);
        vis[i] = p.visible;
        for (int a = 0; a < 4; ++a) rect[4 * i + a] = p.rect[a];
        key[i] = p.depth_key;
        float *o32 = f32 + F32_N * i;
        o32[0] = p.u; o32[1] = p.v; o32[2] = p.A; o32[3] = p.B; o32[4] = p.C; o32[5] = p.rx; o32[6] = p.ry;
        double *o = f64 + 12 * i;
        memset(o, 0, sizeof(double) * 12);
        if (p.visible) {
            proj64_t q;
            project_fp64(&k, degree, r, &q);
            o[0] = q.u; o[1] = q.v; o[2] = q.A; o[3] = q.B; o[4] = q.C; o[5] = q.opacity;
            o[6] = q.rgb[0]; o[7] = q.rgb[1]; o[8] = q.rgb[2]; o[9] = q.depth;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Tile x depth ordering: pairs (tile, depth key, i) sorted ascending (the      */
/* 3DGS sort reused by the paper).  tile_start has n_tiles + 1 entries.        */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t tile; uint32_t key; int64_t i; } pair_t;
static int cmp_pair(const void *a, const void *b) {
    const pair_t *x = a, *y = b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->i > y->i) - (x->i < y->i);
}

/* Tile support test D9 (float32, evaluated as written).  The support exponent
 * p(x, y) = -1/2 (A dx^2 + 2 B dx dy + C dy^2), dx = u - x, dy = v - y, is a
 * concave quadratic; its maximum over the rectangle spanned by the tile's pixel
 * centres is 0 if (u, v) lies inside, else it lies on an edge, where it is the
 * 1-D maximum clamped to the edge.  The pair is kept iff that maximum is at
 * least -4.5 - 0.01; the margin makes the test conservative against rounding,
 * so a dropped pair never had a pixel passing D8 and the image is unchanged. */
static float edge_p(float A, float B, float C, float dx, float dy) {
    return -0.5f * (A * dx * dx + C * dy * dy) - B * dx * dy;
}

int or_tile_keep(float u, float v, float A, float B, float C, int tx, int ty) {
    float X0 = (float)(TILE * tx) + 0.5f, X1 = X0 + 15.0f;
    float Y0 = (float)(TILE * ty) + 0.5f, Y1 = Y0 + 15.0f;
    if (u >= X0 && u <= X1 && v >= Y0 && v <= Y1) return 1;
    float best = -INFINITY;
    float xs[2] = {X0, X1}, ys[2] = {Y0, Y1};
    for (int k = 0; k < 2; ++k) {
        float dx = u - xs[k];                       /* vertical edge x = xs[k] */
        float y = fminf(fmaxf(v + (B * dx) / C, Y0), Y1);
        best = fmaxf(best, edge_p(A, B, C, dx, v - y));
        float dy = v - ys[k];                       /* horizontal edge y = ys[k] */
        float x = fminf(fmaxf(u + (B * dy) / A, X0), X1);
        best = fmaxf(best, edge_p(A, B, C, u - x, dy));
    }
    return best >= -4.51f;
}

int or_sort_pairs(int64_t n, const int32_t *vis, const int32_t *rect, const uint32_t *key, const float *f32,
                  int TX, int TY, int64_t cap, int64_t *n_pairs, int64_t *pair_i, int64_t *tile_start) {
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i)
        if (vis[i]) np += (int64_t)(rect[4 * i + 2] - rect[4 * i]) * (rect[4 * i + 3] - rect[4 * i + 1]);
    if (np > cap) { *n_pairs = np; return -1; }
    pair_t *p = malloc(sizeof(pair_t) * (size_t)(np + 1));
    int64_t w = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!vis[i]) continue;
        const float *g = f32 + F32_N * i;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {
                if (!or_tile_keep(g[0], g[1], g[2], g[3], g[4], tx, ty)) continue;
                p[w].tile = (int64_t)ty * TX + tx; p[w].key = key[i]; p[w].i = i; ++w;
            }
    }
    np = w;
    *n_pairs = np;
    qsort(p, (size_t)np, sizeof(pair_t), cmp_pair);
    int64_t nt = (int64_t)TX * TY;
    for (int64_t t = 0; t <= nt; ++t) tile_start[t] = 0;
    for (int64_t e = 0; e < np; ++e) { pair_i[e] = p[e].i; tile_start[p[e].tile + 1]++; }
    for (int64_t t = 0; t < nt; ++t) tile_start[t + 1] += tile_start[t];
    free(p);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Blend (Eq. 1 and Eq. 2): front-to-back per pixel over its tile's list.      */
/* Support test D8 in float32; alpha = min(0.99, sigma exp(p)) in float64.    */
/* Eq. 1 is truncated once the transmittance falls below 1e-4: the Gaussian   */
/* that takes T below the bound is still blended and the pixel stops after    */
/* it, so the neglected tail is at most 1e-4 times the largest colour.        */
/* ------------------------------------------------------------------------- */
/* Block support test D10 (float32, evaluated as written): the predicate the
 * CUDA blend uses to skip a Gaussian for a whole 8x8 pixel block, kept here
 * for the brute-force check that it is conservative; or_blend and
 * or_blend_backward below do not call it.  The image is cut into 8x8 pixel
 * blocks (four per tile); block (bx0, by0) has pixel centres bx0 + 0.5 ..
 * bx0 + 7.5 (same in y), centre bx0 + 4 and half span 3.5.  Gaussian g (u, v,
 * rx, ry = g[0], g[1], g[5], g[6]) is kept for the block iff its support box
 * |u - x| <= rx, |v - y| <= ry can reach a centre of the block. */
int or_block_keep(const float *g, int px, int py) {
    float wcx = (float)(px & ~7) + 4.0f, wcy = (float)(py & ~7) + 4.0f;
    return !(fabsf(g[0] - wcx) > g[5] + 3.5f || fabsf(g[1] - wcy) > g[6] + 3.5f);
}

static inline float support_p(float u, float v, float A, float B, float C, int px, int py) {
    float dx = u - ((float)px + 0.5f), dy = v - ((float)py + 0.5f);
    float nha = -0.5f * A, nhc = -0.5f * C, nb = -B;
    return fmaf(nb * dx, dy, fmaf(nhc * dy, dy, (nha * dx) * dx));
}

/* win (x0, y0, x1, y1) restricts the work to a pixel window (NULL: all). */
int or_blend(int W, int H, const double *bg, const int64_t *tile_start, const int64_t *pair_i,
             const float *f32, const double *f64, double *image, int32_t *n_contrib, double *T_final,
             const int32_t *win) {
    int TX = (W + TILE - 1) / TILE;
    int wx0 = win ? win[0] : 0, wy0 = win ? win[1] : 0, wx1 = win ? win[2] : W, wy1 = win ? win[3] : H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int py = wy0; py < wy1; ++py)
        for (int px = wx0; px < wx1; ++px) {
            int64_t t = (int64_t)(py / TILE) * TX + px / TILE;
            double T = 1.0, C[3] = {0, 0, 0};
            int32_t last = 0;
            for (int64_t e = tile_start[t]; e < tile_start[t + 1]; ++e) {
                int64_t i = pair_i[e];
                const float *g = f32 + F32_N * i;
                if (support_p(g[0], g[1], g[2], g[3], g[4], px, py) < SUPPORT_P) continue;
                const double *q = f64 + 12 * i;
                double dx = q[0] - (px + 0.5), dy = q[1] - (py + 0.5);
                double p = -0.5 * (q[2] * dx * dx + q[4] * dy * dy) - q[3] * dx * dy;
                double alpha = q[5] * exp(p);
                if (alpha > ALPHA_MAX) alpha = ALPHA_MAX;
                for (int ch = 0; ch < 3; ++ch) C[ch] += q[6 + ch] * alpha * T;
                T = T * (1.0 - alpha);
                last = (int32_t)(e - tile_start[t] + 1);
                if (T < T_MIN) break;
            }
            double *o = image + 3 * ((int64_t)py * W + px);
            for (int ch = 0; ch < 3; ++ch) o[ch] = C[ch] + T * bg[ch];
            if (n_contrib) n_contrib[(int64_t)py * W + px] = last;
            if (T_final) T_final[(int64_t)py * W + px] = T;
        }
    return 0;
}

/* g += v (an atomic add in the OpenMP build, where pixel rows run in parallel) */
static inline void accum(double *g, double v) {
#pragma omp atomic
    *g += v;
}

/* Backward of the blend: exact derivative of or_blend with the decisions held
 * fixed.  For each pixel, with T_i the transmittance in front of Gaussian i and
 * R_i the colour composited behind it (background included):
 *   dC/dc_i = alpha_i T_i,  dC/dalpha_i = c_i T_i - R_i / (1 - alpha_i).
 * Outputs per selected Gaussian: g2d[9i..] = dL/d(u, v, A, B, C, opacity, r, g, b). */
int or_blend_backward(int W, int H, const double *bg, const int64_t *tile_start, const int64_t *pair_i,
                      const float *f32, const double *f64, const double *dL_dimg, int64_t n, double *g2d,
                      const int32_t *win) {
    int wx0 = win ? win[0] : 0, wy0 = win ? win[1] : 0, wx1 = win ? win[2] : W, wy1 = win ? win[3] : H;
    int TX = (W + TILE - 1) / TILE;
    memset(g2d, 0, sizeof(double) * 9 * (size_t)n);
    int64_t maxlen = 0;
    for (int64_t t = 0; t < (int64_t)TX * ((H + TILE - 1) / TILE); ++t)
        if (tile_start[t + 1] - tile_start[t] > maxlen) maxlen = tile_start[t + 1] - tile_start[t];
#pragma omp parallel
    {
    int64_t *li = malloc(sizeof(int64_t) * (size_t)(maxlen + 1));
    double *la = malloc(sizeof(double) * (size_t)(maxlen + 1)), *lT = malloc(sizeof(double) * (size_t)(maxlen + 1));
    double *lp = malloc(sizeof(double) * (size_t)(maxlen + 1)), *lg = malloc(sizeof(double) * (size_t)(maxlen + 1));
    int *lclamp = malloc(sizeof(int) * (size_t)(maxlen + 1));
#pragma omp for schedule(dynamic, 1)
    for (int py = wy0; py < wy1; ++py)
        for (int px = wx0; px < wx1; ++px) {
            int64_t t = (int64_t)(py / TILE) * TX + px / TILE;
            double T = 1.0;
            int64_t cnt = 0;
            for (int64_t e = tile_start[t]; e < tile_start[t + 1]; ++e) {
                int64_t i = pair_i[e];
                const float *g = f32 + F32_N * i;
                if (support_p(g[0], g[1], g[2], g[3], g[4], px, py) < SUPPORT_P) continue;
                const double *q = f64 + 12 * i;
                double dx = q[0] - (px + 0.5), dy = q[1] - (py + 0.5);
                double p = -0.5 * (q[2] * dx * dx + q[4] * dy * dy) - q[3] * dx * dy;
                double G = exp(p), alpha = q[5] * G;
                int clamped = 0;
                if (alpha > ALPHA_MAX) { alpha = ALPHA_MAX; clamped = 1; }
                li[cnt] = i; la[cnt] = alpha; lT[cnt] = T; lp[cnt] = p; lg[cnt] = G; lclamp[cnt] = clamped; ++cnt;
                T = T * (1.0 - alpha);
                if (T < T_MIN) break;
            }
            const double *dC = dL_dimg + 3 * ((int64_t)py * W + px);
            double Rb[3] = {T * bg[0], T * bg[1], T * bg[2]};       /* colour behind, from the back */
            for (int64_t m = cnt - 1; m >= 0; --m) {
                int64_t i = li[m];
                const double *q = f64 + 12 * i;
                double alpha = la[m], Ti = lT[m];
                double dL_dalpha = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    accum(&g2d[9 * i + 6 + ch], dC[ch] * alpha * Ti);
                    dL_dalpha += dC[ch] * (q[6 + ch] * Ti - Rb[ch] / (1.0 - alpha));
                }
                for (int ch = 0; ch < 3; ++ch) Rb[ch] += q[6 + ch] * alpha * Ti;
                if (lclamp[m]) continue;
                double dx = q[0] - (px + 0.5), dy = q[1] - (py + 0.5);
                double dL_dp = dL_dalpha * alpha;
                accum(&g2d[9 * i + 5], dL_dalpha * lg[m]);
                accum(&g2d[9 * i + 0], dL_dp * (-(q[2] * dx + q[3] * dy)));
                accum(&g2d[9 * i + 1], dL_dp * (-(q[4] * dy + q[3] * dx)));
                accum(&g2d[9 * i + 2], dL_dp * (-0.5 * dx * dx));
                accum(&g2d[9 * i + 3], dL_dp * (-dx * dy));
                accum(&g2d[9 * i + 4], dL_dp * (-0.5 * dy * dy));
            }
        }
    free(li); free(la); free(lT); free(lp); free(lg); free(lclamp);
    }
    return 0;
}

/* Backward of the projection and colour: dL/d(record) for each selected
 * Gaussian from its 2D gradients (exact derivative of project_fp64). */
int or_project_backward(int64_t n, const int64_t *sel, int stride, int degree, const float *row_rec,
                        const float *cam, const int32_t *vis, const double *g2d, double *g_rec) {
    cam_t k;
    cam_setup(cam, &k);
    memset(g_rec, 0, sizeof(double) * (size_t)(n * stride));
    int K = sh_count(degree);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        if (!vis[i]) continue;
        const float *r = row_rec + sel[i] * stride;
        const double *g = g2d + 9 * i;
        double *o = g_rec + i * stride;
        /* ---- forward recomputation ---- */
        double d[3], t[3];
        for (int a = 0; a < 3; ++a) d[a] = (double)r[REC_MU + a] - (double)k.pos[a];
        for (int a = 0; a < 3; ++a) t[a] = k.R[a][0] * d[0] + k.R[a][1] * d[1] + k.R[a][2] * d[2];
        double q[4];
        for (int a = 0; a < 4; ++a) q[a] = r[REC_Q + a];
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qh[4];
        for (int a = 0; a < 4; ++a) qh[a] = q[a] / qn;
        double R[3][3], s[3], M[3][3], S[3][3];
        quat_to_rot_d(qh, R);
        for (int a = 0; a < 3; ++a) s[a] = r[REC_S + a];
        for (int i2 = 0; i2 < 3; ++i2)
            for (int j = 0; j < 3; ++j) M[i2][j] = R[i2][j] * s[j];
        for (int i2 = 0; i2 < 3; ++i2)
            for (int j = 0; j < 3; ++j) S[i2][j] = M[i2][0] * M[j][0] + M[i2][1] * M[j][1] + M[i2][2] * M[j][2];
        double tz = t[2], tx = t[0], ty = t[1];
        double limx = k.limx, limy = k.limy;
        double txtz = tx / tz, tytz = ty / tz;
        int clx = (txtz < -limx || txtz > limx), cly = (tytz < -limy || tytz > limy);
        double sx = txtz < 0 ? -1.0 : 1.0, sy = tytz < 0 ? -1.0 : 1.0;
        double txc = clx ? sx * limx * tz : tx, tyc = cly ? sy * limy * tz : ty;
        double J[2][3] = {{k.fx / tz, 0.0, -k.fx * txc / (tz * tz)}, {0.0, k.fy / tz, -k.fy * tyc / (tz * tz)}};
        double T[2][3];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                T[a][b] = 0.0;
                for (int m = 0; m < 3; ++m) T[a][b] += J[a][m] * k.R[m][b];
            }
        double S2[2][2];
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 2; ++c) {
                S2[a][c] = 0.0;
                for (int i2 = 0; i2 < 3; ++i2)
                    for (int j = 0; j < 3; ++j) S2[a][c] += T[a][i2] * S[i2][j] * T[c][j];
            }
        double a_ = S2[0][0] + DILATION, b_ = S2[0][1], c_ = S2[1][1] + DILATION;
        double det = a_ * c_ - b_ * b_;
        double Qm[2][2] = {{c_ / det, -b_ / det}, {-b_ / det, a_ / det}};
        /* ---- colour ---- */
        double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dir[3] = {d[0] / dn, d[1] / dn, d[2] / dn};
        double Y[64], dY[192];
        if (K > 0) or_sh_eval(degree, dir, Y, dY);
        double gdir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            double raw = r[REC_B + ch];
            for (int kk = 0; kk < K; ++kk) raw += Y[kk] * r[REC_F + 3 * kk + ch];
            if (raw < 0.0) continue;
            double gc = g[6 + ch];
            o[REC_B + ch] = gc;
            for (int kk = 0; kk < K; ++kk) {
                o[REC_F + 3 * kk + ch] = gc * Y[kk];
                double f = r[REC_F + 3 * kk + ch];
                for (int a = 0; a < 3; ++a) gdir[a] += gc * f * dY[3 * kk + a];
            }
        }
        double gd[3];
        double dot = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
        for (int a = 0; a < 3; ++a) gd[a] = (gdir[a] - dir[a] * dot) / dn;
        /* ---- opacity ---- */
        o[REC_OP] = g[5];
        /* ---- conic -> 2D covariance ---- */
        double gQ[2][2] = {{g[2], 0.5 * g[3]}, {0.5 * g[3], g[4]}};
        double tmp[2][2], gS2[2][2];
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 2; ++c) tmp[a][c] = Qm[a][0] * gQ[0][c] + Qm[a][1] * gQ[1][c];
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 2; ++c) gS2[a][c] = -(tmp[a][0] * Qm[0][c] + tmp[a][1] * Qm[1][c]);
        /* S2 = T S T^T: gS = T^T gS2 T ; gT = 2 gS2 T S */
        double gS[3][3], gT[2][3];
        for (int i2 = 0; i2 < 3; ++i2)
            for (int j = 0; j < 3; ++j) {
                gS[i2][j] = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int c = 0; c < 2; ++c) gS[i2][j] += T[a][i2] * gS2[a][c] * T[c][j];
            }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                gT[a][b] = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int m = 0; m < 3; ++m) gT[a][b] += 2.0 * gS2[a][c] * T[c][m] * S[m][b];
            }
        /* T = J W: gJ = gT W^T */
        double gJ[2][3];
        for (int a = 0; a < 2; ++a)
            for (int m = 0; m < 3; ++m) {
                gJ[a][m] = 0.0;
                for (int b = 0; b < 3; ++b) gJ[a][m] += gT[a][b] * k.R[m][b];
            }
        double gt[3] = {0, 0, 0};
        gt[2] += -k.fx / (tz * tz) * gJ[0][0] - k.fy / (tz * tz) * gJ[1][1];
        if (!clx) { gt[0] += -k.fx / (tz * tz) * gJ[0][2]; gt[2] += 2.0 * k.fx * tx / (tz * tz * tz) * gJ[0][2]; }
        else gt[2] += k.fx * txc / (tz * tz * tz) * gJ[0][2];
        if (!cly) { gt[1] += -k.fy / (tz * tz) * gJ[1][2]; gt[2] += 2.0 * k.fy * ty / (tz * tz * tz) * gJ[1][2]; }
        else gt[2] += k.fy * tyc / (tz * tz * tz) * gJ[1][2];
        /* mean in pixels */
        gt[0] += k.fx / tz * g[0];
        gt[2] += -k.fx * tx / (tz * tz) * g[0];
        gt[1] += k.fy / tz * g[1];
        gt[2] += -k.fy * ty / (tz * tz) * g[1];
        for (int a = 0; a < 3; ++a)
            o[REC_MU + a] = gd[a] + k.R[0][a] * gt[0] + k.R[1][a] * gt[1] + k.R[2][a] * gt[2];
        /* Sigma = M M^T, M = R diag(s) */
        double gM[3][3];
        for (int i2 = 0; i2 < 3; ++i2)
            for (int j = 0; j < 3; ++j) gM[i2][j] = 2.0 * (gS[i2][0] * M[0][j] + gS[i2][1] * M[1][j] + gS[i2][2] * M[2][j]);
        double gR[3][3];
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int i2 = 0; i2 < 3; ++i2) { acc += gM[i2][j] * R[i2][j]; gR[i2][j] = gM[i2][j] * s[j]; }
            o[REC_S + j] = acc;
        }
        double w = qh[0], x = qh[1], y = qh[2], z = qh[3];
        double gq[4];
        gq[0] = 2.0 * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
        gq[1] = 2.0 * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - w * gR[1][2] + z * gR[2][0] + w * gR[2][1])
              - 4.0 * x * (gR[1][1] + gR[2][2]);
        gq[2] = 2.0 * (x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] - w * gR[2][0] + z * gR[2][1])
              - 4.0 * y * (gR[0][0] + gR[2][2]);
        gq[3] = 2.0 * (-w * gR[0][1] + x * gR[0][2] + w * gR[1][0] + y * gR[1][2] + x * gR[2][0] + y * gR[2][1])
              - 4.0 * z * (gR[0][0] + gR[1][1]);
        double qd = gq[0] * qh[0] + gq[1] * qh[1] + gq[2] * qh[2] + gq[3] * qh[3];
        for (int a = 0; a < 4; ++a) o[REC_Q + a] = (gq[a] - qh[a] * qd) / qn;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Sparse Adam over the cut (appendix "Implementation Details": only the      */
/* nodes of the cut set are optimised; Adam after Kingma and Ba).  For every  */
/* listed row r with gradient row g (its first `used` columns) and per-column */
/* learning rates lr[c]:                                                       */
/*   t_r <- t_r + 1                                                            */
/*   m <- b1 m + (1 - b1) g ;  v <- b2 v + (1 - b2) g^2                        */
/*   p <- p - lr_c (m / (1 - b1^t_r)) / (sqrt(v / (1 - b2^t_r)) + eps)        */
/* Each row counts its own steps, so its bias correction covers the steps it  */
/* took part in.  Rows not listed are untouched.  float64 throughout.         */
/* ------------------------------------------------------------------------- */
int or_adam_sparse(int64_t n_rows, const int64_t *rows, const double *grads, int stride, int used,
                   const double *lr, double b1, double b2, double eps, double *params, double *m, double *v,
                   uint32_t *t) {
    for (int64_t i = 0; i < n_rows; ++i) {
        const int64_t r = rows[i];
        t[r] += 1;
        const double bc1 = 1.0 - pow(b1, (double)t[r]), bc2 = 1.0 - pow(b2, (double)t[r]);
        for (int c = 0; c < used; ++c) {
            const double g = grads[i * stride + c];
            double *mm = m + r * stride + c, *vv = v + r * stride + c;
            *mm = b1 * *mm + (1.0 - b1) * g;
            *vv = b2 * *vv + (1.0 - b2) * g * g;
            params[r * stride + c] -= lr[c] * (*mm / bc1) / (sqrt(*vv / bc2) + eps);
        }
    }
    return 0;
}
