// Densification planning on the device (Sec. 3 "Densification"; appendix
// "Respawning, Densifying, and Pruning Gaussians").
//
// The rows of the scene are classified in parallel:
//   dead       a leaf with a parent whose opacity is below min_opacity, or
//              flagged stale (the pruning rule zeroes the opacity of Gaussians
//              that have not contributed for a while), except the left child
//              of a node whose two children are both dead (only the right one
//              is respawned; the left one waits for a later densification);
//   candidate  a leaf that is neither transparent nor stale and whose maximal
//              screen-space gradient reaches the threshold (the selection of
//              hierarchical 3DGS).
// Dead rows are compacted in ascending order; candidate rows are sorted by
// gradient, largest first, ties by row (a stable radix sort of the descending
// key over rows in ascending order).  The host pairs the i-th dead row with the
// i-th candidate (respawn) and lets the remaining candidates spawn while the
// node budget allows: the operations lodgs_scene_densify applies.
#include <algorithm>
#include <vector>

#include "lodgs_internal.cuh"

using namespace lodgs;

namespace {

constexpr int DB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + DB - 1) / DB); }

__global__ void k_parents(const int32_t *__restrict__ left, const int32_t *__restrict__ right, int64_t M,
                          int32_t *__restrict__ parent, uint8_t *__restrict__ is_left) {
    const int64_t u = blockIdx.x * (int64_t)DB + threadIdx.x;
    if (u >= M || left[u] < 0) return;
    parent[left[u]] = (int32_t)u;
    parent[right[u]] = (int32_t)u;
    is_left[left[u]] = 1;
}

__global__ void k_rows_of_nodes(const int32_t *__restrict__ node_of_row, int64_t M, int32_t *__restrict__ row_of) {
    const int64_t r = blockIdx.x * (int64_t)DB + threadIdx.x;
    if (r < M) row_of[node_of_row[r]] = (int32_t)r;
}

// per row: 1 a transparent or stale leaf, 3 one that has a parent (dead before the sibling rule), else 0
__global__ void k_low(const float *__restrict__ rows, int stride, const int32_t *__restrict__ node_of_row,
                      const int32_t *__restrict__ left, const int32_t *__restrict__ parent,
                      const uint8_t *__restrict__ stale, float min_opacity, int64_t M, uint8_t *__restrict__ low) {
    const int64_t r = blockIdx.x * (int64_t)DB + threadIdx.x;
    if (r >= M) return;
    const int32_t u = node_of_row[r];
    const bool leaf = left[u] < 0;
    const bool lw = leaf && (rows[r * stride + REC_OP] < min_opacity || (stale && stale[r]));
    low[r] = (uint8_t)(lw ? (parent[u] >= 0 ? 3 : 1) : 0);
}

// Order-preserving key of a float: ascending keys give ascending floats.
__device__ __forceinline__ uint32_t float_key(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_flags(const float *__restrict__ grad, const int32_t *__restrict__ node_of_row,
                        const int32_t *__restrict__ left, const int32_t *__restrict__ right,
                        const int32_t *__restrict__ parent, const uint8_t *__restrict__ is_left,
                        const int32_t *__restrict__ row_of, const uint8_t *__restrict__ low, float threshold,
                        int64_t M, uint32_t *__restrict__ dead, uint32_t *__restrict__ cand) {
    const int64_t r = blockIdx.x * (int64_t)DB + threadIdx.x;
    if (r >= M) return;
    const int32_t u = node_of_row[r];
    bool d = low[r] == 3;
    if (d && is_left[u]) {                       // both children dead: only the right one respawns
        const int32_t sib = right[parent[u]];
        d = low[row_of[sib]] != 3;
    }
    dead[r] = d ? 1u : 0u;
    cand[r] = (left[u] < 0 && low[r] == 0 && grad[r] >= threshold) ? 1u : 0u;
}

__global__ void k_compact(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos, int64_t M,
                          const float *__restrict__ grad, uint32_t *__restrict__ rows_out,
                          uint32_t *__restrict__ keys_out) {
    const int64_t r = blockIdx.x * (int64_t)DB + threadIdx.x;
    if (r >= M || !flag[r]) return;
    rows_out[pos[r]] = (uint32_t)r;
    if (keys_out) keys_out[pos[r]] = ~float_key(grad[r] + 0.0f);  // largest first; -0 and +0 tie
}

// scratch released at scope exit (the call synchronises its stream first)
struct Scratch {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() {
        cudaStreamSynchronize(st);
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T> cudaError_t get(T **p, size_t n) {
        cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

}  // namespace

extern "C" int lodgs_densify_plan(lodgs_scene *sc, const float *rows, const float *grad_max, const uint8_t *stale,
                                  float grad_threshold, float min_opacity, int64_t max_nodes, lodgs_densify_op *ops,
                                  int64_t capacity, int64_t *n_ops, int64_t *n_spawn, void *stream) {
    if (!sc || !grad_max || !n_ops || !n_spawn || capacity < 0 || (capacity > 0 && !ops)) {
        set_error("densify_plan: NULL argument or negative capacity");
        return LODGS_E_INVALID;
    }
    if (!rows) rows = sc->d_rows;
    if (!rows) {
        set_error("densify_plan: the scene's records are not on the device; pass the records");
        return LODGS_E_INVALID;
    }
    const int64_t M = sc->n_nodes;
    cudaStream_t st = (cudaStream_t)stream;
    Scratch s(st);
    int32_t *parent, *row_of;
    uint8_t *is_left, *low;
    uint32_t *dead, *cand, *pos_d, *pos_c, *tot, *d_m, *bsum, *rows_d, *rows_c, *keys, *keys_alt, *vals_alt, *hist;
    LODGS_CUDA(s.get(&parent, M)); LODGS_CUDA(s.get(&row_of, M)); LODGS_CUDA(s.get(&is_left, M));
    LODGS_CUDA(s.get(&low, M)); LODGS_CUDA(s.get(&dead, M)); LODGS_CUDA(s.get(&cand, M));
    LODGS_CUDA(s.get(&pos_d, M)); LODGS_CUDA(s.get(&pos_c, M)); LODGS_CUDA(s.get(&tot, 2));
    LODGS_CUDA(s.get(&d_m, 1)); LODGS_CUDA(s.get(&bsum, 2 * SCAN_GRID_MAX)); LODGS_CUDA(s.get(&rows_d, M));
    LODGS_CUDA(s.get(&rows_c, M)); LODGS_CUDA(s.get(&keys, M)); LODGS_CUDA(s.get(&keys_alt, M));
    LODGS_CUDA(s.get(&vals_alt, M)); LODGS_CUDA(s.get(&hist, SORT_HIST));
    LODGS_CUDA(cudaMemsetAsync(parent, 0xff, M * 4, st));
    LODGS_CUDA(cudaMemsetAsync(is_left, 0, M, st));
    const uint32_t M32 = (uint32_t)M;
    LODGS_CUDA(cudaMemcpyAsync(d_m, &M32, 4, cudaMemcpyHostToDevice, st));
    k_parents<<<nblk(M), DB, 0, st>>>(sc->d_left, sc->d_right, M, parent, is_left);
    k_rows_of_nodes<<<nblk(M), DB, 0, st>>>(sc->d_node_of_row, M, row_of);
    k_low<<<nblk(M), DB, 0, st>>>(rows, sc->stride, sc->d_node_of_row, sc->d_left, parent, stale, min_opacity, M,
                                  low);
    k_flags<<<nblk(M), DB, 0, st>>>(grad_max, sc->d_node_of_row, sc->d_left, sc->d_right, parent, is_left, row_of,
                                    low, grad_threshold, M, dead, cand);
    count_launches(4);
    if (int rc = scan_exclusive(dead, pos_d, d_m, M32, bsum, tot, st)) return rc;
    if (int rc = scan_exclusive(cand, pos_c, d_m, M32, bsum + SCAN_GRID_MAX, tot + 1, st)) return rc;
    k_compact<<<nblk(M), DB, 0, st>>>(dead, pos_d, M, grad_max, rows_d, nullptr);
    k_compact<<<nblk(M), DB, 0, st>>>(cand, pos_c, M, grad_max, rows_c, keys);
    count_launches(2);
    bool alt = false;
    if (int rc = radix_sort_pairs(keys, rows_c, keys_alt, vals_alt, tot + 1, M32, 0, 32, hist, st, &alt)) return rc;
    const uint32_t *sorted_c = alt ? vals_alt : rows_c;
    uint32_t nn[2];
    LODGS_CUDA(cudaMemcpyAsync(nn, tot, 8, cudaMemcpyDeviceToHost, st));
    LODGS_CUDA(cudaStreamSynchronize(st));
    const int64_t nd = nn[0], nc = nn[1];
    std::vector<uint32_t> hd((size_t)nd), hc((size_t)nc);
    if (nd) LODGS_CUDA(cudaMemcpyAsync(hd.data(), rows_d, nd * 4, cudaMemcpyDeviceToHost, st));
    if (nc) LODGS_CUDA(cudaMemcpyAsync(hc.data(), sorted_c, nc * 4, cudaMemcpyDeviceToHost, st));
    LODGS_CUDA(cudaStreamSynchronize(st));
    const int64_t nr = std::min(nd, nc);
    int64_t ns = nc - nr;
    if (max_nodes >= 0) ns = std::min<int64_t>(ns, std::max<int64_t>(0, (max_nodes - M) / 2));
    *n_spawn = ns;
    *n_ops = ns + nr;
    if (ns + nr > capacity) {
        set_error("densify_plan: ops capacity below the planned operations (*n_ops)");
        return LODGS_E_INVALID;
    }
    for (int64_t i = 0; i < ns; ++i) ops[i] = {LODGS_DENSIFY_SPAWN, 0, (int64_t)hc[nr + i], -1};
    for (int64_t i = 0; i < nr; ++i) ops[ns + i] = {LODGS_DENSIFY_RESPAWN, 0, (int64_t)hc[i], (int64_t)hd[i]};
    return LODGS_OK;
}
