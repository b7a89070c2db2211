// Gradient of a multi-view batch loss on the union of the views' cuts.
//
// Each view's backward writes one gradient row per node of its own LoD cut;
// only cut-set nodes receive gradients (appendix "Implementation Details").  For
// a batch of views the rows of a node selected by several views must be summed.
// The selected rows of all views are concatenated, stably radix-sorted by node
// row, split into runs of equal rows (scan of run starts), and each run is
// summed by one warp in view order, so the result is deterministic and no
// atomics are needed.
#include <algorithm>
#include <vector>

#include "lodgs_internal.cuh"

using namespace lodgs;

namespace {

constexpr int BB = 256;

__global__ void k_iota(uint32_t *__restrict__ v, uint32_t base, uint32_t n) {
    uint32_t i = blockIdx.x * BB + threadIdx.x;
    if (i < n) v[i] = base + i;
}

__global__ void k_run_starts(const uint32_t *__restrict__ key, uint32_t n, uint32_t *__restrict__ flag) {
    uint32_t p = blockIdx.x * BB + threadIdx.x;
    if (p < n) flag[p] = (p == 0 || key[p] != key[p - 1]) ? 1u : 0u;
}

__global__ void k_runs(const uint32_t *__restrict__ key, const uint32_t *__restrict__ flag,
                       const uint32_t *__restrict__ pos, uint32_t n, uint32_t *__restrict__ out_rows,
                       uint32_t *__restrict__ run_start) {
    uint32_t p = blockIdx.x * BB + threadIdx.x;
    if (p >= n) return;
    if (flag[p]) {
        out_rows[pos[p]] = key[p];
        run_start[pos[p]] = p;
    }
    if (p == n - 1) run_start[pos[p] + flag[p]] = n;      // sentinel: one past the last run
}

// one warp per run: sum the rows of its entries (vals = global entry index) in order
__global__ void k_sum_runs(const uint32_t *__restrict__ run_start, const uint32_t *__restrict__ d_nruns,
                           const uint32_t *__restrict__ vals, const uint64_t *__restrict__ grad_ptr,
                           const uint32_t *__restrict__ view_off, int n_views, int stride,
                           float *__restrict__ out) {
    const uint32_t nruns = *d_nruns;
    const int lane = threadIdx.x & 31;
    for (uint32_t u = (blockIdx.x * BB + threadIdx.x) >> 5; u < nruns; u += (gridDim.x * BB) >> 5) {
        const uint32_t s = run_start[u], e = run_start[u + 1];
        for (int c = lane; c < stride; c += 32) {
            float acc = 0.f;
            for (uint32_t p = s; p < e; ++p) {
                const uint32_t g = vals[p];
                int v = 0;
                while (v + 1 < n_views && view_off[v + 1] <= g) ++v;
                const float *rows = reinterpret_cast<const float *>(grad_ptr[v]);
                acc += rows[(size_t)(g - view_off[v]) * stride + c];
            }
            out[(size_t)u * stride + c] = acc;
        }
    }
}

int nb(uint64_t n) { return (int)std::max<uint64_t>(1, (n + BB - 1) / BB); }

}  // namespace

extern "C" int lodgs_accumulate_grads(lodgs_scene *sc, lodgs_frame *const *frames, const float *const *grads,
                                      int n_views, uint32_t *out_rows, float *out_grads, int64_t capacity,
                                      uint32_t *d_count, void *stream) {
    if (!sc || !frames || !grads || n_views < 1 || !out_rows || !out_grads || !d_count) {
        set_error("accumulate_grads: NULL argument or no views");
        return LODGS_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<uint32_t> off(n_views + 1, 0);
    std::vector<uint64_t> gp(n_views);
    for (int v = 0; v < n_views; ++v) {
        lodgs_frame *fr = frames[v];
        if (!fr || fr->scene != sc || fr->layout_version != sc->layout_version || !fr->rendered || !grads[v]) {
            set_error("accumulate_grads: every view needs a rendered frame of this scene's current layout and its "
                      "gradient rows");
            return LODGS_E_STATE;
        }
        LODGS_CUDA(cudaStreamSynchronize(fr->stream));
        off[v + 1] = off[v] + fr->h_cnt[C_NSEL_EFF];
        gp[v] = (uint64_t)(uintptr_t)grads[v];
    }
    const uint32_t T = off[n_views];
    if ((int64_t)T > capacity) { set_error("accumulate_grads: capacity below the total selection"); return LODGS_E_INVALID; }
    if (T == 0) { LODGS_CUDA(cudaMemsetAsync(d_count, 0, 4, st)); return LODGS_OK; }
    // stream-ordered temporaries
    uint32_t *buf = nullptr;
    const size_t words = 2 * (size_t)n_views + (size_t)T * 7 + SORT_HIST + SCAN_GRID_MAX + 8 + (size_t)(n_views + 1) + 64;
    LODGS_CUDA(cudaMallocAsync((void **)&buf, words * 4, st));
    uint64_t *gptr = reinterpret_cast<uint64_t *>(buf);    // first, so it is 8-byte aligned
    uint32_t *key = buf + 2 * n_views, *val = key + T, *key2 = val + T, *val2 = key2 + T, *flag = val2 + T,
             *pos = flag + T, *run_start = pos + T, *hist = run_start + T + 1, *bsum = hist + SORT_HIST,
             *dn = bsum + SCAN_GRID_MAX, *voff = dn + 8;
    for (int v = 0; v < n_views; ++v) {
        const uint32_t n = off[v + 1] - off[v];
        if (!n) continue;
        LODGS_CUDA(cudaMemcpyAsync(key + off[v], frames[v]->f.sel_rows, n * 4, cudaMemcpyDeviceToDevice, st));
        k_iota<<<nb(n), BB, 0, st>>>(val + off[v], off[v], n);
        count_launches(1);
    }
    LODGS_CUDA(cudaMemcpyAsync(dn, &T, 4, cudaMemcpyHostToDevice, st));
    LODGS_CUDA(cudaMemcpyAsync(voff, off.data(), (n_views + 1) * 4, cudaMemcpyHostToDevice, st));
    LODGS_CUDA(cudaMemcpyAsync(gptr, gp.data(), n_views * 8, cudaMemcpyHostToDevice, st));
    int bits = 1;
    while ((1ull << bits) < (uint64_t)sc->n_nodes) ++bits;
    bool alt = false;
    int rc = radix_sort_pairs(key, val, key2, val2, dn, T, 0, bits, hist, st, &alt);
    if (rc) { cudaFreeAsync(buf, st); return rc; }
    const uint32_t *sk = alt ? key2 : key, *sv = alt ? val2 : val;
    k_run_starts<<<nb(T), BB, 0, st>>>(sk, T, flag);
    count_launches(1);
    rc = scan_exclusive(flag, pos, dn, T, bsum, d_count, st);
    if (rc) { cudaFreeAsync(buf, st); return rc; }
    k_runs<<<nb(T), BB, 0, st>>>(sk, flag, pos, T, out_rows, run_start);
    count_launches(1);
    k_sum_runs<<<1184, BB, 0, st>>>(run_start, d_count, sv, gptr, voff, n_views, sc->stride, out_grads);
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    LODGS_CUDA(cudaFreeAsync(buf, st));
    return LODGS_OK;
}
