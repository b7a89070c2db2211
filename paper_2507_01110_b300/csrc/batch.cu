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

// One warp per run (a node row selected by several views).  The lanes find
// the view and row address of up to 32 entries of the run at once; the warp
// then loads eight entries' rows at a time, each lane two columns (a float2
// when VEC == 2, columns lane and lane + 32 otherwise), and adds them in entry
// order (view order), so the sum is the deterministic view-ordered one while
// the run's row loads are in flight together.  Rows are at most 64 floats.
constexpr int SUM_GROUP = 8;

template <int VEC>
__global__ void __launch_bounds__(BB) k_sum_runs(const uint32_t *__restrict__ run_start,
                                                 const uint32_t *__restrict__ d_nruns,
                                                 const uint32_t *__restrict__ vals,
                                                 const uint64_t *__restrict__ grad_ptr,
                                                 const uint32_t *__restrict__ view_off, int n_views, int stride,
                                                 float *__restrict__ out) {
    const uint32_t nruns = *d_nruns;
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = (gridDim.x * BB) >> 5;
    for (uint32_t u = (blockIdx.x * BB + threadIdx.x) >> 5; u < nruns; u += nwarps) {
        const uint32_t s = run_start[u], e = run_start[u + 1];
        float a0 = 0.f, a1 = 0.f;                        // this lane's two columns
        for (uint32_t p0 = s; p0 < e; p0 += 32) {
            const uint32_t L = e - p0 < 32u ? e - p0 : 32u;
            uint64_t rp = 0;                             // entry p0 + lane: its row's address
            if ((uint32_t)lane < L) {
                const uint32_t g = vals[p0 + lane];
                int lo = 0, hi = n_views;                // the last view v with view_off[v] <= g
                while (hi - lo > 1) {
                    const int m = (lo + hi) >> 1;
                    if (view_off[m] <= g) lo = m; else hi = m;
                }
                rp = grad_ptr[lo] + (uint64_t)(g - view_off[lo]) * (uint64_t)stride * 4u;
            }
            for (uint32_t k0 = 0; k0 < L; k0 += SUM_GROUP) {
                float x0[SUM_GROUP], x1[SUM_GROUP];
#pragma unroll
                for (int k = 0; k < SUM_GROUP; ++k) {
                    const uint64_t r = __shfl_sync(0xffffffffu, rp, (int)k0 + k);
                    x0[k] = x1[k] = 0.f;
                    if (k0 + k < L) {
                        const float *row = reinterpret_cast<const float *>(r);
                        if (VEC == 2) {
                            if (2 * lane < stride) {
                                const float2 t = reinterpret_cast<const float2 *>(row)[lane];
                                x0[k] = t.x;
                                x1[k] = t.y;
                            }
                        } else {
                            if (lane < stride) x0[k] = row[lane];
                            if (lane + 32 < stride) x1[k] = row[lane + 32];
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < SUM_GROUP; ++k) {
                    if (k0 + k < L) {
                        a0 += x0[k];
                        a1 += x1[k];
                    }
                }
            }
        }
        float *o = out + (size_t)u * stride;
        if (VEC == 2) {
            if (2 * lane < stride) reinterpret_cast<float2 *>(o)[lane] = make_float2(a0, a1);
        } else {
            if (lane < stride) o[lane] = a0;
            if (lane + 32 < stride) o[lane + 32] = a1;
        }
    }
}

// The row address of every entry (its view's gradient array at the entry's
// index within the view), one coalesced pass, so that the summation below
// starts each run's row loads one step after reading the run's bounds.
__global__ void k_entry_addr(const uint32_t *__restrict__ vals, uint32_t n, const uint64_t *__restrict__ grad_ptr,
                             const uint32_t *__restrict__ view_off, int n_views, int stride,
                             uint64_t *__restrict__ addr) {
    const uint32_t p = blockIdx.x * BB + threadIdx.x;
    if (p >= n) return;
    const uint32_t g = vals[p];
    int lo = 0, hi = n_views;                            // the last view v with view_off[v] <= g
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (view_off[m] <= g) lo = m; else hi = m;
    }
    addr[p] = grad_ptr[lo] + (uint64_t)(g - view_off[lo]) * (uint64_t)stride * 4u;
}

// Runs summed by lane groups: LPR = stride / 4 lanes per run, each lane one
// float4 column of the row, 32 / LPR runs per warp and RUNS_UNROLL of those
// groups per iteration, so that many runs' row loads are in flight at once.
// Each column is summed in entry order (view order) from 0, as k_sum_runs does.
constexpr int RUNS_UNROLL = 4;

template <int LPR>
__global__ void __launch_bounds__(BB) k_sum_runs4(const uint32_t *__restrict__ run_start,
                                                  const uint32_t *__restrict__ d_nruns,
                                                  const uint64_t *__restrict__ addr, float4 *__restrict__ out) {
    constexpr int RPW = 32 / LPR;                        // runs per warp
    const uint32_t nruns = *d_nruns;
    const int lane = threadIdx.x & 31, grp = lane / LPR, c = lane % LPR;
    const bool lane_on = grp < RPW;
    const uint64_t w = (blockIdx.x * BB + threadIdx.x) >> 5, nw = (gridDim.x * BB) >> 5;
    for (uint64_t base = w * RPW * RUNS_UNROLL; base < nruns; base += nw * RPW * RUNS_UNROLL) {
        uint32_t s[RUNS_UNROLL], e[RUNS_UNROLL];
        float4 acc[RUNS_UNROLL];
#pragma unroll
        for (int j = 0; j < RUNS_UNROLL; ++j) {
            const uint64_t u = base + (uint64_t)j * RPW + grp;
            s[j] = e[j] = 0;
            if (lane_on && u < nruns) {
                s[j] = run_start[u];
                e[j] = run_start[u + 1];
            }
            acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (uint32_t k = 0;; ++k) {
            bool any = false;
            float4 x[RUNS_UNROLL];
#pragma unroll
            for (int j = 0; j < RUNS_UNROLL; ++j) {
                if (s[j] + k < e[j]) {
                    x[j] = reinterpret_cast<const float4 *>(addr[s[j] + k])[c];
                    any = true;
                }
            }
#pragma unroll
            for (int j = 0; j < RUNS_UNROLL; ++j) {
                if (s[j] + k < e[j]) {
                    acc[j].x += x[j].x; acc[j].y += x[j].y; acc[j].z += x[j].z; acc[j].w += x[j].w;
                }
            }
            if (!__any_sync(0xffffffffu, any)) break;
        }
#pragma unroll
        for (int j = 0; j < RUNS_UNROLL; ++j) {
            const uint64_t u = base + (uint64_t)j * RPW + grp;
            if (lane_on && u < nruns) out[u * LPR + c] = acc[j];
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
        if (!fr || fr->scene != sc || fr->layout_version != sc->layout_version || !fr->rendered) {
            set_error("accumulate_grads: every view needs a rendered frame of this scene's current layout");
            return LODGS_E_STATE;
        }
        LODGS_CUDA(cudaStreamSynchronize(fr->stream));
        if (!grads[v] && fr->h_cnt[C_NSEL_EFF] > 0) {        // a view that selected nothing may pass NULL
            set_error("accumulate_grads: a view with selected nodes needs its gradient rows");
            return LODGS_E_STATE;
        }
        off[v + 1] = off[v] + fr->h_cnt[C_NSEL_EFF];
        gp[v] = (uint64_t)(uintptr_t)grads[v];
    }
    if (sc->stride > 64 || (sc->stride & 1)) { set_error("accumulate_grads: rows of at most 64 floats"); return LODGS_E_INVALID; }
    const uint32_t T = off[n_views];
    if ((int64_t)T > capacity) { set_error("accumulate_grads: capacity below the total selection"); return LODGS_E_INVALID; }
    if (T == 0) { LODGS_CUDA(cudaMemsetAsync(d_count, 0, 4, st)); return LODGS_OK; }
    // stream-ordered temporaries
    uint32_t *buf = nullptr;
    // float4 rows when every row array is 16-byte aligned (row strides are multiples of 16 bytes)
    bool vec4 = ((uintptr_t)out_grads & 15u) == 0 && sc->stride % 4 == 0;
    for (int v = 0; v < n_views; ++v) vec4 = vec4 && (gp[v] & 15u) == 0;
    const size_t words = 2 * (size_t)n_views + (size_t)T * (vec4 ? 9 : 7) + SORT_HIST + SCAN_GRID_MAX + 8 +
                         (size_t)(n_views + 1) + 64;
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
    const int lpr = sc->stride / 4;
    if (vec4 && (lpr == 4 || lpr == 6 || lpr == 10 || lpr == 16)) {
        uint64_t *addr = reinterpret_cast<uint64_t *>(((uintptr_t)(voff + n_views + 1) + 7u) & ~(uintptr_t)7u);
        k_entry_addr<<<nb(T), BB, 0, st>>>(sv, T, gptr, voff, n_views, sc->stride, addr);
        float4 *o4 = reinterpret_cast<float4 *>(out_grads);
        if (lpr == 16) k_sum_runs4<16><<<1184, BB, 0, st>>>(run_start, d_count, addr, o4);
        else if (lpr == 10) k_sum_runs4<10><<<1184, BB, 0, st>>>(run_start, d_count, addr, o4);
        else if (lpr == 6) k_sum_runs4<6><<<1184, BB, 0, st>>>(run_start, d_count, addr, o4);
        else k_sum_runs4<4><<<1184, BB, 0, st>>>(run_start, d_count, addr, o4);
        count_launches(2);
    } else {
        // float2 rows when every row array is 8-byte aligned (strides are even)
        bool vec2 = ((uintptr_t)out_grads & 7u) == 0;
        for (int v = 0; v < n_views; ++v) vec2 = vec2 && (gp[v] & 7u) == 0;
        if (vec2)
            k_sum_runs<2><<<1184, BB, 0, st>>>(run_start, d_count, sv, gptr, voff, n_views, sc->stride, out_grads);
        else
            k_sum_runs<1><<<1184, BB, 0, st>>>(run_start, d_count, sv, gptr, voff, n_views, sc->stride, out_grads);
        count_launches(1);
    }
    LODGS_CUDA(cudaGetLastError());
    LODGS_CUDA(cudaFreeAsync(buf, st));
    return LODGS_OK;
}
