// Gradient of a multi-view batch loss on the union of the views' cuts.
//
// Each view's backward writes one gradient row per node of its own LoD cut;
// only cut-set nodes receive gradients (appendix "Implementation Details").  For
// a batch of views the rows of a node selected by several views must be summed.
// The entries (a view's selected rows) are grouped by node row in view order:
// for up to 8 views from one byte of view bits per node row (no sort, see
// k_mark_views); for more views by a stable radix sort of the concatenated
// rows, split into runs of equal rows (scan of run starts).  Each run is
// summed in view order, so the result is deterministic and no float atomics
// are needed.
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

// ---- grouping without a sort (up to 8 views) ----
// Every view's selection is ascending and holds a row once, so the (row, view)
// order of the entries that the stable sort gives can be built from one byte
// per node row: bit v set when view v selected the row.  The union rows are
// the rows with a nonzero byte (ascending), a row's run starts after the
// entries of the union rows before it (the popcounts), and view v's entry of
// row r sits at the run's start plus the number of earlier views that selected
// r.  Bytes are packed four to a word.
constexpr int CH_WORDS = 1024;                 // mask words per chunk (one block of BB threads, 4 words each)
constexpr int CH_PER_THREAD = CH_WORDS / BB;

__global__ void k_mark_views(const uint32_t *__restrict__ sel, uint32_t n, int v, uint32_t *__restrict__ mask) {
    const uint32_t i = blockIdx.x * BB + threadIdx.x;
    if (i >= n) return;
    const uint32_t r = sel[i];
    atomicOr(&mask[r >> 2], (1u << v) << (8 * (r & 3u)));
}

__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t w) {
    return (uint32_t)((w & 0xffu) != 0) + (uint32_t)((w & 0xff00u) != 0) + (uint32_t)((w & 0xff0000u) != 0) +
           (uint32_t)((w & 0xff000000u) != 0);
}

// union rows (cu) and entries (ce) of each chunk
__global__ void __launch_bounds__(BB) k_chunk_counts(const uint32_t *__restrict__ mask, uint64_t n_words,
                                                     uint32_t *__restrict__ cu, uint32_t *__restrict__ ce) {
    __shared__ uint32_t s_u[BB / 32], s_e[BB / 32];
    const uint64_t w0 = (uint64_t)blockIdx.x * CH_WORDS + (uint64_t)threadIdx.x * CH_PER_THREAD;
    uint32_t nu = 0, ne = 0;
#pragma unroll
    for (int k = 0; k < CH_PER_THREAD; ++k) {
        const uint32_t w = w0 + k < n_words ? mask[w0 + k] : 0u;
        nu += nonzero_bytes(w);
        ne += __popc(w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nu += __shfl_xor_sync(0xffffffffu, nu, o);
        ne += __shfl_xor_sync(0xffffffffu, ne, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s_u[warp] = nu; s_e[warp] = ne; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0, b = 0;
#pragma unroll
        for (int w = 0; w < BB / 32; ++w) { a += s_u[w]; b += s_e[w]; }
        cu[blockIdx.x] = a;
        ce[blockIdx.x] = b;
    }
}

// The union rows of each chunk in ascending order: out_rows[u], the start of
// their run of entries (run_start[u], and the end of the last run at
// run_start[U]) and slot[r] = u for the entry pass.  cu_off / ce_off: the
// exclusive scans of the chunks' counts; *d_nruns: the union row count U.
__global__ void __launch_bounds__(BB) k_chunk_write(const uint32_t *__restrict__ mask, uint64_t n_words,
                                                    const uint32_t *__restrict__ cu_off,
                                                    const uint32_t *__restrict__ ce_off,
                                                    const uint32_t *__restrict__ d_nruns,
                                                    uint32_t *__restrict__ out_rows, uint32_t *__restrict__ run_start,
                                                    uint32_t *__restrict__ slot) {
    __shared__ uint32_t s_u[BB / 32], s_e[BB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t ubase = cu_off[blockIdx.x], ebase = ce_off[blockIdx.x];
    const uint32_t U = *d_nruns;
    // CH_PER_THREAD rounds of BB consecutive words (one per thread, so that
    // neighbouring threads write neighbouring rows), each with block-wide
    // exclusive scans of the union rows and entries, in row order
    for (int k = 0; k < CH_PER_THREAD; ++k) {
        const uint64_t wi = (uint64_t)blockIdx.x * CH_WORDS + (uint64_t)k * BB + threadIdx.x;
        const uint32_t w = wi < n_words ? mask[wi] : 0u;
        const uint32_t nu = nonzero_bytes(w), ne = __popc(w);
        uint32_t xu = nu, xe = ne;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yu = __shfl_up_sync(0xffffffffu, xu, o), ye = __shfl_up_sync(0xffffffffu, xe, o);
            if (lane >= o) { xu += yu; xe += ye; }
        }
        if (lane == 31) { s_u[warp] = xu; s_e[warp] = xe; }
        __syncthreads();
        uint32_t u = ubase + xu - nu, e = ebase + xe - ne, tu = 0, te = 0;
#pragma unroll
        for (int j = 0; j < BB / 32; ++j) {
            const uint32_t a = s_u[j], b = s_e[j];
            if (j < warp) { u += a; e += b; }
            tu += a;
            te += b;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t m = (w >> (8 * b)) & 0xffu;
            if (!m) continue;
            const uint32_t r = (uint32_t)(wi * 4u + b);
            out_rows[u] = r;
            run_start[u] = e;
            slot[r] = u;
            e += __popc(m);
            if (u + 1 == U) run_start[U] = e;            // one past the last run
            ++u;
        }
        ubase += tu;
        ebase += te;
        __syncthreads();                                 // s_u and s_e are rewritten next round
    }
}

// Place view v's entries (index i in the view, row sel[i]) in (row, view)
// order: the entry id (vals) and, if addr is given, its gradient row's address.
__global__ void k_place_entries(const uint32_t *__restrict__ sel, uint32_t n, int v, uint32_t first,
                                uint64_t grad_base, int stride, const uint32_t *__restrict__ mask,
                                const uint32_t *__restrict__ slot, const uint32_t *__restrict__ run_start,
                                uint32_t *__restrict__ vals, uint64_t *__restrict__ addr) {
    const uint32_t i = blockIdx.x * BB + threadIdx.x;
    if (i >= n) return;
    const uint32_t r = sel[i];
    const uint32_t m = (mask[r >> 2] >> (8 * (r & 3u))) & 0xffu;
    const uint32_t p = run_start[slot[r]] + (uint32_t)__popc(m & ((1u << v) - 1u));
    vals[p] = first + i;
    if (addr) addr[p] = grad_base + (uint64_t)i * (uint64_t)stride * 4u;
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

// The runs summed into out_grads: the lane-group kernel over the entries' row
// addresses (addr) when rows are float4-aligned and their width is one it is
// instantiated for, else one warp per run over the entry ids (sv).
int launch_sums(const lodgs_scene *sc, bool vec4, bool vec2, const uint32_t *run_start, const uint32_t *d_count,
                const uint32_t *sv, const uint64_t *addr, const uint64_t *gptr, const uint32_t *voff, int n_views,
                float *out_grads, cudaStream_t st) {
    const int lpr = sc->stride / 4;
    if (vec4 && addr && (lpr == 4 || lpr == 6 || lpr == 10 || lpr == 16)) {
        float4 *o4 = reinterpret_cast<float4 *>(out_grads);
        if (lpr == 16) k_sum_runs4<16><<<1184, BB, 0, st>>>(run_start, d_count, addr, o4);
        else if (lpr == 10) k_sum_runs4<10><<<1184, BB, 0, st>>>(run_start, d_count, addr, o4);
        else if (lpr == 6) k_sum_runs4<6><<<1184, BB, 0, st>>>(run_start, d_count, addr, o4);
        else k_sum_runs4<4><<<1184, BB, 0, st>>>(run_start, d_count, addr, o4);
    } else if (vec2) {
        k_sum_runs<2><<<1184, BB, 0, st>>>(run_start, d_count, sv, gptr, voff, n_views, sc->stride, out_grads);
    } else {
        k_sum_runs<1><<<1184, BB, 0, st>>>(run_start, d_count, sv, gptr, voff, n_views, sc->stride, out_grads);
    }
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

// Grouping by view masks (up to 8 views; see k_mark_views), then the sums.
int accumulate_by_mask(const lodgs_scene *sc, lodgs_frame *const *frames, const std::vector<uint32_t> &off,
                       const std::vector<uint64_t> &gp, int n_views, uint32_t *out_rows, float *out_grads,
                       uint32_t *d_count, bool vec4, bool vec2, cudaStream_t st) {
    const uint32_t T = off[n_views];
    const uint64_t M = (uint64_t)sc->n_nodes;
    const uint64_t n_chunks = ((M + 3) / 4 + CH_WORDS - 1) / CH_WORDS;
    const uint64_t W = n_chunks * CH_WORDS;                 // mask words, whole chunks
    const size_t words = 2 * (size_t)n_views + 2 * (size_t)T + 2 +          // gptr, addr (8-byte words first)
                         W + M + 4 * n_chunks + SCAN_GRID_MAX + 8 + (size_t)(n_views + 1) + (size_t)T + 1 + T;
    uint32_t *buf = nullptr;
    LODGS_CUDA(cudaMallocAsync((void **)&buf, words * 4, st));
    uint64_t *gptr = reinterpret_cast<uint64_t *>(buf);
    uint64_t *addr = gptr + n_views;
    uint32_t *mask = reinterpret_cast<uint32_t *>(addr + T + 1), *slot = mask + W, *cu = slot + M,
             *ce = cu + n_chunks, *cu_off = ce + n_chunks, *ce_off = cu_off + n_chunks,
             *bsum = ce_off + n_chunks, *dn = bsum + SCAN_GRID_MAX, *voff = dn + 8, *run_start = voff + n_views + 1,
             *sv = run_start + T + 1;
    int rc = LODGS_OK;
    const uint32_t nc = (uint32_t)n_chunks;
    LODGS_CUDA(cudaMemsetAsync(mask, 0, W * 4, st));
    LODGS_CUDA(cudaMemcpyAsync(dn, &nc, 4, cudaMemcpyHostToDevice, st));
    LODGS_CUDA(cudaMemcpyAsync(voff, off.data(), (n_views + 1) * 4, cudaMemcpyHostToDevice, st));
    LODGS_CUDA(cudaMemcpyAsync(gptr, gp.data(), n_views * 8, cudaMemcpyHostToDevice, st));
    for (int v = 0; v < n_views; ++v) {
        const uint32_t n = off[v + 1] - off[v];
        if (!n) continue;
        k_mark_views<<<nb(n), BB, 0, st>>>(frames[v]->f.sel_rows, n, v, mask);
        count_launches(1);
    }
    k_chunk_counts<<<nc, BB, 0, st>>>(mask, W, cu, ce);
    count_launches(1);
    rc = scan_exclusive(cu, cu_off, dn, nc, bsum, d_count, st);
    if (!rc) rc = scan_exclusive(ce, ce_off, dn, nc, bsum, dn + 1, st);
    if (rc) { cudaFreeAsync(buf, st); return rc; }
    k_chunk_write<<<nc, BB, 0, st>>>(mask, W, cu_off, ce_off, d_count, out_rows, run_start, slot);
    count_launches(1);
    for (int v = 0; v < n_views; ++v) {
        const uint32_t n = off[v + 1] - off[v];
        if (!n) continue;
        k_place_entries<<<nb(n), BB, 0, st>>>(frames[v]->f.sel_rows, n, v, off[v], gp[v], sc->stride, mask, slot,
                                              run_start, sv, vec4 ? addr : nullptr);
        count_launches(1);
    }
    LODGS_CUDA(cudaGetLastError());
    rc = launch_sums(sc, vec4, vec2, run_start, d_count, sv, addr, gptr, voff, n_views, out_grads, st);
    cudaFreeAsync(buf, st);
    return rc;
}

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
    // float4 rows when every row array is 16-byte aligned (row strides are multiples of 16 bytes),
    // float2 rows when every row array is 8-byte aligned (strides are even)
    bool vec4 = ((uintptr_t)out_grads & 15u) == 0 && sc->stride % 4 == 0;
    for (int v = 0; v < n_views; ++v) vec4 = vec4 && (gp[v] & 15u) == 0;
    bool vec2 = ((uintptr_t)out_grads & 7u) == 0;
    for (int v = 0; v < n_views; ++v) vec2 = vec2 && (gp[v] & 7u) == 0;
    if (n_views <= 8)
        return accumulate_by_mask(sc, frames, off, gp, n_views, out_rows, out_grads, d_count, vec4, vec2, st);
    // more views: the entries sorted by node row (stream-ordered temporaries)
    uint32_t *buf = nullptr;
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
    uint64_t *addr = nullptr;
    if (vec4 && (lpr == 4 || lpr == 6 || lpr == 10 || lpr == 16)) {
        addr = reinterpret_cast<uint64_t *>(((uintptr_t)(voff + n_views + 1) + 7u) & ~(uintptr_t)7u);
        k_entry_addr<<<nb(T), BB, 0, st>>>(sv, T, gptr, voff, n_views, sc->stride, addr);
        count_launches(1);
    }
    rc = launch_sums(sc, vec4, vec2, run_start, d_count, sv, addr, gptr, voff, n_views, out_grads, st);
    if (rc) { cudaFreeAsync(buf, st); return rc; }
    LODGS_CUDA(cudaGetLastError());
    LODGS_CUDA(cudaFreeAsync(buf, st));
    return LODGS_OK;
}
