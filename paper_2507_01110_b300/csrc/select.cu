// LoD cut selection (Sec. 4.3, Algorithms 1 and 2).
//
// a1  Upper hierarchy.  Algorithm 1 visits an entry iff every ancestor was
//     visited and descended into (not culled, not fine enough, not an SPT
//     root).  Each thread decides one entry by evaluating its own test and then
//     walking its ancestor chain (the upper hierarchy is small: ~2 entries per
//     SPT), so no level-by-level frontier or host round trip is needed.  An
//     ordered two-pass compaction emits the selected upper rows and the SPT
//     roots to cut, both ascending.
// a2  SPTs.  Per SPT root, a binary search on the descending parent bounds `hi`
//     gives the prefix [0, high) of possibly selected entries (Alg. 2); a flat,
//     load-balanced pass over the concatenated prefixes keeps the entries with
//     lo <= x (Eq. 4) and compacts them in order.
//
// Compiled with -fmad=false: the tests are evaluated exactly as written.
#include "lodgs_internal.cuh"

namespace lodgs {
namespace {

constexpr int SB = 256;
constexpr int SEL_GRID = 296;
// blocks of the SPT passes: one wave of 6 blocks per SM, so that each block
// walks few tiles (every tile is a few dependent global-load rounds)
constexpr int SPT_GRID = 148 * 6;
static_assert(SPT_GRID <= SEL_BLOCK_COUNTS && SEL_GRID <= SEL_BLOCK_COUNTS, "per-block counts buffer");

enum { OUT_NONE = 0, OUT_SELECT = 1, OUT_SPT = 2 };

// One view's selection buffers.  Every selection kernel takes the views of a
// batch by value and serves view blockIdx.y of them: lodgs_select_lod is a
// batch of one, lodgs_select_lod_batch a batch of up to SEL_BATCH_MAX.
struct SelPtrs {
    const View *view;
    uint32_t *cnt, *bc, *sel_rows, *sel_src, *emit_j, *high, *work_off, *scan_bsum;
    float *emit_x, *up_x;
    uint8_t *up_out;
    const uint32_t *emit_src;
};
constexpr int SEL_BATCH_MAX = SCAN_BATCH_MAX;
struct SelBatch {
    SelPtrs v[SEL_BATCH_MAX];
};

// Algorithm 1 outcome for upper entry u; *x_out = tau * d / f of the entry.
__device__ int upper_outcome(const UpperEntry *__restrict__ up, int u, const CamK &k, float *x_out) {
    UpperEntry e = up[u];
    float t[3], dist;
    cam_view(k, e.mu[0], e.mu[1], e.mu[2], t, &dist);
    if (cam_culled(k, t, e.maxs)) return OUT_NONE;
    float x = dist * k.inv_k;
    int out;
    if (e.kind == KIND_SPT) { out = OUT_SPT; x = x * k.spt_scale; }   // LoD noise on the SPT distances
    else if (e.kind == KIND_LEAF) out = OUT_SELECT;
    else if (e.S <= x) out = OUT_SELECT;
    else return OUT_NONE;
    *x_out = x;
    for (int a = e.parent; a >= 0; a = up[a].parent) {      // every ancestor must have descended
        UpperEntry f = up[a];
        cam_view(k, f.mu[0], f.mu[1], f.mu[2], t, &dist);
        if (cam_culled(k, t, f.maxs)) return OUT_NONE;
        if (f.S <= dist * k.inv_k) return OUT_NONE;          // an ancestor was selected
    }
    return out;
}

__device__ __forceinline__ void grid_chunk(uint32_t n, uint32_t &begin, uint32_t &end) {
    uint32_t G = gridDim.x;
    uint32_t per = (n + G - 1) / G;
    per = (per + SB - 1) / SB * SB;
    uint64_t b = (uint64_t)blockIdx.x * per;
    begin = b < n ? (uint32_t)b : n;
    uint64_t e2 = b + per;
    end = e2 < n ? (uint32_t)e2 : n;
}

// inclusive block scan of one value per thread (SB threads); returns exclusive
// prefix, *total gets the block total
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SB / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SB / 32) s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t excl = (warp ? s_warp[warp - 1] : 0u) + x - v;
    *total = s_warp[SB / 32 - 1];
    __syncthreads();
    return excl;
}

__device__ __forceinline__ uint32_t block_prefix(const uint32_t *__restrict__ counts, uint32_t *s_warp) {
    uint32_t s = 0;
    for (uint32_t b = threadIdx.x; b < blockIdx.x; b += SB) s += counts[b];
    uint32_t tot;
    block_scan(s, s_warp, &tot);
    return tot;
}

// ---- a1 --------------------------------------------------------------------
// Counts per block; with a cache (up_out, up_x) the outcomes are kept for the
// write pass, which then skips the ancestor walks.
__global__ void __launch_bounds__(SB) k_upper_count(const UpperEntry *__restrict__ up, uint32_t U, SelBatch B) {
    pdl_wait();
    const SelPtrs &P = B.v[blockIdx.y];
    const CamK &k = P.view->k;
    uint32_t *__restrict__ bc = P.bc;
    uint8_t *__restrict__ up_out = P.up_out;
    float *__restrict__ up_x = P.up_x;
    __shared__ uint32_t s_warp[32];
    uint32_t begin, end;
    grid_chunk(U, begin, end);
    uint32_t packed = 0;
    for (uint32_t u = begin + threadIdx.x; u < end; u += SB) {
        float x = 0.f;
        int o = upper_outcome(up, (int)u, k, &x);
        packed += o == OUT_SELECT ? 1u : (o == OUT_SPT ? 0x10000u : 0u);
        if (up_out) { up_out[u] = (uint8_t)o; up_x[u] = x; }
    }
    uint32_t tot;
    block_scan(packed, s_warp, &tot);   // counts per block < 65536 per field (U / grid)
    if (threadIdx.x == 0) bc[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SB) k_upper_write(const UpperEntry *__restrict__ up, uint32_t U, SelBatch B) {
    pdl_wait();
    const SelPtrs &P = B.v[blockIdx.y];
    const CamK &k = P.view->k;
    const uint32_t *__restrict__ bc = P.bc;
    const uint8_t *__restrict__ up_out = P.up_out;
    const float *__restrict__ up_x = P.up_x;
    uint32_t *__restrict__ sel_rows = P.sel_rows, *__restrict__ sel_src = P.sel_src, *__restrict__ emit_j = P.emit_j;
    float *__restrict__ emit_x = P.emit_x;
    uint32_t *__restrict__ cnt = P.cnt;
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_off_sel, s_off_emit;
    uint32_t sel_before = 0, emit_before = 0;
    {
        uint32_t s = 0, e = 0;
        for (uint32_t b = threadIdx.x; b < blockIdx.x; b += SB) { s += bc[b] & 0xffffu; e += bc[b] >> 16; }
        uint32_t ts, te;
        block_scan(s, s_warp, &ts);
        block_scan(e, s_warp, &te);
        sel_before = ts; emit_before = te;
    }
    if (threadIdx.x == 0) { s_off_sel = sel_before; s_off_emit = emit_before; }
    __syncthreads();
    uint32_t begin, end;
    grid_chunk(U, begin, end);
    for (uint32_t t0 = begin; t0 < end; t0 += SB) {
        uint32_t u = t0 + threadIdx.x;
        float x = 0.f;
        int o = OUT_NONE;
        if (u < end) {
            if (up_out) { o = up_out[u]; x = up_x[u]; }
            else o = upper_outcome(up, (int)u, k, &x);
        }
        uint32_t packed = o == OUT_SELECT ? 1u : (o == OUT_SPT ? 0x10000u : 0u);
        uint32_t tot;
        uint32_t ex = block_scan(packed, s_warp, &tot);
        uint32_t os = s_off_sel, oe = s_off_emit;
        if (o == OUT_SELECT) {
            sel_rows[os + (ex & 0xffffu)] = (uint32_t)up[u].ref;
            if (sel_src) sel_src[os + (ex & 0xffffu)] = (uint32_t)up[u].ref;   // upper rows are resident
        }
        if (o == OUT_SPT) {
            emit_j[oe + (ex >> 16)] = (uint32_t)up[u].ref;
            emit_x[oe + (ex >> 16)] = x;
        }
        __syncthreads();
        if (threadIdx.x == 0) { s_off_sel = os + (tot & 0xffffu); s_off_emit = oe + (tot >> 16); }
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        cnt[C_NUP] = s_off_sel;
        cnt[C_NEMIT] = s_off_emit;
    }
}

// ---- a2 --------------------------------------------------------------------

// Number of leading entries of arr[0, n) that satisfy `pred`, which must hold
// on a prefix (a monotone predicate over sorted data), found by one warp: each
// round tests 32 evenly spaced pivots of the unresolved range and keeps the
// gap between the last pivot that holds and the first that does not, so a
// range of n entries takes about log_33(n) dependent load rounds instead of
// log_2(n).  All lanes of the warp must call it with the same arguments.
template <typename T, typename Pred>
__device__ __forceinline__ uint32_t warp_prefix_count(const T *__restrict__ arr, uint32_t n, Pred pred) {
    const uint32_t lane = threadIdx.x & 31;
    uint32_t a = 0, b = n;                                  // [0, a) hold, [b, n) do not
    while (b - a > 32) {
        const uint64_t span = b - a;
        const uint32_t m = a + (uint32_t)(span * (lane + 1) / 33);         // a < m < b
        const uint32_t c = __popc(__ballot_sync(0xffffffffu, pred(arr[m])));
        const uint32_t m_last = a + (uint32_t)(span * c / 33);             // pivot c - 1 (c > 0)
        const uint32_t m_first = a + (uint32_t)(span * (c + 1) / 33);      // pivot c (c < 32)
        if (c > 0) a = m_last + 1;
        if (c < 32) b = m_first;
    }
    const bool in = lane < b - a;
    return a + __popc(__ballot_sync(0xffffffffu, in && pred(arr[a + lane])));
}

// One warp per emitted SPT: high = the first entry with hi <= x (entries are
// sorted by descending hi).
__global__ void __launch_bounds__(SB) k_spt_high(const uint32_t *__restrict__ spt_base, const float *__restrict__ hi_row,
                                                 SelBatch B) {
    pdl_wait();
    const SelPtrs &P = B.v[blockIdx.y];
    const uint32_t *__restrict__ cnt_in = P.cnt, *__restrict__ emit_j = P.emit_j;
    const float *__restrict__ emit_x = P.emit_x;
    uint32_t *__restrict__ high = P.high;
    const uint32_t n = cnt_in[C_NEMIT];
    const uint32_t warps = gridDim.x * (SB / 32);
    for (uint32_t q = blockIdx.x * (SB / 32) + (threadIdx.x >> 5); q < n; q += warps) {
        const uint32_t j = emit_j[q];
        const float x = emit_x[q];
        const uint32_t base = spt_base[j];
        const uint32_t h = warp_prefix_count(hi_row + base, spt_base[j + 1] - base, [x](float hi) { return hi > x; });
        if ((threadIdx.x & 31) == 0) high[q] = h;
    }
}

// The work items (SPT entries to test) of a tile of SB consecutive items belong
// to at most SB consecutive emitted SPTs (each SPT has at least one item, its
// root), starting at the SPT of the tile's first item.  A tile stages those
// SPTs' item offsets, row bases, query values (and record slots) in shared
// memory, so each item's SPT is found by a short shared-memory search instead
// of a dependent chain of global loads.
struct SptTile {
    uint32_t off[SB], base[SB], src[SB];
    float x[SB];
    uint32_t count;
};

// last emitted SPT whose first item is <= w (work_off ascends from 0); one warp
__device__ __forceinline__ uint32_t spt_of_item(uint32_t w, uint32_t n_emit, const uint32_t *__restrict__ work_off) {
    return warp_prefix_count(work_off, n_emit, [w](uint32_t o) { return o <= w; }) - 1;
}

__device__ __forceinline__ void stage_tile(SptTile &T, uint32_t q0, uint32_t t_last, uint32_t n_emit,
                                           const uint32_t *__restrict__ work_off, const uint32_t *__restrict__ emit_j,
                                           const float *__restrict__ emit_x, const uint32_t *__restrict__ spt_base,
                                           const uint32_t *__restrict__ emit_src) {
    const uint32_t q = q0 + threadIdx.x;
    const uint32_t wo = q < n_emit ? work_off[q] : 0xffffffffu;
    const int in_tile = q < n_emit && wo <= t_last;            // a prefix of the candidates
    const int count = __syncthreads_count(in_tile);
    if (in_tile) {
        T.off[threadIdx.x] = wo;
        T.base[threadIdx.x] = spt_base[emit_j[q]];
        T.x[threadIdx.x] = emit_x[q];
        if (emit_src) T.src[threadIdx.x] = emit_src[q];
    }
    if (threadIdx.x == 0) T.count = (uint32_t)count;
    __syncthreads();
}

// SPT entry w of the tile: row, slot offset within its SPT, and the interval test lo <= x
__device__ __forceinline__ bool tile_item(const SptTile &T, uint32_t w, const float *__restrict__ lo_row,
                                          uint32_t *row, uint32_t *lq, uint32_t *e) {
    uint32_t a = 0, b = T.count;
    while (b - a > 1) {
        uint32_t m = (a + b) >> 1;
        if (T.off[m] <= w) a = m; else b = m;
    }
    *lq = a;
    *e = w - T.off[a];
    *row = T.base[a] + *e;
    return lo_row[*row] <= T.x[a];
}

__global__ void __launch_bounds__(SB) k_spt_count(const uint32_t *__restrict__ spt_base, const float *__restrict__ lo_row,
                                                  SelBatch B) {
    pdl_wait();
    const SelPtrs &P = B.v[blockIdx.y];
    const uint32_t *__restrict__ cnt_in = P.cnt, *__restrict__ work_off = P.work_off, *__restrict__ emit_j = P.emit_j;
    const float *__restrict__ emit_x = P.emit_x;
    uint32_t *__restrict__ bc = P.bc;
    __shared__ uint32_t s_warp[32];
    __shared__ SptTile T;
    __shared__ uint32_t s_q;
    const uint32_t W = cnt_in[C_WORK], n_emit = cnt_in[C_NEMIT];
    uint32_t begin, end;
    grid_chunk(W, begin, end);
    if (threadIdx.x < 32 && begin < end) {
        const uint32_t q = spt_of_item(begin, n_emit, work_off);
        if (threadIdx.x == 0) s_q = q;
    }
    __syncthreads();
    uint32_t c = 0;
    for (uint32_t t0 = begin; t0 < end; t0 += SB) {
        const uint32_t t_last = min(t0 + SB, end) - 1;
        const uint32_t q0 = s_q;
        stage_tile(T, q0, t_last, n_emit, work_off, emit_j, emit_x, spt_base, nullptr);
        const uint32_t w = t0 + threadIdx.x;
        uint32_t row, lq, e;
        if (w <= t_last && tile_item(T, w, lo_row, &row, &lq, &e)) ++c;
        __syncthreads();
        if (threadIdx.x == 0) s_q = q0 + T.count - 1;           // the next tile starts in the last SPT or later
        __syncthreads();
    }
    uint32_t tot;
    block_scan(c, s_warp, &tot);
    if (threadIdx.x == 0) bc[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SB) k_spt_write(const uint32_t *__restrict__ spt_base, const float *__restrict__ lo_row,
                                                  SelBatch B) {
    pdl_wait();
    const SelPtrs &P = B.v[blockIdx.y];
    uint32_t *__restrict__ cnt = P.cnt;
    const uint32_t *__restrict__ work_off = P.work_off, *__restrict__ emit_j = P.emit_j, *__restrict__ bc = P.bc;
    const float *__restrict__ emit_x = P.emit_x;
    uint32_t *__restrict__ sel_rows = P.sel_rows, *__restrict__ sel_src = P.sel_src;
    const uint32_t *__restrict__ emit_src = P.emit_src;
    __shared__ uint32_t s_warp[32];
    __shared__ SptTile T;
    __shared__ uint32_t s_off, s_q;
    uint32_t W = cnt[C_WORK], n_emit = cnt[C_NEMIT], n_up = cnt[C_NUP];
    uint32_t before = block_prefix(bc, s_warp);
    uint32_t begin, end;
    grid_chunk(W, begin, end);
    if (threadIdx.x < 32) {
        const uint32_t q = begin < end ? spt_of_item(begin, n_emit, work_off) : 0u;
        if (threadIdx.x == 0) { s_off = n_up + before; s_q = q; }
    }
    __syncthreads();
    for (uint32_t t0 = begin; t0 < end; t0 += SB) {
        const uint32_t t_last = min(t0 + SB, end) - 1;
        const uint32_t q0 = s_q;
        stage_tile(T, q0, t_last, n_emit, work_off, emit_j, emit_x, spt_base, emit_src);
        const uint32_t w = t0 + threadIdx.x;
        uint32_t row = 0, lq = 0, e = 0;
        const bool keep = w <= t_last && tile_item(T, w, lo_row, &row, &lq, &e);
        uint32_t tot;
        uint32_t ex = block_scan(keep ? 1u : 0u, s_warp, &tot);
        uint32_t o = s_off;
        if (keep) {
            sel_rows[o + ex] = row;
            if (sel_src) sel_src[o + ex] = T.src[lq] + e;      // record slot of entry e of this SPT
        }
        __syncthreads();
        if (threadIdx.x == 0) { s_off = o + tot; s_q = q0 + T.count - 1; }
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        cnt[C_NSEL] = s_off;
        cnt[C_NSPTSEL] = s_off - n_up;
    }
}

__global__ void k_set_view(View v, View *__restrict__ dst, uint32_t *__restrict__ cnt) {
    pdl_wait();
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&v);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t i = threadIdx.x; i < sizeof(View) / 4; i += blockDim.x) d[i] = s[i];
    if (cnt)                                      // and clear the frame's counters (a new selection)
        for (uint32_t i = threadIdx.x; i < C_COUNT; i += blockDim.x) cnt[i] = 0u;
}

// k views at once: block b uploads view b and clears its frame's counters
struct ViewBatch {
    View v[SEL_BATCH_MAX];
    View *dst[SEL_BATCH_MAX];
    uint32_t *cnt[SEL_BATCH_MAX];
};
__global__ void k_set_views(ViewBatch b) {
    pdl_wait();
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&b.v[blockIdx.x]);
    uint32_t *d = reinterpret_cast<uint32_t *>(b.dst[blockIdx.x]);
    for (uint32_t i = threadIdx.x; i < sizeof(View) / 4; i += blockDim.x) d[i] = s[i];
    for (uint32_t i = threadIdx.x; i < C_COUNT; i += blockDim.x) b.cnt[blockIdx.x][i] = 0u;
}

SelPtrs sel_ptrs(FrameBufs &f, bool with_src) {
    SelPtrs p{};
    p.view = f.d_view;
    p.cnt = f.cnt;
    p.bc = f.block_counts;
    p.sel_rows = f.sel_rows;
    p.sel_src = with_src ? f.sel_src : nullptr;
    p.emit_j = f.emit_j;
    p.high = f.high;
    p.work_off = f.work_off;
    p.scan_bsum = f.scan_bsum;
    p.emit_x = f.emit_x;
    p.up_x = f.up_x;
    p.up_out = f.up_out;
    p.emit_src = with_src ? f.emit_src : nullptr;
    return p;
}

// the passes of Algorithms 1-2 for views[0, k) of a batch (the count pass
// keeps each upper entry's outcome for the write pass)
int launch_upper(const lodgs_scene *sc, const SelBatch &b, int k, cudaStream_t st) {
    const uint32_t U = (uint32_t)sc->n_upper;
    LODGS_CUDA(pdl_launch(k_upper_count, dim3(SEL_GRID, k), SB, st, sc->d_upper, U, b));
    count_launches(1);
    LODGS_CUDA(pdl_launch(k_upper_write, dim3(SEL_GRID, k), SB, st, sc->d_upper, U, b));
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

int launch_high(const lodgs_scene *sc, const SelBatch &b, int k, cudaStream_t st) {
    const unsigned hb = (unsigned)std::min<int64_t>(SPT_GRID, std::max<int64_t>(1, (sc->n_spt + SB / 32 - 1) / (SB / 32)));
    LODGS_CUDA(pdl_launch(k_spt_high, dim3(hb, k), SB, st, sc->d_spt_base, sc->d_hi, b));
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

int launch_spt(const lodgs_scene *sc, const SelBatch &b, int k, cudaStream_t st) {
    ScanBatch s{};
    for (int v = 0; v < k; ++v) {
        s.in[v] = b.v[v].high;
        s.out[v] = b.v[v].work_off;
        s.d_n[v] = b.v[v].cnt + C_NEMIT;
        s.block_sums[v] = b.v[v].scan_bsum;
        s.d_total[v] = b.v[v].cnt + C_WORK;
    }
    if (int rc = scan_exclusive_batch(s, k, (uint32_t)sc->n_spt, st)) return rc;
    LODGS_CUDA(pdl_launch(k_spt_count, dim3(SPT_GRID, k), SB, st, sc->d_spt_base, sc->d_lo, b));
    count_launches(1);
    LODGS_CUDA(pdl_launch(k_spt_write, dim3(SPT_GRID, k), SB, st, sc->d_spt_base, sc->d_lo, b));
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

}  // namespace

// The view goes to the device as a kernel argument: the copy is asynchronous,
// needs no host staging buffer, and is ordered on the stream like the kernels.
int launch_set_view(const View &v, View *dst, cudaStream_t st, uint32_t *zero_cnt) {
    LODGS_CUDA(pdl_launch(k_set_view, 1, 32, st, v, dst, zero_cnt));
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

int launch_select_upper(const lodgs_scene *sc, FrameBufs &f, bool with_src, cudaStream_t st) {
    SelBatch b{};
    b.v[0] = sel_ptrs(f, with_src);
    return launch_upper(sc, b, 1, st);
}

int launch_spt_high(const lodgs_scene *sc, FrameBufs &f, cudaStream_t st) {
    SelBatch b{};
    b.v[0] = sel_ptrs(f, false);
    return launch_high(sc, b, 1, st);
}

int launch_select_spt(const lodgs_scene *sc, FrameBufs &f, bool with_src, cudaStream_t st) {
    SelBatch b{};
    b.v[0] = sel_ptrs(f, with_src);
    return launch_spt(sc, b, 1, st);
}

int launch_select(const lodgs_scene *sc, FrameBufs &f, cudaStream_t st) {
    FrameBufs *fs[1] = {&f};
    return launch_select_batch(sc, fs, nullptr, 1, st);
}

// views[v] (if given) is uploaded to frame v and its counters cleared first
int launch_select_batch(const lodgs_scene *sc, FrameBufs *const *fs, const View *views, int k, cudaStream_t st) {
    if (k < 1 || k > SEL_BATCH_MAX) { set_error("select: batch size out of range"); return LODGS_E_INVALID; }
    if (views) {
        ViewBatch vb{};
        for (int v = 0; v < k; ++v) { vb.v[v] = views[v]; vb.dst[v] = fs[v]->d_view; vb.cnt[v] = fs[v]->cnt; }
        LODGS_CUDA(pdl_launch(k_set_views, k, 32, st, vb));
        count_launches(1);
    }
    SelBatch b{};
    for (int v = 0; v < k; ++v) b.v[v] = sel_ptrs(*fs[v], false);
    int rc = launch_upper(sc, b, k, st);
    if (!rc) rc = launch_high(sc, b, k, st);
    if (!rc) rc = launch_spt(sc, b, k, st);
    return rc;
}

}  // namespace lodgs
