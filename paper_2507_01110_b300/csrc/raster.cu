// a5-a8: tile x depth ordering and per-tile front-to-back compositing (Eq. 1-2)
// with its backward.
//
// Ordering is done per tile: the (Gaussian, tile) pairs of the selection's tile
// rectangles are enumerated flat, the tile support test drops pairs whose tile
// the ellipse cannot reach, the kept pairs are counted per tile, the counts are
// scanned into tile ranges, the pairs are scattered into their tiles, and one
// block per tile sorts its short list by (depth key, selected index).  The
// result is the (tile, depth, index) order of a full-key sort, in six launches
// instead of a global multi-pass radix sort.  Frames dense enough to have long
// tile lists (a pair workspace of more than 1024 pairs per tile on average)
// take the global route instead: the selected Gaussians are stably sorted by
// depth key, the pairs are emitted in that order, and a stable radix sort on the
// tile id groups them by tile -- the same order.
//
// Blending runs one 128-thread CTA per 16x16 tile; batches of the tile's
// Gaussians are staged in shared memory.  Eq. 1 is truncated once a pixel's
// transmittance falls below 1e-4 (the Gaussian that crosses the bound is still
// blended), so the neglected tail is at most 1e-4 of the colour.  The support test p >= -4.5 uses
// explicitly rounded float32 operations (it decides which pixels a Gaussian
// touches); the alpha, transmittance and colour arithmetic are ordinary fp32.
// The backward walks each tile's list front to back like the forward,
// recomputing transmittance per tile (nothing per pixel is stored), and takes
// the colour behind each Gaussian from the forward's output image.  Within a
// tile each warp owns an 8x8 pixel block and skips the Gaussians whose support
// box misses it (block test, conservative like the tile test).
#include "lodgs_internal.cuh"

namespace lodgs {
namespace {

constexpr int RB = 256;
constexpr int RGRID = 148 * 8;
// Blocks of the pair enumeration kernels: 16 per SM, more than are resident at
// once (six); one resident wave measured slower (pair counting 0.0376 ->
// 0.0408 ms on a 1080p view).
#ifndef LODGS_EMIT_GRID
#define LODGS_EMIT_GRID (148 * 16)
#endif
constexpr int EGRID = LODGS_EMIT_GRID;

// Tile support test (float32, explicitly rounded).  The support exponent is a
// concave quadratic; its maximum over the rectangle of the tile's pixel centres
// is 0 when the mean lies inside, otherwise it lies on an edge at the clamped
// 1-D maximum.  The pair is kept iff that maximum is >= -4.5 - 0.01, a
// conservative margin: a dropped pair has no pixel passing the support test, so
// the image is unchanged while the blend skips tiles the ellipse never reaches.
__device__ __forceinline__ float edge_p(float A, float B, float C, float dx, float dy) {
    const float s = __fadd_rn(__fmul_rn(__fmul_rn(A, dx), dx), __fmul_rn(__fmul_rn(C, dy), dy));
    return __fsub_rn(__fmul_rn(-0.5f, s), __fmul_rn(__fmul_rn(B, dx), dy));
}

__device__ __forceinline__ bool tile_keep(float u, float v, float A, float B, float C, uint32_t tx, uint32_t ty) {
    const float X0 = __fadd_rn((float)(TILE * tx), 0.5f), X1 = __fadd_rn(X0, 15.0f);
    const float Y0 = __fadd_rn((float)(TILE * ty), 0.5f), Y1 = __fadd_rn(Y0, 15.0f);
    if (u >= X0 && u <= X1 && v >= Y0 && v <= Y1) return true;
    float best = -INFINITY;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float xe = k ? X1 : X0, ye = k ? Y1 : Y0;
        const float dx = __fsub_rn(u, xe);
        const float y = fminf(fmaxf(__fadd_rn(v, __fdiv_rn(__fmul_rn(B, dx), C)), Y0), Y1);
        best = fmaxf(best, edge_p(A, B, C, dx, __fsub_rn(v, y)));
        const float dy = __fsub_rn(v, ye);
        const float x = fminf(fmaxf(__fadd_rn(u, __fdiv_rn(__fmul_rn(B, dy), A)), X0), X1);
        best = fmaxf(best, edge_p(A, B, C, __fsub_rn(u, x), dy));
    }
    return best >= -4.51f;
}

// The contiguous run [g0, g1) of 32-pair groups of this warp, out of P pairs
// split evenly over the grid's warps.
__device__ __forceinline__ void warp_groups(uint32_t P, uint32_t &g0, uint32_t &g1) {
    const uint32_t warps = gridDim.x * (blockDim.x >> 5), w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t groups = (P + 31u) / 32u, per = (groups + warps - 1u) / warps;
    const uint64_t b = (uint64_t)w * per, e = b + per;
    g0 = b < groups ? (uint32_t)b : groups;
    g1 = e < groups ? (uint32_t)e : groups;
}

// Owner of pair p = p0 + lane for a warp's 32 consecutive pair indices: the
// largest selected index g with pair_off[g] <= p (pair_off is the exclusive
// scan of the rectangle areas, pair_off[n] = P implied).  One 32-ary search for
// p0 (each round all lanes probe, about 33x narrower per round), then each lane
// searches the 32 offsets from that Gaussian on by shuffles; a lane past them
// (empty rectangles in between) finishes with its own binary search.  Every
// lane of the warp must call this.
__device__ __forceinline__ uint32_t warp_pair_owner(uint32_t p0, uint32_t p, uint32_t n,
                                                    const uint32_t *__restrict__ pair_off, int lane,
                                                    uint32_t hint = 0) {
    // hint: the owner of a pair at or before p0 (0 always qualifies).  When the
    // 32 offsets from it reach past p0, one coalesced load finds p0's owner.
    uint32_t a = hint, b = n;                    // pair_off[a] <= p0 < pair_off[b]
    if (hint > 0) {
        const uint32_t v = hint + lane < n ? pair_off[hint + lane] : 0xffffffffu;
        const uint32_t bal = __ballot_sync(0xffffffffu, v <= p0);
        if (!(bal >> 31 & 1u)) b = hint + (uint32_t)__popc(bal);   // p0's owner is within the window
        else a = hint + 31;
    }
    while (b - a > 32) {
        const uint32_t m = a + (uint32_t)(((uint64_t)(b - a) * (uint32_t)(lane + 1)) / 33u);   // a < m < b
        const uint32_t c = __popc(__ballot_sync(0xffffffffu, pair_off[m] <= p0));
        const uint32_t ma = __shfl_sync(0xffffffffu, m, c > 0 ? (int)c - 1 : 0);
        const uint32_t mb = __shfl_sync(0xffffffffu, m, c < 32 ? (int)c : 31);
        if (c > 0) a = ma;
        if (c < 32) b = mb;
    }
    {
        const uint32_t v = a + lane < b ? pair_off[a + lane] : 0xffffffffu;
        a += __popc(__ballot_sync(0xffffffffu, v <= p0)) - 1;      // pair_off[a] <= p0 holds: >= 1 lane
    }
    const uint32_t w = a + lane < n ? pair_off[a + lane] : 0xffffffffu;
    uint32_t idx = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) {
        const uint32_t v = __shfl_sync(0xffffffffu, w, (int)idx + st);
        if (v <= p) idx += st;
    }
    uint32_t g = a + idx;
    if (idx == 31) {                             // the window may not reach p: finish alone
        uint32_t lo = g, hi = n;
        while (hi - lo > 1) {
            const uint32_t m = (lo + hi) >> 1;
            if (pair_off[m] <= p) lo = m; else hi = m;
        }
        g = lo;
    }
    return g;
}

// ---- global ordering (large frames): depth sort, emission, tile sort ----
// One thread per rectangle pair: pair p belongs to the last depth rank r with
// pair_off[r] <= p (found per warp, warp_pair_owner) and is the k-th tile of
// its rectangle in row-major order.  Pairs whose tile the support ellipse cannot reach get the
// key n_tiles, which the tile sort moves behind every real tile.
__global__ void k_emit(const uint32_t *__restrict__ order, const uint2 *__restrict__ rect,
                       const float4 *__restrict__ sp_a, const float4 *__restrict__ sp_b,
                       const uint32_t *__restrict__ pair_off, uint32_t *__restrict__ cnt, uint64_t cap_pairs,
                       int TX, uint32_t n_tiles, uint32_t *__restrict__ pkey, uint32_t *__restrict__ pval) {
    pdl_wait();
    // pairs beyond the workspace (or an earlier overflow) are not emitted: capacity error
    uint32_t P = cnt[C_NPAIR];
    const bool over = P > cap_pairs || (cnt[C_STATUS] & ST_CAPACITY) ||
                      *reinterpret_cast<const unsigned long long *>(cnt + C_NPAIR64) > 0xffffffffull;
    if (over) P = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        cnt[C_NPAIR_EFF] = P;
        cnt[C_NKEPT_WANT] = cnt[C_NPAIR];           // all rectangle pairs are stored on this path
        if (over) atomicOr(&cnt[C_STATUS], ST_CAPACITY);
    }
    const uint32_t n = cnt[C_NSEL_EFF];
    const int lane = threadIdx.x & 31;
    // each warp takes a contiguous run of 32-pair groups, carrying the owner
    // of its last pair into the next group's search
    uint32_t g0, g1, hint = 0;
    warp_groups(P, g0, g1);
    for (uint32_t gi = g0; gi < g1; ++gi) {
        const uint32_t p0 = gi * 32u, p = p0 + lane;
        const uint32_t a = warp_pair_owner(p0, p, n, pair_off, lane, hint);
        hint = __shfl_sync(0xffffffffu, a, 31);
        if (p >= P) continue;
        const uint32_t g = order[a];
        const uint2 rc = rect[g];
        const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu;
        const uint32_t w = x1 - x0, k = p - pair_off[a];
        const uint32_t ty = y0 + k / w, tx = x0 + k % w;
        const float4 sa = sp_a[g];
        const float nhc = sp_b[g].x;
        const bool keep = tile_keep(sa.x, sa.y, -2.0f * sa.z, -sa.w, -2.0f * nhc, tx, ty);
        pkey[p] = keep ? ty * (uint32_t)TX + tx : n_tiles;
        pval[p] = g;
    }
}

__global__ void k_ranges(const uint32_t *__restrict__ pkey, uint32_t *__restrict__ cnt, uint32_t n_tiles,
                         uint2 *__restrict__ ranges) {
    pdl_wait();
    uint32_t n = cnt[C_NPAIR_EFF];
    for (uint32_t p = blockIdx.x * RB + threadIdx.x; p < n; p += gridDim.x * RB) {
        uint32_t t = pkey[p];
        if (t >= n_tiles) continue;                       // dropped pairs sort behind every tile
        if (p == 0 || pkey[p - 1] != t) ranges[t].x = p;
        if (p + 1 == n || pkey[p + 1] != t) {
            ranges[t].y = p + 1;
            if (p + 1 == n || pkey[p + 1] >= n_tiles) cnt[C_NKEPT] = p + 1;
        }
    }
}

// ---- per-tile ordering ----
// Rectangle pairs are enumerated flat: pair p belongs to the last selected
// Gaussian g with pair_off[g] <= p (binary search over the scan of the
// rectangle areas, selection order) and is the k-th tile of its rectangle in
// row-major order.  Returns the tile of the pair, or -1 when the tile support
// test drops it.
// Tile of pair p of Gaussian g (row-major in its rectangle), whatever the
// support test says.
__device__ __forceinline__ int64_t pair_tile_any(uint32_t p, uint32_t g, const uint32_t *__restrict__ pair_off,
                                                 const uint2 *__restrict__ rect, int TX) {
    const uint2 rc = rect[g];
    const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu;
    const uint32_t w = x1 - x0, k = p - pair_off[g];
    return (int64_t)(y0 + k / w) * TX + (x0 + k % w);
}

// Tile of pair p of Gaussian g (row-major in its rectangle), or -1 when the
// tile support test drops it.
__device__ __forceinline__ int64_t pair_tile(uint32_t p, uint32_t g, const uint32_t *__restrict__ pair_off,
                                             const uint2 *__restrict__ rect, const float4 *__restrict__ sp_a,
                                             const float4 *__restrict__ sp_b, int TX) {
    const uint2 rc = rect[g];
    const uint32_t x0 = rc.x & 0xffffu, y0 = rc.x >> 16, x1 = rc.y & 0xffffu;
    const uint32_t w = x1 - x0, k = p - pair_off[g];
    const uint32_t ty = y0 + k / w, tx = x0 + k % w;
    const float4 sa = sp_a[g];
    const float nhc = sp_b[g].x;
    if (!tile_keep(sa.x, sa.y, -2.0f * sa.z, -sa.w, -2.0f * nhc, tx, ty)) return -1;
    return (int64_t)ty * TX + tx;
}

// Count the kept pairs of every tile (one atomic per group of equal tiles in a
// warp) and record each 32-pair group's kept lanes as a bit mask (keep[gi],
// for the groups below keep_cap), so that the scatter neither repeats the
// support test nor visits groups with nothing kept.
__global__ void __launch_bounds__(RB) k_emit_count(const uint32_t *__restrict__ pair_off,
                                                   const uint2 *__restrict__ rect, const float4 *__restrict__ sp_a,
                                                   const float4 *__restrict__ sp_b, uint32_t *__restrict__ cnt,
                                                   int TX, uint32_t *__restrict__ tile_cnt, uint32_t *__restrict__ keep,
                                                   uint32_t keep_cap) {
    pdl_wait();
    if (cnt[C_STATUS] & ST_CAPACITY) return;
    if (*reinterpret_cast<const unsigned long long *>(cnt + C_NPAIR64) > 0xffffffffull) {   // 32-bit pair indices
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr((uint32_t *)&cnt[C_STATUS], ST_CAPACITY);
        return;
    }
    const uint32_t P = cnt[C_NPAIR], n = cnt[C_NSEL_EFF];
    const int lane = threadIdx.x & 31;
    // whole warps step together so that the match below sees every lane; each
    // warp takes a contiguous run of 32-pair groups (owner search carried over)
    uint32_t g0, g1, hint = 0;
    warp_groups(P, g0, g1);
    for (uint32_t gi = g0; gi < g1; ++gi) {
        const uint32_t p0 = gi * 32u, p = p0 + lane;
        const uint32_t g = warp_pair_owner(p0, p, n, pair_off, lane, hint);
        hint = __shfl_sync(0xffffffffu, g, 31);
        const int64_t t = p < P ? pair_tile(p, g, pair_off, rect, sp_a, sp_b, TX) : -1;
        const uint32_t kept = __ballot_sync(0xffffffffu, t >= 0);
        if (lane == 0 && gi < keep_cap) keep[gi] = kept;
        const uint32_t key = t < 0 ? 0xffffffffu : (uint32_t)t;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        if (t >= 0 && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&tile_cnt[t], (uint32_t)__popc(peers));
    }
}

// Longest-first tile order for the blends.  Blocks are handed to SMs in index
// order as slots free up (greedy list scheduling); in raster order a few long
// tiles that start late keep some SMs busy while the rest idle.  Tiles are
// bucketed by pair count on a log scale (two buckets per power of two) and
// listed largest bucket first; the order within a bucket is arbitrary, as a
// tile's result does not depend on which block computes it.  One block; each
// pass loads TOR_K chunks of counts at once.
constexpr int TOR_THREADS = 1024, TOR_K = 8, TOR_BUCKETS = 64;
__device__ __forceinline__ uint32_t order_bucket(uint32_t n) {
    uint32_t key = n;                                          // 0, 1
    if (n >= 2) {
        const uint32_t l = 31 - __clz(n);                      // 1..31
        key = 2 * l + ((n >> (l - 1)) & 1u);                   // 2..63
    }
    return (TOR_BUCKETS - 1) - key;                            // largest counts first
}

// The order itself, computed by the calling block (TOR_THREADS threads, which
// must see the ranges: written before a barrier, or by an earlier kernel).
__device__ __forceinline__ void block_tile_order(const uint2 *ranges, uint32_t n_tiles,   // no __restrict__:
                                                 uint32_t *__restrict__ order, uint32_t *s_h) {  // written in-kernel
    const int tid = threadIdx.x;
    if (tid < TOR_BUCKETS) s_h[tid] = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n_tiles; base += TOR_K * TOR_THREADS) {
        uint2 r[TOR_K];
#pragma unroll
        for (int i = 0; i < TOR_K; ++i) {
            const uint32_t t = base + i * TOR_THREADS + tid;
            r[i] = t < n_tiles ? ranges[t] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int i = 0; i < TOR_K; ++i)
            if (base + i * TOR_THREADS + tid < n_tiles) atomicAdd(&s_h[order_bucket(r[i].y - r[i].x)], 1u);
    }
    __syncthreads();
    if (tid < 32) {                                            // exclusive scan of the 64 buckets
        const uint32_t a = s_h[2 * tid], b = s_h[2 * tid + 1];
        uint32_t x = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (tid >= o) x += y;
        }
        const uint32_t ex = x - (a + b);
        s_h[2 * tid] = ex;
        s_h[2 * tid + 1] = ex + a;
    }
    __syncthreads();
    for (uint32_t base = 0; base < n_tiles; base += TOR_K * TOR_THREADS) {
        uint2 r[TOR_K];
#pragma unroll
        for (int i = 0; i < TOR_K; ++i) {
            const uint32_t t = base + i * TOR_THREADS + tid;
            r[i] = t < n_tiles ? ranges[t] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int i = 0; i < TOR_K; ++i) {
            const uint32_t t = base + i * TOR_THREADS + tid;
            if (t < n_tiles) order[atomicAdd(&s_h[order_bucket(r[i].y - r[i].x)], 1u)] = t;
        }
    }
}

__global__ void __launch_bounds__(TOR_THREADS) k_tile_order(const uint2 *__restrict__ ranges, uint32_t n_tiles,
                                                            uint32_t *__restrict__ order) {
    pdl_wait();
    __shared__ uint32_t s_h[TOR_BUCKETS];
    block_tile_order(ranges, n_tiles, order, s_h);
}

// One block: exclusive scan of the tile counts.  Writes the tile ranges, turns
// the counts into scatter cursors (the tile's first slot) and records the kept
// pair total, flagging a capacity error when it exceeds the pair buffers.
// Each pass loads TO_K chunks of TO_THREADS consecutive counts at once (one
// load latency per pass instead of one per chunk), scans each chunk within
// its warps, scans the warp totals of every chunk in one warp per chunk, and
// adds the chunks' totals in order.
constexpr int TO_THREADS = 1024;
static_assert(TO_THREADS == TOR_THREADS, "the offsets block also computes the tile order");
constexpr int TO_K = 8;
__global__ void __launch_bounds__(TO_THREADS) k_tile_offsets(uint32_t *__restrict__ tile_cnt, uint32_t n_tiles,
                                                             uint64_t cap_pairs, uint32_t *__restrict__ cnt,
                                                             uint2 *__restrict__ ranges,
                                                             uint32_t *__restrict__ tile_order) {
    pdl_wait();
    constexpr int NWT = TO_THREADS / 32;
    static_assert(TO_K <= NWT, "one warp scans each chunk's warp totals");
    __shared__ uint32_t s_warp[TO_K][NWT];
    __shared__ unsigned long long s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    for (uint32_t base = 0; base < n_tiles; base += TO_K * TO_THREADS) {
        uint32_t v[TO_K], x[TO_K];
#pragma unroll
        for (int i = 0; i < TO_K; ++i) {
            const uint32_t t = base + i * TO_THREADS + tid;
            v[i] = t < n_tiles ? tile_cnt[t] : 0u;
        }
#pragma unroll
        for (int i = 0; i < TO_K; ++i) {
            x[i] = v[i];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x[i], o);
                if (lane >= o) x[i] += y;
            }
            if (lane == 31) s_warp[i][warp] = x[i];
        }
        __syncthreads();
        if (warp < TO_K) {
            uint32_t w = s_warp[warp][lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_warp[warp][lane] = w;
        }
        __syncthreads();
        unsigned long long chunk = s_carry;
#pragma unroll
        for (int i = 0; i < TO_K; ++i) {
            const uint32_t t = base + i * TO_THREADS + tid;
            const unsigned long long off = chunk + (warp ? s_warp[i][warp - 1] : 0u) + x[i] - v[i];
            if (t < n_tiles) {
                const uint32_t o32 = off > 0xffffffffull ? 0xffffffffu : (uint32_t)off;
                ranges[t] = make_uint2(o32, o32 + v[i]);
                tile_cnt[t] = o32;
            }
            chunk += s_warp[i][NWT - 1];
        }
        __syncthreads();
        if (tid == 0) s_carry = chunk;
        __syncthreads();
    }
    if (tid == 0) {
        const unsigned long long total = s_carry;
        cnt[C_NKEPT_WANT] = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
        if (total > cap_pairs) {                     // kept pairs beyond the workspace: capacity error
            atomicOr(&cnt[C_STATUS], ST_CAPACITY);
            cnt[C_NKEPT] = 0;
        } else {
            cnt[C_NKEPT] = (uint32_t)total;
        }
    }
    __shared__ uint32_t s_h[TOR_BUCKETS];
    block_tile_order(ranges, n_tiles, tile_order, s_h);      // this block's range writes precede its barriers
}

// Scatter the kept pairs into their tiles' slots (in any order within a tile:
// the per-tile sort fixes it): depth key and selected index.
__global__ void __launch_bounds__(RB) k_emit_scatter(const uint32_t *__restrict__ pair_off,
                                                     const uint2 *__restrict__ rect, const float4 *__restrict__ sp_a,
                                                     const float4 *__restrict__ sp_b,
                                                     const uint32_t *__restrict__ dkey, const uint32_t *__restrict__ cnt,
                                                     int TX, uint32_t *__restrict__ cursor, uint32_t *__restrict__ pkey,
                                                     uint32_t *__restrict__ pval, const uint32_t *__restrict__ keep,
                                                     uint32_t keep_cap) {
    pdl_wait();
    if (cnt[C_STATUS] & ST_CAPACITY) return;
    const uint32_t P = cnt[C_NPAIR], n = cnt[C_NSEL_EFF];
    const int lane = threadIdx.x & 31;
    uint32_t g0, g1, hint = 0;
    warp_groups(P, g0, g1);
    for (uint32_t gi = g0; gi < g1; ++gi) {
        const bool known = gi < keep_cap;               // the count pass recorded this group's kept lanes
        const uint32_t kept = known ? keep[gi] : 0xffffffffu;
        if (kept == 0u) continue;                       // warp-uniform; the carried hint stays a lower bound
        const uint32_t p0 = gi * 32u, p = p0 + lane;
        const uint32_t g = warp_pair_owner(p0, p, n, pair_off, lane, hint);
        hint = __shfl_sync(0xffffffffu, g, 31);
        int64_t t = -1;
        if (p < P && (kept >> lane & 1u))
            t = known ? pair_tile_any(p, g, pair_off, rect, TX) : pair_tile(p, g, pair_off, rect, sp_a, sp_b, TX);
        const uint32_t key = t < 0 ? 0xffffffffu : (uint32_t)t;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        uint32_t slot = 0;
        if (t >= 0 && lane == leader) slot = atomicAdd(&cursor[t], (uint32_t)__popc(peers));
        slot = __shfl_sync(0xffffffffu, slot, leader) + __popc(peers & ((1u << lane) - 1u));
        if (t >= 0) {
            pkey[slot] = dkey[g];
            pval[slot] = g;
        }
    }
}

// One block per tile: sort the tile's pairs by (depth key, selected index) --
// the order of the (tile, depth, index) sort -- and leave the indices in pval.
// Up to TS_RANK pairs: rank by counting (one pass, no barriers); up to TS_SMEM:
// a bitonic network in shared memory, whose comparators always put the
// smaller key at the lower index (a flip stage, then half-cleaners), so
// positions past the list end act as +infinity and need no storage.  Longer
// lists: TS_SMEM-sized chunks sorted that way, then merged pairwise (each merge
// split evenly over the block's threads along its merge path), alternating
// between the pair arrays and a 64-bit scratch array.  The block also clears
// the tile's counter for the next render.
constexpr int TS_THREADS = 256, TS_RANK = 256, TS_SMEM = 2048;

// a tile's keys, held either as 64-bit words or split over the pair arrays
struct TileKeys {
    uint32_t *K, *V;                  // split: depth key (high word), selected index (low word)
    unsigned long long *S;            // or whole keys
    __device__ __forceinline__ unsigned long long get(uint32_t i) const {
        return S ? S[i] : ((unsigned long long)K[i] << 32 | V[i]);
    }
    __device__ __forceinline__ void put(uint32_t i, unsigned long long v) const {
        if (S) S[i] = v;
        else { K[i] = (uint32_t)(v >> 32); V[i] = (uint32_t)v; }
    }
};

template <typename Load, typename Store>
__device__ __forceinline__ void bitonic_sort(uint32_t L, Load load, Store store) {
    uint32_t N = 1;
    while (N < L) N <<= 1;
    for (uint32_t k = 2; k <= N; k <<= 1) {
        for (uint32_t c = threadIdx.x; c < N / 2; c += TS_THREADS) {      // flip: i against its mirror in the block
            const uint32_t h = k >> 1, i = (c / h) * k + (c % h), j = (c / h) * k + (k - 1 - (c % h));
            if (j < L) {
                const unsigned long long a = load(i), b = load(j);
                if (a > b) { store(i, b); store(j, a); }
            }
        }
        __syncthreads();
        for (uint32_t st = k >> 2; st >= 1; st >>= 1) {                    // half-cleaners
            for (uint32_t c = threadIdx.x; c < N / 2; c += TS_THREADS) {
                const uint32_t i = (c / st) * 2 * st + (c % st), j = i + st;
                if (j < L) {
                    const unsigned long long a = load(i), b = load(j);
                    if (a > b) { store(i, b); store(j, a); }
                }
            }
            __syncthreads();
        }
    }
}

// Merge the sorted runs src[a0, a1) and src[a1, a2) into dst[a0, a2) with the
// whole block: thread t writes outputs [t n / T, (t + 1) n / T) after locating
// its start on the merge path by binary search (keys are distinct).
__device__ void merge_runs(const TileKeys &src, const TileKeys &dst, uint32_t a0, uint32_t a1, uint32_t a2) {
    const uint32_t na = a1 - a0, nb = a2 - a1, n = na + nb;
    const uint32_t d0 = (uint32_t)((uint64_t)n * threadIdx.x / TS_THREADS);
    const uint32_t d1 = (uint32_t)((uint64_t)n * (threadIdx.x + 1) / TS_THREADS);
    if (d0 == d1) return;
    // i = number of A elements among the first d0 outputs
    uint32_t lo = d0 > nb ? d0 - nb : 0, hi = d0 < na ? d0 : na;
    while (lo < hi) {
        const uint32_t i = (lo + hi) >> 1;                      // is A[i] before B[d0 - i - 1]?
        if (src.get(a0 + i) < src.get(a1 + d0 - i - 1)) lo = i + 1; else hi = i;
    }
    uint32_t i = lo, j = d0 - lo;
    for (uint32_t d = d0; d < d1; ++d) {
        const bool takeA = j >= nb || (i < na && src.get(a0 + i) < src.get(a1 + j));
        dst.put(a0 + d, takeA ? src.get(a0 + i++) : src.get(a1 + j++));
    }
}

__global__ void __launch_bounds__(TS_THREADS) k_tile_sort(const uint2 *__restrict__ ranges,
                                                          uint32_t *__restrict__ tile_cnt,
                                                          const uint32_t *__restrict__ cnt, uint32_t *pkey,
                                                          uint32_t *pval, unsigned long long *scratch,
                                                          const uint32_t *__restrict__ tile_order) {
    pdl_wait();
    __shared__ unsigned long long s_k[TS_SMEM];
    const uint32_t t = tile_order[blockIdx.x];
    if (threadIdx.x == 0) tile_cnt[t] = 0;               // counters start at zero for the next render
    if (cnt[C_STATUS] & ST_CAPACITY) return;
    const uint2 rg = ranges[t];
    const uint32_t L = rg.y - rg.x;
    if (L <= 1) return;
    uint32_t *K = pkey + rg.x, *V = pval + rg.x;
    const TileKeys split{K, V, nullptr}, whole{nullptr, nullptr, scratch + rg.x};
    if (L <= TS_SMEM) {
        for (uint32_t i = threadIdx.x; i < L; i += TS_THREADS) s_k[i] = split.get(i);
        __syncthreads();
        if (L <= TS_RANK) {                              // keys are distinct (indices are)
            if (threadIdx.x < L) {
                const unsigned long long me = s_k[threadIdx.x];
                uint32_t r = 0;
                for (uint32_t j = 0; j < L; ++j) r += s_k[j] < me;
                V[r] = (uint32_t)me;
            }
            return;
        }
        bitonic_sort(L, [&](uint32_t i) { return s_k[i]; },
                     [&](uint32_t i, unsigned long long v) { s_k[i] = v; });
        for (uint32_t i = threadIdx.x; i < L; i += TS_THREADS) V[i] = (uint32_t)s_k[i];
        return;
    }
    // long list: sorted chunks into the scratch array, then merge passes
    for (uint32_t c0 = 0; c0 < L; c0 += TS_SMEM) {
        const uint32_t Lc = min((uint32_t)TS_SMEM, L - c0);
        for (uint32_t i = threadIdx.x; i < Lc; i += TS_THREADS) s_k[i] = split.get(c0 + i);
        __syncthreads();
        bitonic_sort(Lc, [&](uint32_t i) { return s_k[i]; },
                     [&](uint32_t i, unsigned long long v) { s_k[i] = v; });
        for (uint32_t i = threadIdx.x; i < Lc; i += TS_THREADS) whole.put(c0 + i, s_k[i]);
        __syncthreads();
    }
    bool in_whole = true;
    for (uint32_t w = TS_SMEM; w < L; w <<= 1) {
        const TileKeys &src = in_whole ? whole : split, &dst = in_whole ? split : whole;
        for (uint32_t a0 = 0; a0 < L; a0 += 2 * w) {
            const uint32_t a1 = min(a0 + w, L), a2 = min(a0 + 2 * w, L);
            merge_runs(src, dst, a0, a1, a2);           // a lone last run is copied
        }
        __syncthreads();
        in_whole = !in_whole;
    }
    if (in_whole)
        for (uint32_t i = threadIdx.x; i < L; i += TS_THREADS) V[i] = (uint32_t)whole.get(i);
}

// The support exponent p = -1/2 d^T Q d (d = mean - pixel centre) decides which
// pixels a Gaussian touches, so it is evaluated with explicitly rounded float32
// operations: p = fma(-B dx, dy, fma(-C/2 dy, dy, (-A/2 dx) dx)).
constexpr float SUPPORT_P = -4.5f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float T_MIN = 1e-4f;
constexpr int BATCH = 256;            // Gaussians staged in shared memory per round

// per-warp sums of two per-thread counters, one 64-bit atomic each per warp
__device__ __forceinline__ void add_work(unsigned long long *work, uint32_t a, uint32_t b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(work, (unsigned long long)a);
        atomicAdd(work + 1, (unsigned long long)b);
    }
}

// Sum 9 per-lane values over the warp and add the totals to dst[0..8] in shared
// memory.  Values 0..7 use a transposed butterfly: at each exchange a lane keeps
// half of its values and receives its partner's share of that half (4, 2, 1
// shuffles over lane bits 4, 3, 2), while value 8 is summed plainly beside
// them.  The exchange over bit 1 is transposed too, between the lane's one
// remaining value and value 8, and bit 0 is a plain exchange: 12 shuffles in
// all instead of 9 x 5.  Afterwards lane 4i holds the total of value i and
// lane 2 that of value 8; one shared-memory atomic adds all nine.
__device__ __forceinline__ void warp_sum9_to_smem(float v[9], int lane, float *dst) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
    float w4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float send = h16 ? v[i] : v[i + 4];
        float keep = h16 ? v[i + 4] : v[i];
        w4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float s8 = v[8] + __shfl_xor_sync(0xffffffffu, v[8], 16);
    float w2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float send = h8 ? w4[i] : w4[i + 2];
        float keep = h8 ? w4[i + 2] : w4[i];
        w2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    s8 += __shfl_xor_sync(0xffffffffu, s8, 8);
    float w1;
    {
        float send = h4 ? w2[0] : w2[1];
        float keep = h4 ? w2[1] : w2[0];
        w1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    s8 += __shfl_xor_sync(0xffffffffu, s8, 4);
    {                                   // bit 1: value (lanes with bit 1 clear) against value 8 (set)
        float send = h2 ? w1 : s8;
        float keep = h2 ? s8 : w1;
        w1 = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    w1 += __shfl_xor_sync(0xffffffffu, w1, 1);
    if ((lane & 3) == 0 || lane == 2) {
        const int idx = h2 ? 8 : (h16 ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0);
        atomicAdd(dst + idx, w1);
    }
}

// Warp-block layout of a 16x16 tile (128 threads, 2 pixels each): warp w owns
// the 8x8 pixel block at ((w & 1) * 8, (w >> 1) * 8) of the tile, lane l the
// pixels (l & 7, (l >> 3) + 4k), k = 0, 1.  When a batch of the tile's
// Gaussians is staged, each Gaussian gets a 4-bit mask of the blocks its
// support box reaches (the block test), and each warp compacts the batch to
// the Gaussians whose mask holds its block; it then runs over that list only,
// skipping the blend body of a Gaussian no lane's pixel passes the support
// test for.
constexpr int PIX = 2;
constexpr int BNT = TILE_PIX / PIX;
constexpr int NWARP = BNT / 32;
// resident CTAs per SM the register allocation is held to (occupancy)
#ifndef LODGS_FWD_MINB
#define LODGS_FWD_MINB 7
#endif
#ifndef LODGS_BWD_PIX
#define LODGS_BWD_PIX 2      // pixels per lane of the backward blend (2 or 4)
#endif
// Both blends take a lane's two pixels through packed .f32x2 add/mul/fma
// (Blackwell): each half is rounded exactly as the scalar operation, so the
// result is the scalar path's, and the FP32 pipe issues about half the
// instructions.  0 selects the scalar loops (the backward's four-pixel form
// always uses them).
#ifndef LODGS_FWD_F32X2
#define LODGS_FWD_F32X2 1
#endif
#ifndef LODGS_BWD_F32X2
#define LODGS_BWD_F32X2 1
#endif
constexpr int BWD_PIX = LODGS_BWD_PIX;
// LODGS_BWD_MINB (if defined): resident CTAs per SM the backward's registers
// are held to; by default the compiler chooses (56 registers, 9 CTAs)
#ifdef LODGS_BWD_MINB
#define BWD_BOUNDS(nt) __launch_bounds__(nt, LODGS_BWD_MINB)
#else
#define BWD_BOUNDS(nt) __launch_bounds__(nt)
#endif
constexpr float BLOCK_HALF = 3.5f;     // half span of an 8x8 block's pixel centres
constexpr float LOG2E = 1.44269504088896341f;

// 2^x and 1/x on the special function unit, denormals flushed: the blend only
// takes 2^x for x >= -4.5 log2(e) and 1/x for x >= 0.01, where neither an input
// nor a result is denormal.  exp(p) = 2^(p log2 e).
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct BlockPix {
    int w, px, py0;       // warp (block), this lane's column and first row
    float xc;             // pixel-centre x
};

__device__ __forceinline__ BlockPix block_pix(int tile, int TX, int tid) {
    const int w = tid >> 5, lane = tid & 31;
    BlockPix b;
    b.w = w;
    b.px = (tile % TX) * TILE + (w & 1) * 8 + (lane & 7);
    b.py0 = (tile / TX) * TILE + (w >> 1) * 8 + (lane >> 3);
    b.xc = (float)b.px + 0.5f;
    return b;
}

// Blocks of tile (tx0, ty0) that the support box of a Gaussian (mean a.x,
// a.y; half extents c.y, c.z) can reach: bit 2 * by + bx for the block at
// (tx0 + 8 bx, ty0 + 8 by), whose pixel centres have centre (+4, +4) and half
// span 3.5.  Float32, evaluated as written (the block test).
__device__ __forceinline__ uint32_t block_mask(const float4 &a, const float4 &c, int tx0, int ty0) {
    const float hx = __fadd_rn(c.y, BLOCK_HALF), hy = __fadd_rn(c.z, BLOCK_HALF);
    const bool x0 = !(fabsf(__fsub_rn(a.x, __fadd_rn((float)tx0, 4.0f))) > hx);
    const bool x1 = !(fabsf(__fsub_rn(a.x, __fadd_rn((float)(tx0 + 8), 4.0f))) > hx);
    const bool y0 = !(fabsf(__fsub_rn(a.y, __fadd_rn((float)ty0, 4.0f))) > hy);
    const bool y1 = !(fabsf(__fsub_rn(a.y, __fadd_rn((float)(ty0 + 8), 4.0f))) > hy);
    return (uint32_t)(x0 && y0) | (uint32_t)(x1 && y0) << 1 | (uint32_t)(x0 && y1) << 2 |
           (uint32_t)(x1 && y1) << 3;
}

// This warp's list of the staged entries [0, n) whose mask meets the warp's
// blocks (wmask), in ascending order; returns its length.
__device__ __forceinline__ int warp_list(const uint8_t *s_m, int n, uint32_t wmask, int lane, uint8_t *list) {
    int len = 0;
    for (int q0 = 0; q0 < n; q0 += 32) {
        const int q = q0 + lane;
        const bool mine = q < n && (s_m[q] & wmask);
        const unsigned bal = __ballot_sync(0xffffffffu, mine);
        if (mine) list[len + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)q;
        len += __popc(bal);
    }
    __syncwarp();
    return len;
}

// Live-pixel box: once some of a warp's pixels have stopped, the warp builds
// its next lists against the box of the pixel centres still live (centre cx,
// cy; half spans hx, hy) instead of its whole block.  A Gaussian whose support
// box misses it reaches no live pixel (the argument of the block test), so the
// pixels meet exactly the Gaussians they met before: only list entries that
// would have been walked without a hit go.  A long tile list whose block keeps
// one unsaturated pixel then no longer costs a walk of the whole list.  The
// blends take this form (BOX) for frames on the global ordering, the ones with
// long tile lists; elsewhere the lists end before the box would pay for the
// registers it takes.
__device__ __forceinline__ void live_box(float xc, const float *yc, const bool *live, int np, int lane,
                                         float4 *box) {
    float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int k = 0; k < np; ++k) {
        if (live[k]) {
            x0 = fminf(x0, xc); x1 = fmaxf(x1, xc);
            y0 = fminf(y0, yc[k]); y1 = fmaxf(y1, yc[k]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
    }
    // pixel centres are k + 0.5: the centre and half spans are exact
    if (x0 <= x1 && lane == 0) *box = make_float4(0.5f * (x0 + x1), 0.5f * (y0 + y1), 0.5f * (x1 - x0), 0.5f * (y1 - y0));
    __syncwarp();
}

// warp_list restricted to the entries whose support box (half extents r) also
// reaches the live box (centre box.x, box.y; half spans box.z, box.w).
__device__ __forceinline__ int warp_list_box(const uint8_t *s_m, const float4 *s_a, const float2 *s_r, int n,
                                             uint32_t wmask, const float4 &box, int lane, uint8_t *list) {
    const float cx = box.x, cy = box.y, hx = box.z, hy = box.w;
    int len = 0;
    for (int q0 = 0; q0 < n; q0 += 32) {
        const int q = q0 + lane;
        bool mine = false;
        if (q < n && (s_m[q] & wmask)) {
            const float4 a = s_a[q];
            const float2 r = s_r[q];
            mine = !(fabsf(__fsub_rn(a.x, cx)) > __fadd_rn(r.x, hx)) && !(fabsf(__fsub_rn(a.y, cy)) > __fadd_rn(r.y, hy));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, mine);
        if (mine) list[len + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)q;
        len += __popc(bal);
    }
    __syncwarp();
    return len;
}

// COUNT: tally the work counters (profiling launches only).  BOX: live-box lists.
template <bool COUNT, bool BOX>
__global__ void __launch_bounds__(BNT, LODGS_FWD_MINB)
    k_blend(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ pval, const float4 *__restrict__ sp_a,
            const float4 *__restrict__ sp_b, const float4 *__restrict__ sp_c, const uint32_t *__restrict__ cnt, int W,
            int H, int TX, const View *__restrict__ view, float *__restrict__ image,
            unsigned long long *__restrict__ work, const uint32_t *__restrict__ tile_order) {
    pdl_wait();
    __shared__ float4 s_a[BATCH], s_b[BATCH];
    __shared__ float s_c[BATCH];
    __shared__ float2 s_r[BOX ? BATCH : 1];
    __shared__ float4 s_box[BOX ? NWARP : 1];
    __shared__ uint8_t s_m[BATCH];
    __shared__ uint8_t s_list[NWARP][BATCH];
    if (cnt[C_STATUS] & ST_CAPACITY) return;
    const float bg0 = view->bg[0], bg1 = view->bg[1], bg2 = view->bg[2];
    const int tile = (int)tile_order[blockIdx.x], tid = threadIdx.x, lane = tid & 31;
    const int tx0 = (tile % TX) * TILE, ty0 = (tile / TX) * TILE;
    const BlockPix bp = block_pix(tile, TX, tid);
    float yc[PIX], T[PIX], c0[PIX], c1[PIX], c2[PIX];
    bool live[PIX];
    bool done = true;
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int py = bp.py0 + 4 * k;
        yc[k] = (float)py + 0.5f;
        T[k] = 1.0f; c0[k] = c1[k] = c2[k] = 0.f;
        live[k] = bp.px < W && py < H;
        done &= !live[k];
    }
    uint32_t n_eval = 0, n_blend = 0;
    bool whole = true, shrunk = false;      // BOX: lists against the block until a pixel stops
    const uint2 rg = ranges[tile];
    for (uint32_t base = rg.x; base < rg.y; base += BATCH) {
        if (__syncthreads_count(done) == BNT) break;
        const int n = min((uint32_t)BATCH, rg.y - base);
        for (int q = tid; q < n; q += BNT) {
            const uint32_t g = pval[base + q];
            const float4 a = sp_a[g], c = sp_c[g];
            s_a[q] = a;
            s_b[q] = sp_b[g];
            s_c[q] = c.x;
            if constexpr (BOX) s_r[q] = make_float2(c.y, c.z);
            s_m[q] = (uint8_t)block_mask(a, c, tx0, ty0);
        }
        __syncthreads();
        if (__all_sync(0xffffffffu, done)) continue;
        int len;
        if constexpr (BOX) {
            if (shrunk) {
                live_box(bp.xc, yc, live, PIX, lane, &s_box[bp.w]);
                whole = false;
                shrunk = false;
            }
            len = whole ? warp_list(s_m, n, 1u << bp.w, lane, s_list[bp.w])
                        : warp_list_box(s_m, s_a, s_r, n, 1u << bp.w, s_box[bp.w], lane, s_list[bp.w]);
        } else {
            len = warp_list(s_m, n, 1u << bp.w, lane, s_list[bp.w]);
        }
        for (int i = 0; i < len; ++i) {
            const int j = s_list[bp.w][i];
            const float4 a = s_a[j];
            const float4 b = s_b[j];
            const float dx = __fsub_rn(a.x, bp.xc);
            const float hxx = __fmul_rn(__fmul_rn(a.z, dx), dx), bx = __fmul_rn(a.w, dx);
#if LODGS_FWD_F32X2
            {
                // the same float32 operations as below, two pixels per packed instruction
                const float2 dy = __fadd2_rn(make_float2(a.y, a.y), make_float2(-yc[0], -yc[1]));
                const float2 p2 = __ffma2_rn(make_float2(bx, bx), dy,
                                             __ffma2_rn(__fmul2_rn(make_float2(b.x, b.x), dy), dy,
                                                        make_float2(hxx, hxx)));
                const bool h0 = live[0] && p2.x >= SUPPORT_P, h1 = live[1] && p2.y >= SUPPORT_P;
                if (COUNT) n_eval += PIX;
                // no vote to skip a Gaussian no lane reaches: a lane that misses
                // gets alpha = 0, which leaves its colour and T exactly as they
                // were, and the packed body costs less than the vote and branch
                // (measured: forward render 0.1708 -> 0.1664 ms per 1080p view)
                const float cb = s_c[j];
                const float2 pl = __fmul2_rn(p2, make_float2(LOG2E, LOG2E));
                const float2 raw = __fmul2_rn(make_float2(b.y, b.y),
                                              make_float2(h0 ? ex2_ftz(pl.x) : 0.f, h1 ? ex2_ftz(pl.y) : 0.f));
                const float2 alpha = make_float2(fminf(ALPHA_MAX, raw.x), fminf(ALPHA_MAX, raw.y));
                const float2 T2 = make_float2(T[0], T[1]);
                const float2 w = __fmul2_rn(alpha, T2);
                const float2 c02 = __ffma2_rn(make_float2(b.z, b.z), w, make_float2(c0[0], c0[1]));
                const float2 c12 = __ffma2_rn(make_float2(b.w, b.w), w, make_float2(c1[0], c1[1]));
                const float2 c22 = __ffma2_rn(make_float2(cb, cb), w, make_float2(c2[0], c2[1]));
                const float2 Tn = __fmul2_rn(T2, __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-alpha.x, -alpha.y)));
                c0[0] = c02.x; c0[1] = c02.y; c1[0] = c12.x; c1[1] = c12.y; c2[0] = c22.x; c2[1] = c22.y;
                T[0] = Tn.x; T[1] = Tn.y;
                if (COUNT) n_blend += (uint32_t)h0 + (uint32_t)h1;
                const bool s0 = h0 && Tn.x < T_MIN, s1 = h1 && Tn.y < T_MIN;
                live[0] = live[0] && !s0;
                live[1] = live[1] && !s1;
                if (__any_sync(0xffffffffu, s0 || s1)) {
                    if (BOX) shrunk = true;
                    done = !live[0] && !live[1];
                    if (__all_sync(0xffffffffu, done)) break;
                }
                continue;
            }
#endif
            float p[PIX];
            bool hit[PIX], any = false;
#pragma unroll
            for (int k = 0; k < PIX; ++k) {
                const float dy = __fsub_rn(a.y, yc[k]);
                p[k] = __fmaf_rn(bx, dy, __fmaf_rn(__fmul_rn(b.x, dy), dy, hxx));
                hit[k] = live[k] && p[k] >= SUPPORT_P;
                any |= hit[k];
            }
            if (COUNT) n_eval += PIX;
            if (!__any_sync(0xffffffffu, any)) continue;
            const float cb = s_c[j];
            bool died = false;
#pragma unroll
            for (int k = 0; k < PIX; ++k) {     // predicated: alpha = 0 leaves T and the colour unchanged
                if (COUNT) n_blend += hit[k];
                const float alpha = hit[k] ? fminf(ALPHA_MAX, b.y * ex2_ftz(p[k] * LOG2E)) : 0.f;
                const float w = alpha * T[k];
                c0[k] += b.z * w; c1[k] += b.w * w; c2[k] += cb * w;
                T[k] = T[k] * (1.0f - alpha);
                const bool stop = hit[k] && T[k] < T_MIN;
                live[k] = live[k] && !stop;
                died |= stop;
            }
            if (__any_sync(0xffffffffu, died)) {
                if (BOX) shrunk = true;
                done = true;
#pragma unroll
                for (int k = 0; k < PIX; ++k) done &= !live[k];
                if (__all_sync(0xffffffffu, done)) break;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int py = bp.py0 + 4 * k;
        if (bp.px < W && py < H) {
            const size_t o = (size_t)py * W + bp.px;
            float *img = image + o * 3;
            img[0] = c0[k] + T[k] * bg0; img[1] = c1[k] + T[k] * bg1; img[2] = c2[k] + T[k] * bg2;
        }
    }
    if (COUNT) add_work(work, n_eval, n_blend);
}

// Backward of the blend, front to back over each tile's list like the forward,
// recomputing each pixel's transmittance per tile (nothing per pixel is stored
// by the forward).  With T_i the transmittance in front of Gaussian i, A_i the
// colour composited in front of it and C the forward's output (background
// included), the colour behind i is S_i = C - A_i - c_i alpha_i T_i, and
//   dL/dc_i = G alpha_i T_i,   dL/dalpha_i = T_i G.c_i - G.S_i / (1 - alpha_i),
// with G = dL/dC.  Each pixel carries the scalar g = G.(C - A), which drops by
// alpha_i T_i G.c_i at every contribution, so G.S_i needs no colour sums.  T is
// rebuilt with the forward's own float operations, so the backward visits
// exactly the contributions the forward blended and stops where it stopped.  The nine per-Gaussian sums of a warp are reduced in
// registers and added to shared memory; each batch's sums go to global memory
// with 16-byte atomics.
// BP pixels per lane: 2 (a warp per 8x8 block, 128 threads per tile) or 4 (a
// warp per 8x16 column of two blocks, 64 threads per tile).
// L1 (1: float32 target, 2: 8-bit target read as byte / 255, correctly
// rounded): dL/dC is not read but formed from the image and the target as the
// L1 loss's gradient, l1_scale * sign(C - target), and the block adds its
// sum |C - target| to *loss_sum (the training loss folded into the backward:
// no separate pass over the image, no dL/dC buffer).  0: dL/dC from dL_dimg.
template <bool COUNT, int BP, int L1, bool BOX>
__global__ void BWD_BOUNDS(TILE_PIX / BP)
    k_blend_bwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ pval,
                const float4 *__restrict__ sp_a, const float4 *__restrict__ sp_b, const float4 *__restrict__ sp_c,
                const uint32_t *__restrict__ cnt, int W, int H, int TX, const float *__restrict__ image,
                const float *__restrict__ dL_dimg, float *__restrict__ g2d, unsigned long long *__restrict__ work,
                const void *__restrict__ target, float l1_scale, float *__restrict__ loss_sum,
                const uint32_t *__restrict__ tile_order) {
    pdl_wait();
    constexpr int NT = TILE_PIX / BP, NW = NT / 32;
    __shared__ float4 s_a[BATCH], s_b[BATCH];
    __shared__ float s_c[BATCH];
    __shared__ float2 s_r[BOX ? BATCH : 1];
    __shared__ float4 s_box[BOX ? NW : 1];
    __shared__ uint32_t s_g[BATCH];
    __shared__ float s_grad[BATCH][9];
    __shared__ uint8_t s_m[BATCH];
    __shared__ uint8_t s_list[NW][BATCH];
    if (cnt[C_STATUS] & ST_CAPACITY) return;
    const int tile = (int)tile_order[blockIdx.x], tid = threadIdx.x, lane = tid & 31;
    const int tx0 = (tile % TX) * TILE, ty0 = (tile / TX) * TILE;
    const BlockPix bp = block_pix(tile, TX, tid);
    // blocks this warp covers: (w & 1, (w >> 1) + k / 2) for its pixel rows k
    uint32_t wmask = 0;
#pragma unroll
    for (int k = 0; k < BP; k += 2) wmask |= 1u << (((bp.w >> 1) + k / 2) * 2 + (bp.w & 1));
    float yc[BP], T[BP], gS[BP], G[BP][3];
    bool live[BP];
    bool done = true;
    float l1 = 0.f;
#pragma unroll
    for (int k = 0; k < BP; ++k) {
        const int py = bp.py0 + 4 * k;
        yc[k] = (float)py + 0.5f;
        T[k] = 1.0f;
        live[k] = bp.px < W && py < H;
        G[k][0] = G[k][1] = G[k][2] = gS[k] = 0.f;
        if (live[k]) {
            const size_t o = ((size_t)py * W + bp.px) * 3;
            const float c0 = image[o], c1 = image[o + 1], c2 = image[o + 2];
            if (L1) {
                float tg[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
                    tg[ch] = L1 == 2 ? __fdiv_rn((float)static_cast<const uint8_t *>(target)[o + ch], 255.0f)
                                     : static_cast<const float *>(target)[o + ch];
                const float d[3] = {c0 - tg[0], c1 - tg[1], c2 - tg[2]};
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    G[k][ch] = l1_scale * (d[ch] > 0.f ? 1.f : (d[ch] < 0.f ? -1.f : 0.f));
                    l1 += fabsf(d[ch]);
                }
            } else {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) G[k][ch] = dL_dimg[o + ch];
            }
            gS[k] = G[k][0] * c0 + G[k][1] * c1 + G[k][2] * c2;                       // G.C
        }
        done &= !live[k];
    }
    if (L1) {                                                                    // the tile's loss sum
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        __shared__ float s_l1[NW];
        if (lane == 0) s_l1[bp.w] = l1;
        __syncthreads();
        if (tid == 0) {
            float sum = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) sum += s_l1[w];
            atomicAdd(loss_sum, sum);
        }
    }
    uint32_t n_eval = 0, n_contrib = 0;
    // packed form of the two pixels' state (LODGS_BWD_F32X2, BP == 2): .x the
    // upper pixel, .y the lower one; ngs = -G.S
    float2 T2 = make_float2(T[0], T[BP > 1 ? 1 : 0]), ngs2 = make_float2(-gS[0], -gS[BP > 1 ? 1 : 0]);
    const float2 nyc2 = make_float2(-yc[0], -yc[BP > 1 ? 1 : 0]);
    const float2 G02 = make_float2(G[0][0], G[BP > 1 ? 1 : 0][0]), G12 = make_float2(G[0][1], G[BP > 1 ? 1 : 0][1]);
    const float2 G22 = make_float2(G[0][2], G[BP > 1 ? 1 : 0][2]);
    bool whole = true, shrunk = false;      // BOX: lists against the blocks until a pixel stops
    const uint2 rg = ranges[tile];
    for (uint32_t base = rg.x; base < rg.y; base += BATCH) {
        if (__syncthreads_count(done) == NT) break;
        const int n = min((uint32_t)BATCH, rg.y - base);
        for (int q = tid; q < n; q += NT) {
            const uint32_t g = pval[base + q];
            const float4 a = sp_a[g], c = sp_c[g];
            s_g[q] = g;
            s_a[q] = a;
            s_b[q] = sp_b[g];
            s_c[q] = c.x;
            if constexpr (BOX) s_r[q] = make_float2(c.y, c.z);
            s_m[q] = (uint8_t)block_mask(a, c, tx0, ty0);
#pragma unroll
            for (int v = 0; v < 9; ++v) s_grad[q][v] = 0.f;
        }
        __syncthreads();
        if (!__all_sync(0xffffffffu, done)) {
            int len;
            if constexpr (BOX) {
                if (shrunk) {
                    live_box(bp.xc, yc, live, BP, lane, &s_box[bp.w]);
                    whole = false;
                    shrunk = false;
                }
                len = whole ? warp_list(s_m, n, wmask, lane, s_list[bp.w])
                            : warp_list_box(s_m, s_a, s_r, n, wmask, s_box[bp.w], lane, s_list[bp.w]);
            } else {
                len = warp_list(s_m, n, wmask, lane, s_list[bp.w]);
            }
            for (int i = 0; i < len; ++i) {
                const int j = s_list[bp.w][i];
                const float4 a = s_a[j];
                const float4 b = s_b[j];
                const float dx = __fsub_rn(a.x, bp.xc);
                const float hxx = __fmul_rn(__fmul_rn(a.z, dx), dx), bx = __fmul_rn(a.w, dx);
#if LODGS_BWD_F32X2
                if constexpr (BP == 2) {
                    // the same float32 operations as below, two pixels per packed
                    // instruction (add/mul/fma .f32x2 round each half as the scalar op)
                    const float2 dy = __fadd2_rn(make_float2(a.y, a.y), nyc2);
                    const float2 p = __ffma2_rn(make_float2(bx, bx), dy,
                                                __ffma2_rn(__fmul2_rn(make_float2(b.x, b.x), dy), dy,
                                                           make_float2(hxx, hxx)));
                    const bool h0 = live[0] && p.x >= SUPPORT_P, h1 = live[1] && p.y >= SUPPORT_P;
                    if (COUNT) n_eval += 2;
                    if (!__any_sync(0xffffffffu, h0 || h1)) continue;   // here the skip pays (measured)
                    const float cb = s_c[j];
                    const float2 pl = __fmul2_rn(p, make_float2(LOG2E, LOG2E));
                    const float2 e = make_float2(h0 ? ex2_ftz(pl.x) : 0.f, h1 ? ex2_ftz(pl.y) : 0.f);
                    const float2 raw = __fmul2_rn(make_float2(b.y, b.y), e);
                    const float2 alpha = make_float2(fminf(ALPHA_MAX, raw.x), fminf(ALPHA_MAX, raw.y));
                    const float2 w = __fmul2_rn(alpha, T2);
                    const float2 gc = __ffma2_rn(G22, make_float2(cb, cb),
                                                 __ffma2_rn(G12, make_float2(b.w, b.w),
                                                            __fmul2_rn(G02, make_float2(b.z, b.z))));
                    ngs2 = __ffma2_rn(w, gc, ngs2);                                      // -G.S_i
                    const float2 om = __fadd2_rn(make_float2(1.0f, 1.0f), make_float2(-alpha.x, -alpha.y));
                    const float2 dA = __ffma2_rn(make_float2(rcp_ftz(om.x), rcp_ftz(om.y)), ngs2,
                                                 __fmul2_rn(T2, gc));
                    float2 de = __fmul2_rn(dA, e);
                    de.x = raw.x <= ALPHA_MAX ? de.x : 0.f;                              // 0 where clamped
                    de.y = raw.y <= ALPHA_MAX ? de.y : 0.f;
                    const float2 t = __fmul2_rn(de, dy);
                    const float2 t2 = __fmul2_rn(t, dy);
                    const float2 gw0 = __fmul2_rn(G02, w), gw1 = __fmul2_rn(G12, w), gw2 = __fmul2_rn(G22, w);
                    T2 = __fmul2_rn(T2, om);                                            // as the forward
                    if (COUNT) n_contrib += (uint32_t)h0 + (uint32_t)h1;
                    const bool s0 = h0 && T2.x < T_MIN, s1 = h1 && T2.y < T_MIN;
                    live[0] = live[0] && !s0;
                    live[1] = live[1] && !s1;
                    const float q0 = de.x + de.y, q1 = t.x + t.y;
                    const float dq0 = dx * q0;
                    float gv[9] = {dq0, q1, dx * dq0, dx * q1, t2.x + t2.y, q0, gw0.x + gw0.y, gw1.x + gw1.y,
                                   gw2.x + gw2.y};
                    warp_sum9_to_smem(gv, lane, s_grad[j]);
                    if (__any_sync(0xffffffffu, s0 || s1)) {
                        if (BOX) shrunk = true;
                        done = !live[0] && !live[1];
                        if (__all_sync(0xffffffffu, done)) break;
                    }
                    continue;
                }
#endif
                float p[BP], dyk[BP];
                bool hit[BP], any = false;
#pragma unroll
                for (int k = 0; k < BP; ++k) {
                    dyk[k] = __fsub_rn(a.y, yc[k]);
                    p[k] = __fmaf_rn(bx, dyk[k], __fmaf_rn(__fmul_rn(b.x, dyk[k]), dyk[k], hxx));
                    hit[k] = live[k] && p[k] >= SUPPORT_P;
                    any |= hit[k];
                }
                if (COUNT) n_eval += BP;
                if (!__any_sync(0xffffffffu, any)) continue;
                const float cb = s_c[j];
                // predicated: a lane whose pixel misses gets alpha = e = 0, which
                // leaves T and G.S unchanged and makes every term below zero.
                // Where alpha is not clamped, dL/dp = alpha dL/dalpha = o de with
                // de = e dL/dalpha (o the opacity), and de itself is dL/do.  With
                // p = a.z dx^2 + a.w dx dy + b.x dy^2 the mean and conic gradients
                // are linear in the moments q0 = sum de, q1 = sum de dy,
                // q2 = sum de dy^2 over the lane's pixels (which share dx).  The
                // warp reduces dx q0, q1, dx^2 q0, dx q1, q2 and q0 (= dL/do); the
                // flush applies o and the coefficients 2 a.z, a.w, 2 b.x.
                float q0 = 0.f, q1 = 0.f, q2 = 0.f, gr = 0.f, gg = 0.f, gb = 0.f;
                bool died = false;
#pragma unroll
                for (int k = 0; k < BP; ++k) {
                    if (COUNT) n_contrib += hit[k];
                    const float dy = dyk[k];
                    const float e = hit[k] ? ex2_ftz(p[k] * LOG2E) : 0.f;
                    const float raw = b.y * e;
                    const float alpha = fminf(ALPHA_MAX, raw);
                    const float w = alpha * T[k];
                    const float gc = G[k][0] * b.z + G[k][1] * b.w + G[k][2] * cb;
                    gS[k] -= w * gc;                                                      // G.S_i
                    const float dA = T[k] * gc - rcp_ftz(1.0f - alpha) * gS[k];
                    const float de = raw <= ALPHA_MAX ? dA * e : 0.f;                    // 0 where clamped
                    const float t = de * dy;
                    q0 += de;
                    q1 += t;
                    q2 = __fmaf_rn(t, dy, q2);
                    gr += G[k][0] * w;
                    gg += G[k][1] * w;
                    gb += G[k][2] * w;
                    T[k] = T[k] * (1.0f - alpha);                                         // as the forward
                    const bool stop = hit[k] && T[k] < T_MIN;
                    live[k] = live[k] && !stop;
                    died |= stop;
                }
                const float dq0 = dx * q0;
                float gv[9] = {dq0, q1, dx * dq0, dx * q1, q2, q0, gr, gg, gb};
                warp_sum9_to_smem(gv, lane, s_grad[j]);
                if (__any_sync(0xffffffffu, died)) {
                    if (BOX) shrunk = true;
                    done = true;
#pragma unroll
                    for (int k = 0; k < BP; ++k) done &= !live[k];
                    if (__all_sync(0xffffffffu, done)) break;
                }
            }
        }
        __syncthreads();
        for (int q = tid; q < n; q += NT) {
            float *o = g2d + (size_t)s_g[q] * G2D_STRIDE;
            // moments -> d(u, v) and d(conic) with this Gaussian's opacity and coefficients
            const float o_ = s_b[q].y;
            const float r0 = o_ * s_grad[q][0], r1 = o_ * s_grad[q][1], r2 = o_ * s_grad[q][2];
            const float r3 = o_ * s_grad[q][3], r4 = o_ * s_grad[q][4];
            const float az = s_a[q].z, aw = s_a[q].w, bxc = s_b[q].x;
            const float4 x0 = make_float4(2.0f * az * r0 + aw * r1, aw * r0 + 2.0f * bxc * r1, -0.5f * r2, -r3);
            const float4 x1 = make_float4(-0.5f * r4, s_grad[q][5], s_grad[q][6], s_grad[q][7]);
            if (x0.x != 0.f || x0.y != 0.f || x0.z != 0.f || x0.w != 0.f)
                atomicAdd(reinterpret_cast<float4 *>(o), x0);
            if (x1.x != 0.f || x1.y != 0.f || x1.z != 0.f || x1.w != 0.f)
                atomicAdd(reinterpret_cast<float4 *>(o + 4), x1);
            if (s_grad[q][8] != 0.f) atomicAdd(o + 8, s_grad[q][8]);
        }
    }
    if (COUNT) add_work(work + 2, n_eval, n_contrib);
}


}  // namespace

int ceil_log2(uint64_t x) {
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

// Per-tile ordering for frames whose pair workspace averages at most this many
// pairs per tile; the global sorts for denser frames (long tile lists).
constexpr uint64_t PER_TILE_MAX_MEAN = 1024;

int launch_raster(const CamK &k, FrameBufs &f, float *image, cudaStream_t st, const StageMarks &sm) {
    const uint64_t n_tiles = (uint64_t)k.TX * k.TY;
    const bool per_tile = f.ordering == ORDER_PER_TILE ||
                          (f.ordering == ORDER_AUTO && f.cap_pairs <= PER_TILE_MAX_MEAN * n_tiles);
    if (per_tile) {
        f.order = nullptr;
        sm.mark(LODGS_STAGE_COUNT, 0, st);
        int rc = scan_exclusive(f.ntiles, f.pair_off, f.cnt + C_NSEL_EFF, (uint32_t)f.cap_sel, f.scan_bsum,
                                f.cnt + C_NPAIR, st);     // rectangle pairs per selected Gaussian
        if (rc) return rc;
        const uint32_t keep_cap = (uint32_t)std::min<uint64_t>(f.cap_keep, UINT32_MAX);
        LODGS_CUDA(pdl_launch(k_emit_count, EGRID, RB, st, f.pair_off, f.rect, f.sp_a, f.sp_b, f.cnt, k.TX, f.tile_cnt,
                              f.keep, keep_cap));
        LODGS_CUDA(pdl_launch(k_tile_offsets, 1, TO_THREADS, st, f.tile_cnt, (uint32_t)n_tiles, f.cap_pairs, f.cnt,
                              f.ranges, f.tile_order));
        count_launches(2);
        sm.mark(LODGS_STAGE_COUNT, 1, st);
        sm.mark(LODGS_STAGE_EMIT, 0, st);
        LODGS_CUDA(pdl_launch(k_emit_scatter, EGRID, RB, st, f.pair_off, f.rect, f.sp_a, f.sp_b, f.dkey, f.cnt, k.TX,
                              f.tile_cnt, f.pkey, f.pval, f.keep, keep_cap));
        count_launches(1);
        sm.mark(LODGS_STAGE_EMIT, 1, st);
        sm.mark(LODGS_STAGE_TILE_SORT, 0, st);
        LODGS_CUDA(pdl_launch(k_tile_sort, (unsigned)n_tiles, TS_THREADS, st, f.ranges, f.tile_cnt, f.cnt, f.pkey, f.pval,
                              f.pscratch, f.tile_order));
        count_launches(1);
        sm.mark(LODGS_STAGE_TILE_SORT, 1, st);
        f.sorted_pval = f.pval;
        sm.mark(LODGS_STAGE_BLEND, 0, st);
    } else {
        bool alt;
        sm.mark(LODGS_STAGE_COUNT, 0, st);        // depth sort of the selected Gaussians
        int rc = radix_sort_pairs(f.dkey, f.dval, f.dkey_alt, f.dval_alt, f.cnt + C_NSEL_EFF, (uint32_t)f.cap_sel,
                                  0, 32, f.sort_hist, st, &alt);
        if (rc) return rc;
        const uint32_t *order = alt ? f.dval_alt : f.dval;
        f.order = order;
        sm.mark(LODGS_STAGE_COUNT, 1, st);
        sm.mark(LODGS_STAGE_EMIT, 0, st);
        rc = scan_exclusive(f.ntiles, f.pair_off, f.cnt + C_NSEL_EFF, (uint32_t)f.cap_sel, f.scan_bsum,
                            f.cnt + C_NPAIR, st, order);  // tile counts in depth order
        if (rc) return rc;
        LODGS_CUDA(pdl_launch(k_emit, RGRID, RB, st, order, f.rect, f.sp_a, f.sp_b, f.pair_off, f.cnt, f.cap_pairs, k.TX,
                                     (uint32_t)n_tiles, f.pkey, f.pval));
        count_launches(1);
        sm.mark(LODGS_STAGE_EMIT, 1, st);
        sm.mark(LODGS_STAGE_TILE_SORT, 0, st);
        rc = radix_sort_pairs(f.pkey, f.pval, f.pkey_alt, f.pval_alt, f.cnt + C_NPAIR_EFF, (uint32_t)f.cap_pairs, 0,
                              ceil_log2(n_tiles + 1), f.sort_hist, st, &alt);
        if (rc) return rc;
        const uint32_t *skey = alt ? f.pkey_alt : f.pkey;
        f.sorted_pval = alt ? f.pval_alt : f.pval;
        LODGS_CUDA(cudaMemsetAsync(f.ranges, 0, n_tiles * sizeof(uint2), st));
        LODGS_CUDA(pdl_launch(k_ranges, RGRID, RB, st, skey, f.cnt, (uint32_t)n_tiles, f.ranges));
        LODGS_CUDA(pdl_launch(k_tile_order, 1, TOR_THREADS, st, f.ranges, (uint32_t)n_tiles, f.tile_order));
        count_launches(2);
        sm.mark(LODGS_STAGE_TILE_SORT, 1, st);
        sm.mark(LODGS_STAGE_BLEND, 0, st);
    }
    if (f.count_work) LODGS_CUDA(cudaMemsetAsync(f.work, 0, 4 * sizeof(unsigned long long), st));   // profiling only
    const bool box = f.order != nullptr;     // global ordering: a frame with long tile lists
    LODGS_CUDA(pdl_launch_p(0, (f.count_work ? (box ? k_blend<true, true> : k_blend<true, false>)
                                             : (box ? k_blend<false, true> : k_blend<false, false>)), (unsigned)n_tiles, BNT, st,
        f.ranges, f.sorted_pval, f.sp_a, f.sp_b, f.sp_c, f.cnt, k.W, k.H, k.TX, f.d_view, image, f.work,
        f.tile_order));
    count_launches(1);
    sm.mark(LODGS_STAGE_BLEND, 1, st);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

int launch_raster_backward(const CamK &k, FrameBufs &f, const float *image, const float *dL_dimage,
                           const void *target, bool target_u8, float l1_scale, float *loss_sum, bool zero_g2d,
                           cudaStream_t st) {
    const uint64_t n_tiles = (uint64_t)k.TX * k.TY;
    if (zero_g2d)          // the projection zeroes the rows of its selection; a repeated backward re-zeroes
        LODGS_CUDA(cudaMemsetAsync(f.g2d, 0, f.cap_sel * G2D_STRIDE * sizeof(float), st));
    if (f.count_work) LODGS_CUDA(cudaMemsetAsync(f.work + 2, 0, 2 * sizeof(unsigned long long), st));
    const unsigned nb = (unsigned)n_tiles, nt = TILE_PIX / BWD_PIX;
    const bool box = f.order != nullptr;     // the render's global ordering: long tile lists
    if (target) {
        LODGS_CUDA(cudaMemsetAsync(loss_sum, 0, sizeof(float), st));
        auto kern = box ? (target_u8 ? (f.count_work ? k_blend_bwd<true, BWD_PIX, 2, true> : k_blend_bwd<false, BWD_PIX, 2, true>)
                                     : (f.count_work ? k_blend_bwd<true, BWD_PIX, 1, true> : k_blend_bwd<false, BWD_PIX, 1, true>))
                        : (target_u8 ? (f.count_work ? k_blend_bwd<true, BWD_PIX, 2, false> : k_blend_bwd<false, BWD_PIX, 2, false>)
                                     : (f.count_work ? k_blend_bwd<true, BWD_PIX, 1, false> : k_blend_bwd<false, BWD_PIX, 1, false>));
        LODGS_CUDA(pdl_launch_p(0, kern, nb, nt, st, f.ranges, f.sorted_pval, f.sp_a, f.sp_b, f.sp_c, f.cnt, k.W, k.H, k.TX, image,
                                nullptr, f.g2d, f.work, target, l1_scale, loss_sum, f.tile_order));
    } else {
        LODGS_CUDA(pdl_launch_p(0, (box ? (f.count_work ? k_blend_bwd<true, BWD_PIX, 0, true> : k_blend_bwd<false, BWD_PIX, 0, true>)
                                        : (f.count_work ? k_blend_bwd<true, BWD_PIX, 0, false> : k_blend_bwd<false, BWD_PIX, 0, false>)), nb, nt, st,
            f.ranges, f.sorted_pval, f.sp_a, f.sp_b, f.sp_c, f.cnt, k.W, k.H, k.TX, image, dL_dimage, f.g2d, f.work,
            nullptr, 0.f, nullptr, f.tile_order));
    }
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

}  // namespace lodgs
