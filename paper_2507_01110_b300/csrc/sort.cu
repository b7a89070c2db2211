// Stable LSD radix sort of (uint32 key, uint32 value) pairs and exclusive scans.
//
// Both run on a fixed grid and read the element count from device memory, so a
// render needs no host round trip between its stages.  The sort is the
// reduce-then-scan form: per pass an upsweep builds a digit histogram per block
// (each block owns one contiguous chunk), one warp per digit scans that digit's
// block counts, and a downsweep (which scans the 256 digit totals itself) ranks
// each tile of its chunk with warp match/ballot ranking and scatters it.  No
// block waits on another.
#include <algorithm>

#include "lodgs_internal.cuh"

namespace lodgs {

namespace {
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int ST_THREADS = 256;                 // 8 warps
constexpr int ST_WARPS = ST_THREADS / 32;
constexpr int ST_ITEMS = 8;
constexpr int ST_TILE = ST_THREADS * ST_ITEMS;  // 2048 keys per tile
static_assert(RADIX == ST_THREADS, "one thread per digit in the digit scans");

__device__ __forceinline__ void chunk_range(uint32_t n, uint32_t &begin, uint32_t &end) {
    uint32_t G = gridDim.x;
    uint32_t per = (n + G - 1) / G;
    per = (per + ST_TILE - 1) / ST_TILE * ST_TILE;
    uint64_t b = (uint64_t)blockIdx.x * per;
    begin = b < n ? (uint32_t)b : n;
    uint64_t e = b + per;
    end = e < n ? (uint32_t)e : n;
}

__global__ void __launch_bounds__(ST_THREADS) k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                              const uint32_t *__restrict__ d_n, int shift,
                                                              uint32_t mask, uint32_t *__restrict__ hist) {
    pdl_wait();
    __shared__ uint32_t s_cnt[ST_WARPS][RADIX];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < ST_WARPS * RADIX; i += ST_THREADS) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    uint32_t begin, end;
    chunk_range(*d_n, begin, end);
    for (uint32_t i = begin + tid; i < end; i += ST_THREADS) {
        uint32_t d = (keys[i] >> shift) & mask;
        atomicAdd(&s_cnt[warp][d], 1u);
    }
    __syncthreads();
    for (int d = tid; d < RADIX; d += ST_THREADS) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < ST_WARPS; ++w) s += s_cnt[w][d];
        hist[(size_t)d * gridDim.x + blockIdx.x] = s;
    }
}

// Per digit d (one warp each): exclusive scan in place of the per-block counts
// hist[d*G .. d*G+G) and the digit total in totals[d].  All of a digit's counts
// are loaded before any is written back, so the loads overlap.
constexpr int DS_CHUNKS = (SORT_GRID_MAX + 31) / 32;
__global__ void __launch_bounds__(256) k_digit_scan(uint32_t *__restrict__ hist, int G, uint32_t *__restrict__ totals) {
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * 8 + (threadIdx.x >> 5);
    uint32_t *h = hist + (size_t)d * G;
    uint32_t v[DS_CHUNKS];
#pragma unroll
    for (int c = 0; c < DS_CHUNKS; ++c) {
        const int i = c * 32 + lane;
        v[c] = i < G ? h[i] : 0u;
    }
    uint32_t carry = 0;
#pragma unroll
    for (int c = 0; c < DS_CHUNKS; ++c) {
        uint32_t x = v[c];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int i = c * 32 + lane;
        if (i < G) h[i] = carry + x - v[c];
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) totals[d] = carry;
}

__global__ void __launch_bounds__(ST_THREADS) k_radix_downsweep(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, uint32_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, const uint32_t *__restrict__ d_n, int shift, uint32_t mask,
    const uint32_t *__restrict__ hist, const uint32_t *__restrict__ totals) {
    pdl_wait();
    __shared__ uint32_t s_off[RADIX];
    __shared__ uint32_t s_tot[RADIX];
    __shared__ uint32_t s_start[RADIX];           // the tile's digit runs: exclusive scan of s_tot
    __shared__ uint32_t s_sum[ST_WARPS];
    __shared__ uint32_t s_w[ST_WARPS][RADIX];
    __shared__ uint32_t s_k[ST_TILE], s_v[ST_TILE];   // the tile, stably ordered by digit
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {   // digit bases: exclusive scan of the digit totals (RADIX == ST_THREADS)
        uint32_t t = totals[tid];
        uint32_t x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_tot[warp] = x;
        __syncthreads();
        uint32_t wb = 0;
        for (int w = 0; w < warp; ++w) wb += s_tot[w];
        s_off[tid] = wb + x - t + hist[(size_t)tid * gridDim.x + blockIdx.x];
        __syncthreads();
    }
    uint32_t begin, end;
    chunk_range(*d_n, begin, end);
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t t0 = begin; t0 < end; t0 += ST_TILE) {
        for (int i = tid; i < ST_WARPS * RADIX; i += ST_THREADS) (&s_w[0][0])[i] = 0;
        __syncthreads();
        uint32_t key[ST_ITEMS], val[ST_ITEMS], rank[ST_ITEMS];
#pragma unroll
        for (int k = 0; k < ST_ITEMS; ++k) {
            uint32_t idx = t0 + warp * (32 * ST_ITEMS) + k * 32 + lane;
            bool ok = idx < end;
            key[k] = ok ? keys_in[idx] : 0u;
            val[k] = ok ? vals_in[idx] : 0u;
            uint32_t d = ok ? ((key[k] >> shift) & mask) : 0xffffu;
            uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t prior = 0;
            if (ok) prior = s_w[warp][d];
            rank[k] = prior + __popc(peers & lt);
            __syncwarp();
            if (ok && (peers & lt) == 0) s_w[warp][d] = prior + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int d = tid; d < RADIX; d += ST_THREADS) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < ST_WARPS; ++w) {
                uint32_t c = s_w[w][d];
                s_w[w][d] = run;
                run += c;
            }
            s_tot[d] = run;
        }
        __syncthreads();
        {   // where each digit's run starts in the tile (RADIX == ST_THREADS)
            const uint32_t c = s_tot[tid];
            uint32_t x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_sum[warp] = x;
            __syncthreads();
            uint32_t wb = 0;
            for (int w = 0; w < warp; ++w) wb += s_sum[w];
            s_start[tid] = wb + x - c;
        }
        __syncthreads();
        // stage the tile in shared memory in (digit, input order) order, then
        // write each digit's run out contiguously: consecutive threads write
        // consecutive addresses instead of one scattered word per key
#pragma unroll
        for (int k = 0; k < ST_ITEMS; ++k) {
            uint32_t idx = t0 + warp * (32 * ST_ITEMS) + k * 32 + lane;
            if (idx < end) {
                uint32_t d = (key[k] >> shift) & mask;
                uint32_t lp = s_start[d] + s_w[warp][d] + rank[k];
                s_k[lp] = key[k];
                s_v[lp] = val[k];
            }
        }
        __syncthreads();
        const uint32_t nt = end - t0 < (uint32_t)ST_TILE ? end - t0 : (uint32_t)ST_TILE;
        for (uint32_t i = tid; i < nt; i += ST_THREADS) {
            const uint32_t kk = s_k[i];
            const uint32_t d = (kk >> shift) & mask;
            const uint32_t pos = s_off[d] + (i - s_start[d]);
            keys_out[pos] = kk;
            vals_out[pos] = s_v[i];
        }
        __syncthreads();
        for (int d = tid; d < RADIX; d += ST_THREADS) s_off[d] += s_tot[d];
        __syncthreads();
    }
}

// ---- exclusive scan ---------------------------------------------------------
constexpr int SC_THREADS = 512;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;
// scans of at most this many values run in one block (one launch instead of two)
constexpr uint32_t SCAN_ONE_BLOCK = 16384;

__device__ __forceinline__ void scan_chunk(uint32_t n, uint32_t &begin, uint32_t &end) {
    uint32_t G = gridDim.x;
    uint32_t per = (n + G - 1) / G;
    per = (per + SC_TILE - 1) / SC_TILE * SC_TILE;
    uint64_t b = (uint64_t)blockIdx.x * per;
    begin = b < n ? (uint32_t)b : n;
    uint64_t e = b + per;
    end = e < n ? (uint32_t)e : n;
}

__device__ __forceinline__ uint32_t block_reduce_add(uint32_t v, uint32_t *s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;   // valid in warp 0
}

// The scan's two passes as device functions, launched for one array
// (k_scan_reduce, k_scan_down) or for several at once (the _batch kernels: one
// array per grid row blockIdx.y).
__device__ __forceinline__ void scan_reduce_body(const uint32_t *__restrict__ in, const uint32_t *__restrict__ idx,
                                                 const uint32_t *__restrict__ d_n, uint32_t *__restrict__ block_sums) {
    __shared__ uint32_t s_warp[32];
    uint32_t begin, end;
    scan_chunk(*d_n, begin, end);
    uint32_t s = 0;
    for (uint32_t i = begin + threadIdx.x; i < end; i += SC_THREADS) s += in[idx ? idx[i] : i];
    s = block_reduce_add(s, s_warp);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = s;
}

__device__ __forceinline__ void scan_down_body(const uint32_t *in, const uint32_t *__restrict__ idx, uint32_t *out,
                                               const uint32_t *__restrict__ d_n,
                                               const uint32_t *__restrict__ block_sums, uint32_t *d_total) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // offset of this block = sum of the sums of the blocks before it
    uint32_t pre = 0;
    for (uint32_t b = tid; b < blockIdx.x; b += SC_THREADS) pre += block_sums[b];
    pre = block_reduce_add(pre, s_warp);
    if (tid == 0) s_carry = pre;
    __syncthreads();
    uint32_t n = *d_n;
    uint32_t begin, end;
    scan_chunk(n, begin, end);
    for (uint32_t t0 = begin; t0 < end; t0 += SC_TILE) {
        // each thread owns SC_ITEMS consecutive elements
        uint32_t v[SC_ITEMS];
        uint32_t base = t0 + tid * SC_ITEMS;
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < SC_ITEMS; ++k) {
            uint32_t i = base + k;
            v[k] = i < end ? in[idx ? idx[i] : i] : 0u;
            sum += v[k];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < SC_THREADS / 32 ? s_warp[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < SC_THREADS / 32) s_warp[lane] = w;
        }
        __syncthreads();
        uint32_t carry = s_carry;
        uint32_t run = carry + (warp ? s_warp[warp - 1] : 0u) + x - sum;
#pragma unroll
        for (int k = 0; k < SC_ITEMS; ++k) {
            uint32_t i = base + k;
            if (i < end) out[i] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 0) s_carry = carry + s_warp[SC_THREADS / 32 - 1];
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && tid == 0 && d_total) *d_total = s_carry;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const uint32_t *__restrict__ in,
                                                            const uint32_t *__restrict__ idx,
                                                            const uint32_t *__restrict__ d_n,
                                                            uint32_t *__restrict__ block_sums) {
    pdl_wait();
    scan_reduce_body(in, idx, d_n, block_sums);
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_down(const uint32_t *in, const uint32_t *__restrict__ idx,
                                                          uint32_t *out, const uint32_t *__restrict__ d_n,
                                                          const uint32_t *__restrict__ block_sums,
                                                          uint32_t *d_total) {
    pdl_wait();
    scan_down_body(in, idx, out, d_n, block_sums, d_total);
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce_batch(ScanBatch b) {
    pdl_wait();
    const int v = blockIdx.y;
    scan_reduce_body(b.in[v], nullptr, b.d_n[v], b.block_sums[v]);
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_down_batch(ScanBatch b) {
    pdl_wait();
    const int v = blockIdx.y;
    scan_down_body(b.in[v], nullptr, b.out[v], b.d_n[v], b.block_sums[v], b.d_total[v]);
}
}  // namespace

int radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, const uint32_t *d_n,
                     uint32_t max_n, int begin_bit, int end_bit, uint32_t *hist, cudaStream_t st,
                     bool *result_in_alt) {
    bool alt = false;
    if (max_n == 0 || end_bit <= begin_bit) {
        *result_in_alt = false;
        return LODGS_OK;
    }
    // blocks: a fixed count for short sorts (the pass is latency-bound there);
    // long sorts get about 16 tiles per block, up to 8 blocks per SM
    const int G = (int)std::min<uint64_t>(SORT_GRID_MAX,
                                          std::max<uint64_t>(SORT_GRID, (uint64_t)max_n / (ST_TILE * 16)));
    for (int shift = begin_bit; shift < end_bit; shift += RADIX_BITS) {
        int bits = end_bit - shift < RADIX_BITS ? end_bit - shift : RADIX_BITS;
        uint32_t mask = (1u << bits) - 1u;
        const uint32_t *ki = alt ? keys_alt : keys;
        const uint32_t *vi = alt ? vals_alt : vals;
        uint32_t *ko = alt ? keys : keys_alt;
        uint32_t *vo = alt ? vals : vals_alt;
        uint32_t *totals = hist + RADIX * G;
        LODGS_CUDA(pdl_launch(k_radix_upsweep, G, ST_THREADS, st, ki, d_n, shift, mask, hist));
        count_launches(1);
        LODGS_CUDA(pdl_launch(k_digit_scan, RADIX / 8, 256, st, hist, G, totals));
        count_launches(1);
        LODGS_CUDA(pdl_launch(k_radix_downsweep, G, ST_THREADS, st, ki, vi, ko, vo, d_n, shift, mask, hist, totals));
        count_launches(1);
        alt = !alt;
    }
    LODGS_CUDA(cudaGetLastError());
    *result_in_alt = alt;
    return LODGS_OK;
}

int scan_exclusive_batch(const ScanBatch &b, int k, uint32_t max_n, cudaStream_t st) {
    if (k < 1 || k > SCAN_BATCH_MAX) { set_error("scan: batch size out of range"); return LODGS_E_INVALID; }
    if (max_n <= SCAN_ONE_BLOCK) {
        LODGS_CUDA(pdl_launch(k_scan_down_batch, dim3(1, k), SC_THREADS, st, b));
        count_launches(1);
        LODGS_CUDA(cudaGetLastError());
        return LODGS_OK;
    }
    const int G = (int)std::min<uint64_t>(SCAN_GRID_MAX, std::max<uint64_t>(SCAN_GRID, (uint64_t)max_n / (SC_TILE * 4)));
    LODGS_CUDA(pdl_launch(k_scan_reduce_batch, dim3(G, k), SC_THREADS, st, b));
    count_launches(1);
    LODGS_CUDA(pdl_launch(k_scan_down_batch, dim3(G, k), SC_THREADS, st, b));
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

int scan_exclusive(const uint32_t *in, uint32_t *out, const uint32_t *d_n, uint32_t max_n, uint32_t *block_sums,
                   uint32_t *d_total, cudaStream_t st, const uint32_t *idx) {
    if (max_n <= SCAN_ONE_BLOCK) {                 // short scans: one block, no block sums
        LODGS_CUDA(pdl_launch(k_scan_down, 1, SC_THREADS, st, in, idx, out, d_n, block_sums, d_total));
        count_launches(1);
        LODGS_CUDA(cudaGetLastError());
        return LODGS_OK;
    }
    // long scans: about four tiles per block, up to 8 blocks per SM
    const int G = (int)std::min<uint64_t>(SCAN_GRID_MAX, std::max<uint64_t>(SCAN_GRID, (uint64_t)max_n / (SC_TILE * 4)));
    LODGS_CUDA(pdl_launch(k_scan_reduce, G, SC_THREADS, st, in, idx, d_n, block_sums));
    count_launches(1);
    LODGS_CUDA(pdl_launch(k_scan_down, G, SC_THREADS, st, in, idx, out, d_n, block_sums, d_total));
    count_launches(1);
    LODGS_CUDA(cudaGetLastError());
    return LODGS_OK;
}

}  // namespace lodgs
