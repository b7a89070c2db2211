// a3: device node cache fed from pinned host memory (Sec. 4.4 "Caching on the
// GPU"; Eq. 7; Algorithm 3 cache steps).
//
// All records stay in pinned host memory in render-row order; the device holds
// the scene structure (upper hierarchy, SPT intervals), the upper hierarchy's
// records, and a slab of SPT records managed by a host-side LRU allocator.
// Because an SPT's entries are laid out by descending parent bound, every
// entry that a cut at distance x can select lies in the prefix [0, high(x)):
// a miss streams that one contiguous prefix with a single cudaMemcpyAsync on a
// copy stream (no host gather, no reorganisation on the device).
//
// Per view and per SPT root j of the upper cut, with x_j = tau d_j / f:
//   hit       cached and D_min <= x_j / x_cached <= D_max: render the cached
//             cut (the cut at x_cached), as the paper reuses cached SPT cuts;
//   resident  otherwise, if the cached prefix already covers high(x_j): cut at
//             x_j from device-resident records, no transfer;
//   load      otherwise copy the prefix [0, high(x_j)) into the slab (evicting
//             least-recently-used SPTs not used by this view) and cut at x_j;
//             a cached SPT whose prefix is too short keeps its records and
//             streams only the tail: in place when the slab after it is free,
//             else after a device-to-device move of the cached prefix.
// The reuse ratio is taken on x = tau d / f, i.e. on the focal-normalised
// distance, so cameras with different focal lengths share cached cuts.
//
// Training (Algorithm 3: optimise the cached nodes, write them back to host
// memory when the LRU evicts them, flush periodically; Adam state kept in host
// memory beside the records): a training cache mirrors the record slab with
// slabs of the Adam moments and step counts.  A load streams the prefix of all
// four arrays; a sparse Adam step updates the view's cached rows in place and
// flags each row it trained (and the view's SPTs); evicting a trained SPT
// copies its flagged rows of the four arrays back to host memory on the copy
// stream, ahead of any load that reuses the range (same stream, in order).
// Upper rows stay resident and are written back by lodgs_cache_writeback and
// lodgs_cache_flush.
#include <string.h>

#include <list>
#include <map>
#include <set>
#include <new>
#include <string>
#include <vector>

#include "lodgs_internal.cuh"

using namespace lodgs;

namespace {

struct Entry {
    bool valid = false;
    float x = 0.f;            // normalised distance of the cached cut
    uint32_t h = 0;           // cached prefix length (records)
    uint64_t off = 0;         // slab offset (records)
    uint64_t used = 0;        // last view that used the entry
    bool dirty = false;       // trained since it was loaded (training caches)
    std::list<uint32_t>::iterator lru;
};

// One contiguous copy between the device slab and pinned host memory (through
// its device address) or within the slab, in 16-byte units (4-byte units for
// step counts).  Spans are cut into pieces of at most 64 KiB, one CTA each.
struct Piece {
    const void *src;
    void *dst;
    uint32_t n;               // units
    uint32_t word;            // 1: 4-byte units, 0: 16-byte units
};
constexpr uint64_t PIECE_BYTES = 64 << 10;
constexpr int PIECE_THREADS = 256;

// Every piece of one phase in one launch: the host issues a few launches per
// view instead of one cudaMemcpyAsync per SPT and array, and reads of host
// memory keep several 16-byte requests in flight per thread.
__global__ void __launch_bounds__(PIECE_THREADS) k_copy_pieces(const Piece *__restrict__ pieces) {
    const Piece p = pieces[blockIdx.x];
    if (p.word) {
        const uint32_t *__restrict__ src = static_cast<const uint32_t *>(p.src);
        uint32_t *__restrict__ dst = static_cast<uint32_t *>(p.dst);
        for (uint32_t i = threadIdx.x; i < p.n; i += PIECE_THREADS) dst[i] = src[i];
    } else {
        const uint4 *__restrict__ src = static_cast<const uint4 *>(p.src);
        uint4 *__restrict__ dst = static_cast<uint4 *>(p.dst);
#pragma unroll 4
        for (uint32_t i = threadIdx.x; i < p.n; i += PIECE_THREADS) dst[i] = src[i];
    }
}

// Write-back of trained SPT prefixes (and of the upper rows) in two steps, so
// that the link carries write-backs and loads at the same time:
//  k_stage_rows  (copy stream) copies the slots of each span whose dirty flag
//                the Adam step set (record, m, v, step count) into a compact
//                device staging area with their host rows, and clears the
//                flags; the batch's moves and loads may then reuse the slots;
//  k_unstage_rows (the cache's write-back stream) copies the staged rows to
//                the pinned host arrays, while the loads run.
// One warp per row.  Bytes written back are added to *written.
struct RowSpan {
    uint64_t slot, host_row;
    uint32_t n, pad;
};
constexpr uint32_t SPAN_ROWS = 256;
constexpr int UNSTAGE_BLOCKS = 148 * 4;

struct Staging {
    uint4 *rec, *m, *v;       // capacity rows x quads each
    uint32_t *t, *host_row, *n;
};

__global__ void __launch_bounds__(PIECE_THREADS) k_stage_rows(
    const RowSpan *__restrict__ spans, int quads, const uint4 *__restrict__ rec, const uint4 *__restrict__ m,
    const uint4 *__restrict__ v, const uint32_t *__restrict__ t, uint32_t *__restrict__ dirty, Staging sg,
    unsigned long long *__restrict__ written) {
    const RowSpan sp = spans[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t rows = 0;
    for (uint32_t r = warp; r < sp.n; r += PIECE_THREADS / 32) {
        const uint64_t s = sp.slot + r;
        if (!dirty[s]) continue;                                  // warp-uniform
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(sg.n, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        for (int k = lane; k < 3 * quads; k += 32) {
            const int a = k / quads, o = k - a * quads;
            const uint4 *src = a == 0 ? rec : (a == 1 ? m : v);
            uint4 *dst = a == 0 ? sg.rec : (a == 1 ? sg.m : sg.v);
            dst[(size_t)i * quads + o] = src[s * quads + o];
        }
        if (lane == 0) {
            sg.t[i] = t[s];
            sg.host_row[i] = (uint32_t)(sp.host_row + r);
            dirty[s] = 0u;
            ++rows;
        }
    }
    if (lane == 0 && rows)
        atomicAdd(written, (unsigned long long)rows * (3ull * quads * 16ull + 4ull));
}

__global__ void __launch_bounds__(PIECE_THREADS) k_unstage_rows(Staging sg, int quads, uint4 *__restrict__ h_rec,
                                                                uint4 *__restrict__ h_m, uint4 *__restrict__ h_v,
                                                                uint32_t *__restrict__ h_t) {
    const uint32_t n = *sg.n;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (PIECE_THREADS / 32);
    for (uint32_t i = blockIdx.x * (PIECE_THREADS / 32) + (threadIdx.x >> 5); i < n; i += warps) {
        const size_t h = sg.host_row[i];
        for (int k = lane; k < 3 * quads; k += 32) {
            const int a = k / quads, o = k - a * quads;
            const uint4 *src = a == 0 ? sg.rec : (a == 1 ? sg.m : sg.v);
            uint4 *dst = a == 0 ? h_rec : (a == 1 ? h_m : h_v);
            dst[h * quads + o] = src[(size_t)i * quads + o];
        }
        if (lane == 0) h_t[h] = sg.t[i];
    }
}

// copy phases of one batch, issued after its masked write-backs (which read
// slab ranges that moves and loads of the same batch may overwrite): moves,
// whose source ranges are freed only after the batch, then loads
enum : int { PH_MOVE = 0, PH_LOAD = 1, PH_COUNT = 2 };

}  // namespace

struct lodgs_cache {
    lodgs_scene *scene = nullptr;
    uint32_t layout_version = 0;      // the scene layout the host copy and slab follow
    float d_min = 1.f, d_max = 1.f;
    uint64_t slab_records = 0;
    float *h_rows = nullptr;          // pinned, n_nodes x stride
    float *d_records = nullptr;       // device: upper rows then the slab
    // training: Adam moments and step counts, same layouts as h_rows / d_records
    bool train = false, upper_dirty = false;
    float *h_m = nullptr, *h_v = nullptr, *d_m = nullptr, *d_v = nullptr;
    uint32_t *h_t = nullptr, *d_t = nullptr;
    cudaEvent_t adam_done = nullptr;  // after the last Adam step (its stream is the caller's)
    // device addresses of the pinned host arrays (read and written by k_copy_pieces)
    float *hd_rows = nullptr, *hd_m = nullptr, *hd_v = nullptr;
    uint32_t *hd_t = nullptr;
    // pending copies of the current batch, and their staging
    std::vector<Piece> pend[PH_COUNT];
    Piece *h_pieces = nullptr, *d_pieces = nullptr;
    size_t pieces_cap = 0;
    cudaEvent_t pieces_done = nullptr;  // after the last batch's kernels (staging reusable)
    // training: per-slot trained flags (set by the Adam step), masked write-backs
    uint32_t *d_dirty = nullptr, *d_zeros = nullptr;
    unsigned long long *d_written = nullptr;      // bytes the write-backs copied
    std::vector<RowSpan> wb;
    RowSpan *h_spans = nullptr, *d_spans = nullptr;
    size_t spans_cap = 0;
    // staged write-backs: device staging area (stage_cap rows), the stream that
    // copies it to host memory, and events ordering the two
    Staging stage{};
    uint64_t stage_cap = 0;
    cudaStream_t wb_stream = nullptr;
    cudaEvent_t staged = nullptr, unstage_done = nullptr;
    bool unstage_pending = false;
    std::vector<uint32_t> spt_base;   // host copy (n_spt + 1)
    std::vector<Entry> entry;
    std::list<uint32_t> lru;          // front = most recently used
    std::map<uint64_t, uint64_t> free_ranges;   // offset -> length
    std::set<std::pair<uint64_t, uint64_t>> free_by_len;   // (length, offset) of the same ranges
    uint64_t view = 0, cached_records = 0, cached_spts = 0;
    // pinned staging for the per-view decisions
    uint32_t *h_cnt = nullptr, *h_emit_j = nullptr, *h_high = nullptr, *h_src = nullptr;
    float *h_emit_x = nullptr, *h_x_used = nullptr;
    cudaEvent_t copies_done = nullptr;
};

namespace {

// The slab's free space: ranges by offset (for merging neighbours) and by
// length (best fit in O(log n) however fragmented the slab is).
void range_put(lodgs_cache *c, uint64_t off, uint64_t len) {
    c->free_ranges.emplace(off, len);
    c->free_by_len.emplace(len, off);
}

void range_erase(lodgs_cache *c, std::map<uint64_t, uint64_t>::iterator it) {
    c->free_by_len.erase({it->second, it->first});
    c->free_ranges.erase(it);
}

void range_free(lodgs_cache *c, uint64_t off, uint64_t len) {
    auto n = c->free_ranges.lower_bound(off);
    if (n != c->free_ranges.begin()) {                       // merge with the previous range
        auto p = std::prev(n);
        if (p->first + p->second == off) {
            off = p->first;
            len += p->second;
            range_erase(c, p);
        }
    }
    if (n != c->free_ranges.end() && off + len == n->first) { // and with the next one
        len += n->second;
        range_erase(c, n);
    }
    range_put(c, off, len);
}

bool range_alloc(lodgs_cache *c, uint64_t len, uint64_t *off) {
    auto b = c->free_by_len.lower_bound({len, 0});           // best fit: the shortest range that holds len
    if (b == c->free_by_len.end()) return false;
    const uint64_t l = b->first, o = b->second;
    range_erase(c, c->free_ranges.find(o));
    if (l > len) range_put(c, o + len, l - len);
    *off = o;
    return true;
}

void add_span(std::vector<Piece> &v, const void *src, void *dst, uint64_t bytes, bool word) {
    const uint64_t unit = word ? 4 : 16;
    for (uint64_t o = 0; o < bytes; o += PIECE_BYTES) {
        const uint64_t b = std::min<uint64_t>(PIECE_BYTES, bytes - o);
        v.push_back({static_cast<const char *>(src) + o, static_cast<char *>(dst) + o, (uint32_t)(b / unit),
                     word ? 1u : 0u});
    }
}

// n records from slab slot `dev` to/from host row `host`, for the four arrays
// of a training cache (records only otherwise); rows are multiples of 16 bytes
void add_rows(lodgs_cache *c, int phase, uint64_t dev, uint64_t host, uint64_t n, bool to_host) {
    const size_t w = (size_t)c->scene->stride, bytes = n * w * 4;
    std::vector<Piece> &v = c->pend[phase];
    auto span = [&](float *d, float *h) {
        if (to_host) add_span(v, d + dev * w, h + host * w, bytes, false);
        else add_span(v, h + host * w, d + dev * w, bytes, false);
    };
    span(c->d_records, c->hd_rows);
    if (!c->train) return;
    span(c->d_m, c->hd_m);
    span(c->d_v, c->hd_v);
    if (to_host) {
        add_span(v, c->d_t + dev, c->hd_t + host, n * 4, true);
    } else {
        add_span(v, c->hd_t + host, c->d_t + dev, n * 4, true);
        for (uint64_t o = 0; o < n * 4; o += PIECE_BYTES)   // freshly loaded: not trained yet
            v.push_back({c->d_zeros, reinterpret_cast<char *>(c->d_dirty + dev) + o,
                         (uint32_t)(std::min<uint64_t>(PIECE_BYTES, n * 4 - o) / 4), 1u});
    }
}

// masked write-back of n slots from `slot` on to host rows from `host` on
void add_wb(lodgs_cache *c, uint64_t slot, uint64_t host, uint64_t n) {
    for (uint64_t o = 0; o < n; o += SPAN_ROWS)
        c->wb.push_back({slot + o, host + o, (uint32_t)std::min<uint64_t>(SPAN_ROWS, n - o), 0u});
}

// n slab records (and their Adam state) from slot src to slot dst
void add_move(lodgs_cache *c, uint64_t src, uint64_t dst, uint64_t n) {
    const size_t w = (size_t)c->scene->stride, bytes = n * w * 4;
    std::vector<Piece> &v = c->pend[PH_MOVE];
    add_span(v, c->d_records + src * w, c->d_records + dst * w, bytes, false);
    if (!c->train) return;
    add_span(v, c->d_m + src * w, c->d_m + dst * w, bytes, false);
    add_span(v, c->d_v + src * w, c->d_v + dst * w, bytes, false);
    add_span(v, c->d_t + src, c->d_t + dst, n * 4, true);
    add_span(v, c->d_dirty + src, c->d_dirty + dst, n * 4, true);
}

// issue the batch on `st`: one descriptor upload, one launch per non-empty phase
int issue_pieces(lodgs_cache *c, cudaStream_t st) {
    size_t total = 0;
    for (auto &v : c->pend) total += v.size();
    if (!total && c->wb.empty()) return LODGS_OK;
    LODGS_CUDA(cudaEventSynchronize(c->pieces_done));       // the staging of the last batch is free
    // the last batch's write-back to host memory ends before this batch's
    // copies: loads may read host rows it writes, and staging is reused
    if (c->unstage_pending) LODGS_CUDA(cudaStreamWaitEvent(st, c->unstage_done, 0));
    if (!c->wb.empty()) {                                    // masked write-backs go first
        const size_t n = c->wb.size();
        if (n > c->spans_cap) {
            cudaFreeHost(c->h_spans);
            cudaFree(c->d_spans);
            c->h_spans = nullptr;
            c->d_spans = nullptr;
            c->spans_cap = 0;
            const size_t cap = std::max<size_t>(n + n / 2, 1024);
            LODGS_CUDA(cudaMallocHost((void **)&c->h_spans, cap * sizeof(RowSpan)));
            LODGS_CUDA(cudaMalloc((void **)&c->d_spans, cap * sizeof(RowSpan)));
            c->spans_cap = cap;
        }
        memcpy(c->h_spans, c->wb.data(), n * sizeof(RowSpan));
        uint64_t rows = 0;                                   // at most the spans' slots are flagged
        for (const RowSpan &r : c->wb) rows += r.n;
        const int quads = c->scene->stride / 4;
        if (rows > c->stage_cap) {                           // the old area is idle: waited for above
            LODGS_CUDA(cudaStreamSynchronize(st));
            cudaFree(c->stage.rec); cudaFree(c->stage.m); cudaFree(c->stage.v);
            cudaFree(c->stage.t); cudaFree(c->stage.host_row); cudaFree(c->stage.n);
            c->stage = Staging{};
            c->stage_cap = 0;
            const uint64_t cap = std::max<uint64_t>(rows + rows / 2, 4096);
            const size_t rb = (size_t)cap * quads * sizeof(uint4);
            LODGS_CUDA(cudaMalloc((void **)&c->stage.rec, rb));
            LODGS_CUDA(cudaMalloc((void **)&c->stage.m, rb));
            LODGS_CUDA(cudaMalloc((void **)&c->stage.v, rb));
            LODGS_CUDA(cudaMalloc((void **)&c->stage.t, cap * 4));
            LODGS_CUDA(cudaMalloc((void **)&c->stage.host_row, cap * 4));
            LODGS_CUDA(cudaMalloc((void **)&c->stage.n, 4));
            c->stage_cap = cap;
        }
        LODGS_CUDA(cudaMemcpyAsync(c->d_spans, c->h_spans, n * sizeof(RowSpan), cudaMemcpyHostToDevice, st));
        LODGS_CUDA(cudaMemsetAsync(c->stage.n, 0, 4, st));
        k_stage_rows<<<(unsigned)n, PIECE_THREADS, 0, st>>>(
            c->d_spans, quads, reinterpret_cast<const uint4 *>(c->d_records), reinterpret_cast<const uint4 *>(c->d_m),
            reinterpret_cast<const uint4 *>(c->d_v), c->d_t, c->d_dirty, c->stage, c->d_written);
        LODGS_CUDA(cudaEventRecord(c->staged, st));
        LODGS_CUDA(cudaStreamWaitEvent(c->wb_stream, c->staged, 0));
        k_unstage_rows<<<UNSTAGE_BLOCKS, PIECE_THREADS, 0, c->wb_stream>>>(
            c->stage, quads, reinterpret_cast<uint4 *>(c->hd_rows), reinterpret_cast<uint4 *>(c->hd_m),
            reinterpret_cast<uint4 *>(c->hd_v), c->hd_t);
        LODGS_CUDA(cudaEventRecord(c->unstage_done, c->wb_stream));
        c->unstage_pending = true;
        count_launches(2);
        c->wb.clear();
    }
    if (!total) {
        LODGS_CUDA(cudaGetLastError());
        LODGS_CUDA(cudaEventRecord(c->pieces_done, st));
        return LODGS_OK;
    }
    if (total > c->pieces_cap) {
        cudaFreeHost(c->h_pieces);
        cudaFree(c->d_pieces);
        c->h_pieces = nullptr;
        c->d_pieces = nullptr;
        c->pieces_cap = 0;
        const size_t cap = std::max<size_t>(total + total / 2, 4096);
        LODGS_CUDA(cudaMallocHost((void **)&c->h_pieces, cap * sizeof(Piece)));
        LODGS_CUDA(cudaMalloc((void **)&c->d_pieces, cap * sizeof(Piece)));
        c->pieces_cap = cap;
    }
    size_t at = 0, start[PH_COUNT];
    for (int ph = 0; ph < PH_COUNT; ++ph) {
        start[ph] = at;
        if (!c->pend[ph].empty()) memcpy(c->h_pieces + at, c->pend[ph].data(), c->pend[ph].size() * sizeof(Piece));
        at += c->pend[ph].size();
    }
    LODGS_CUDA(cudaMemcpyAsync(c->d_pieces, c->h_pieces, total * sizeof(Piece), cudaMemcpyHostToDevice, st));
    for (int ph = 0; ph < PH_COUNT; ++ph) {
        const size_t n = c->pend[ph].size();
        if (!n) continue;
        k_copy_pieces<<<(unsigned)n, PIECE_THREADS, 0, st>>>(c->d_pieces + start[ph]);
        count_launches(1);
        c->pend[ph].clear();
    }
    LODGS_CUDA(cudaGetLastError());
    LODGS_CUDA(cudaEventRecord(c->pieces_done, st));
    return LODGS_OK;
}

// the records [at, at + len) if a free range starts exactly at `at` and holds them
bool range_take_at(lodgs_cache *c, uint64_t at, uint64_t len) {
    auto it = c->free_ranges.find(at);
    if (it == c->free_ranges.end() || it->second < len) return false;
    const uint64_t rest = it->second - len;
    range_erase(c, it);
    if (rest) range_put(c, at + len, rest);
    return true;
}

// drop SPT j from the cache; a dirty prefix is first queued for write-back to
// host memory (the batch's first phase, ahead of any copy into the range)
void evict(lodgs_cache *c, uint32_t j, int64_t *written) {
    Entry &e = c->entry[j];
    if (e.dirty) {
        const uint64_t U = (uint64_t)c->scene->n_upper_rows;
        add_wb(c, U + e.off, c->spt_base[j], e.h);
        if (written) *written += (int64_t)e.h * c->scene->stride * 4 * (c->train ? 3 : 1) + (c->train ? e.h * 4 : 0);
        e.dirty = false;
    }
    range_free(c, e.off, e.h);
    c->lru.erase(e.lru);
    c->cached_records -= e.h;
    c->cached_spts -= 1;
    e.valid = false;
}

void touch(lodgs_cache *c, uint32_t j) {
    Entry &e = c->entry[j];
    c->lru.erase(e.lru);
    c->lru.push_front(j);
    e.lru = c->lru.begin();
    e.used = c->view;
}

}  // namespace

extern "C" {

int lodgs_cache_create(lodgs_scene *sc, const lodgs_cache_params *p, lodgs_cache **out) {
    if (!sc || !p || !out) { set_error("cache_create: NULL argument"); return LODGS_E_INVALID; }
    *out = nullptr;
    if (!sc->d_rows) { set_error("cache_create: the scene's records are not on the device"); return LODGS_E_STATE; }
    if (!(p->d_min > 0 && p->d_max >= p->d_min) || p->capacity_bytes <= 0) {
        set_error("cache_create: need 0 < d_min <= d_max and capacity_bytes > 0");
        return LODGS_E_INVALID;
    }
    lodgs_cache *c = new (std::nothrow) lodgs_cache();
    if (!c) { set_error("cache_create: host allocation failed"); return LODGS_E_OOM; }
    c->scene = sc;
    c->layout_version = sc->layout_version;
    c->d_min = p->d_min;
    c->d_max = p->d_max;
    const size_t rec = (size_t)sc->stride * sizeof(float);
    c->slab_records = (uint64_t)p->capacity_bytes / rec;
    const int64_t M = sc->n_nodes, S = sc->n_spt, U = sc->n_upper_rows;
    auto fail = [&](int rc) { lodgs_cache_free(c); return rc; };
    cudaError_t e = cudaMallocHost((void **)&c->h_rows, (size_t)M * rec);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cache_create: pinned host records"));
    e = cudaMemcpy(c->h_rows, sc->d_rows, (size_t)M * rec, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cache_create: copy records to host"));
    e = cudaMalloc((void **)&c->d_records, (size_t)(U + c->slab_records) * rec);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cache_create: device cache"));
    if (U) {
        e = cudaMemcpy(c->d_records, sc->d_rows, (size_t)U * rec, cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cache_create: upper rows"));
    }
    c->spt_base.resize(S + 1);
    e = cudaMemcpy(c->spt_base.data(), sc->d_spt_base, (S + 1) * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cache_create: SPT bases"));
    c->entry.resize(S);
    range_put(c, 0, c->slab_records);
    if ((e = cudaHostGetDevicePointer((void **)&c->hd_rows, c->h_rows, 0)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->pieces_done, cudaEventDisableTiming)) != cudaSuccess)
        return fail(cuda_fail(e, "cache_create: device address of the host records"));
    const size_t n = (size_t)std::max<int64_t>(S, 1);
    if ((e = cudaMallocHost((void **)&c->h_cnt, C_COUNT * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_emit_j, n * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_emit_x, n * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_high, n * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_x_used, n * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_src, n * 4)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->copies_done, cudaEventDisableTiming)) != cudaSuccess)
        return fail(cuda_fail(e, "cache_create: staging"));
    if (p->train) {
        const size_t slots = (size_t)(U + c->slab_records);
        c->train = true;
        if ((e = cudaMallocHost((void **)&c->h_m, (size_t)M * rec)) != cudaSuccess ||
            (e = cudaMallocHost((void **)&c->h_v, (size_t)M * rec)) != cudaSuccess ||
            (e = cudaMallocHost((void **)&c->h_t, (size_t)std::max<int64_t>(M, 1) * 4)) != cudaSuccess)
            return fail(cuda_fail(e, "cache_create: pinned Adam state"));
        memset(c->h_m, 0, (size_t)M * rec);
        memset(c->h_v, 0, (size_t)M * rec);
        memset(c->h_t, 0, (size_t)M * 4);
        if ((e = cudaHostGetDevicePointer((void **)&c->hd_m, c->h_m, 0)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer((void **)&c->hd_v, c->h_v, 0)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer((void **)&c->hd_t, c->h_t, 0)) != cudaSuccess)
            return fail(cuda_fail(e, "cache_create: device address of the host Adam state"));
        if ((e = cudaMalloc((void **)&c->d_m, slots * rec)) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_v, slots * rec)) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_t, std::max<size_t>(slots, 1) * 4)) != cudaSuccess)
            return fail(cuda_fail(e, "cache_create: device Adam state"));
        if ((e = cudaMemset(c->d_m, 0, (size_t)U * rec)) != cudaSuccess ||
            (e = cudaMemset(c->d_v, 0, (size_t)U * rec)) != cudaSuccess ||
            (e = cudaMemset(c->d_t, 0, (size_t)U * 4)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c->adam_done, cudaEventDisableTiming)) != cudaSuccess)
            return fail(cuda_fail(e, "cache_create: upper Adam state"));
        if ((e = cudaMalloc((void **)&c->d_dirty, std::max<size_t>(slots, 1) * 4)) != cudaSuccess ||
            (e = cudaMemset(c->d_dirty, 0, std::max<size_t>(slots, 1) * 4)) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_zeros, PIECE_BYTES)) != cudaSuccess ||
            (e = cudaMemset(c->d_zeros, 0, PIECE_BYTES)) != cudaSuccess ||
            (e = cudaMalloc((void **)&c->d_written, 8)) != cudaSuccess ||
            (e = cudaMemset(c->d_written, 0, 8)) != cudaSuccess)
            return fail(cuda_fail(e, "cache_create: trained-row flags"));
        if ((e = cudaStreamCreateWithFlags(&c->wb_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c->staged, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c->unstage_done, cudaEventDisableTiming)) != cudaSuccess)
            return fail(cuda_fail(e, "cache_create: write-back stream"));
    }
    if (p->release_scene_rows) {
        cudaFree(sc->d_rows);
        sc->d_rows = nullptr;
    }
    *out = c;
    return LODGS_OK;
}

void lodgs_cache_free(lodgs_cache *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    cudaFreeHost(c->h_rows);
    cudaFree(c->d_records);
    cudaFreeHost(c->h_cnt); cudaFreeHost(c->h_emit_j); cudaFreeHost(c->h_emit_x); cudaFreeHost(c->h_high);
    cudaFreeHost(c->h_x_used); cudaFreeHost(c->h_src);
    cudaFreeHost(c->h_m); cudaFreeHost(c->h_v); cudaFreeHost(c->h_t);
    cudaFree(c->d_m); cudaFree(c->d_v); cudaFree(c->d_t);
    if (c->copies_done) cudaEventDestroy(c->copies_done);
    if (c->adam_done) cudaEventDestroy(c->adam_done);
    if (c->pieces_done) cudaEventDestroy(c->pieces_done);
    cudaFreeHost(c->h_pieces);
    cudaFree(c->d_pieces);
    cudaFreeHost(c->h_spans);
    cudaFree(c->d_spans);
    cudaFree(c->d_dirty);
    cudaFree(c->d_zeros);
    cudaFree(c->d_written);
    cudaFree(c->stage.rec); cudaFree(c->stage.m); cudaFree(c->stage.v);
    cudaFree(c->stage.t); cudaFree(c->stage.host_row); cudaFree(c->stage.n);
    if (c->staged) cudaEventDestroy(c->staged);
    if (c->unstage_done) cudaEventDestroy(c->unstage_done);
    if (c->wb_stream) cudaStreamDestroy(c->wb_stream);
    delete c;
}

namespace {
// write every dirty SPT prefix and the upper rows back to host memory on `st`
int writeback_all(lodgs_cache *c, cudaStream_t st) {
    if (!c->train) return LODGS_OK;
    LODGS_CUDA(cudaStreamWaitEvent(st, c->adam_done, 0));
    const uint64_t U = (uint64_t)c->scene->n_upper_rows;
    const uint64_t M = (uint64_t)c->scene->n_nodes;
    for (uint32_t j = 0; j < (uint32_t)c->entry.size(); ++j) {
        Entry &e = c->entry[j];
        if (!e.valid || !e.dirty) continue;
        add_wb(c, U + e.off, c->spt_base[j], e.h);
        e.dirty = false;
    }
    if (U && c->upper_dirty) {
        add_wb(c, 0, 0, U);
        c->upper_dirty = false;
    }
    (void)M;
    if (int rc = issue_pieces(c, st)) return rc;
    if (c->unstage_pending) LODGS_CUDA(cudaStreamWaitEvent(st, c->unstage_done, 0));   // host rows written
    return LODGS_OK;
}
}  // namespace

int lodgs_cache_writeback(lodgs_cache *c, void *stream) {
    if (!c) { set_error("cache_writeback: NULL cache"); return LODGS_E_INVALID; }
    return writeback_all(c, (cudaStream_t)stream);
}

int lodgs_cache_written_bytes(lodgs_cache *c, int64_t *bytes) {
    if (!c || !bytes) { set_error("cache_written_bytes: NULL argument"); return LODGS_E_INVALID; }
    *bytes = 0;
    if (!c->train) return LODGS_OK;
    LODGS_CUDA(cudaDeviceSynchronize());
    unsigned long long b = 0;
    LODGS_CUDA(cudaMemcpy(&b, c->d_written, 8, cudaMemcpyDeviceToHost));
    *bytes = (int64_t)b;
    return LODGS_OK;
}

int lodgs_cache_host_state(lodgs_cache *c, float **h_rows, float **h_m, float **h_v, uint32_t **h_t) {
    if (!c) { set_error("cache_host_state: NULL cache"); return LODGS_E_INVALID; }
    if (h_rows) *h_rows = c->h_rows;
    if (h_m) *h_m = c->h_m;
    if (h_v) *h_v = c->h_v;
    if (h_t) *h_t = c->h_t;
    return LODGS_OK;
}

int lodgs_cache_adam_step(lodgs_cache *c, lodgs_frame *fr, const float *grads, int64_t grad_capacity,
                          const float *lr, float b1, float b2, float eps, void *stream) {
    if (!c || !fr || !grads || !lr || grad_capacity < 0) {
        set_error("cache_adam_step: NULL argument or negative capacity");
        return LODGS_E_INVALID;
    }
    if (!c->train) { set_error("cache_adam_step: the cache was not created for training"); return LODGS_E_STATE; }
    if (int rc = check_frame(c->scene, fr, "cache_adam_step")) return rc;
    if (fr->cache != c || fr->cache_view != c->view || !fr->blend_bwd_done) {
        set_error("cache_adam_step: the frame must hold this cache's latest view, rendered and back-propagated");
        return LODGS_E_STATE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const FrameBufs &f = fr->f;
    const int64_t max_n = std::min<int64_t>((int64_t)f.cap_sel, grad_capacity);
    if (int rc = launch_adam(c->scene, c->d_records, c->d_m, c->d_v, c->d_t, f.sel_src, grads, f.cnt + C_NSEL_EFF,
                             max_n, lr, b1, b2, eps, st, c->d_dirty))
        return rc;
    LODGS_CUDA(cudaEventRecord(c->adam_done, st));
    for (Entry &e : c->entry)
        if (e.valid && e.used == c->view) e.dirty = true;
    c->upper_dirty = true;
    return LODGS_OK;
}

int lodgs_cache_flush(lodgs_cache *c) {
    if (!c) { set_error("cache_flush: NULL cache"); return LODGS_E_INVALID; }
    if (c->train) {                                  // trained rows and state go home first
        LODGS_CUDA(cudaDeviceSynchronize());
        if (int rc = writeback_all(c, 0)) return rc;
        LODGS_CUDA(cudaStreamSynchronize(0));
    }
    for (Entry &e : c->entry) e.valid = false;
    c->lru.clear();
    c->free_ranges.clear();
    c->free_by_len.clear();
    range_put(c, 0, c->slab_records);
    c->cached_records = 0;
    c->cached_spts = 0;
    return LODGS_OK;
}

int lodgs_cache_records(lodgs_cache *c, float **d_records) {
    if (!c || !d_records) { set_error("cache_records: NULL argument"); return LODGS_E_INVALID; }
    *d_records = c->d_records;
    return LODGS_OK;
}

int lodgs_stream_nodes(lodgs_scene *sc, lodgs_cache *c, const lodgs_camera *cam, lodgs_frame *fr, void *stream,
                       void *copy_stream, lodgs_stream_stats *stats) {
    if (!c || !cam || c->scene != sc) {
        set_error("stream_nodes: NULL or mismatched argument");
        return LODGS_E_INVALID;
    }
    if (int rc = check_frame(sc, fr, "stream_nodes")) return rc;
    if (fault_hit(LODGS_FAULT_STREAM)) {                    // before any cache or frame state changes
        set_error("stream_nodes: injected copy failure");
        return LODGS_E_CUDA;
    }
    if (c->layout_version != sc->layout_version) {
        set_error("stream_nodes: the cache was created before the scene was densified; create a new cache");
        return LODGS_E_STATE;
    }
    if (!camera_ok(cam)) {
        set_error("stream_nodes: invalid camera");
        return LODGS_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
    FrameBufs &f = fr->f;
    const int64_t M = sc->n_nodes, S = sc->n_spt;
    if (!f.sel_src) LODGS_CUDA(cudaMalloc((void **)&f.sel_src, (size_t)std::max<int64_t>(M, 1) * 4));
    if (!f.emit_src) LODGS_CUDA(cudaMalloc((void **)&f.emit_src, (size_t)std::max<int64_t>(S, 1) * 4));
    fr->stream = st;
    for (bool &r : fr->ran) r = false;
    fr->mark(LODGS_STAGE_SELECT, 0, st);
    if (int rc = lodgs_frame_set_view(fr, cam, nullptr, stream)) return rc;
    LODGS_CUDA(cudaMemsetAsync(f.cnt, 0, C_COUNT * sizeof(uint32_t), st));
    // 1. upper cut and, per SPT root, the prefix needed at the current distance
    if (int rc = launch_select_upper(sc, f, true, st)) return rc;
    if (int rc = launch_spt_high(sc, f, st)) return rc;
    const size_t n = (size_t)std::max<int64_t>(S, 1);
    LODGS_CUDA(cudaMemcpyAsync(c->h_cnt, f.cnt, C_COUNT * 4, cudaMemcpyDeviceToHost, st));
    LODGS_CUDA(cudaMemcpyAsync(c->h_emit_j, f.emit_j, n * 4, cudaMemcpyDeviceToHost, st));
    LODGS_CUDA(cudaMemcpyAsync(c->h_emit_x, f.emit_x, n * 4, cudaMemcpyDeviceToHost, st));
    LODGS_CUDA(cudaMemcpyAsync(c->h_high, f.high, n * 4, cudaMemcpyDeviceToHost, st));
    // this also waits for earlier renders on `st`, which may read slab ranges evicted below
    LODGS_CUDA(cudaStreamSynchronize(st));
    // 2. cache decisions (host); write-backs read rows the last Adam step wrote
    if (c->train) LODGS_CUDA(cudaStreamWaitEvent(cs, c->adam_done, 0));
    c->view += 1;
    lodgs_stream_stats s{};
    const uint32_t n_emit = c->h_cnt[C_NEMIT];
    const size_t rec = (size_t)sc->stride * sizeof(float);
    const uint64_t U = (uint64_t)sc->n_upper_rows;
    std::vector<std::pair<uint64_t, uint64_t>> moved_from;   // slab ranges vacated by moves
    for (uint32_t q = 0; q < n_emit; ++q) {
        const uint32_t j = c->h_emit_j[q];
        const float x = c->h_emit_x[q];
        const uint32_t need = c->h_high[q];
        Entry &e = c->entry[j];
        if (e.valid) {
            const float ratio = x / e.x;
            if (ratio >= c->d_min && ratio <= c->d_max) {
                touch(c, j);
                c->h_x_used[q] = e.x;
                c->h_src[q] = (uint32_t)(U + e.off);
                s.spt_hits += 1;
                continue;
            }
            if (e.h >= need) {
                touch(c, j);
                e.x = x;
                c->h_x_used[q] = x;
                c->h_src[q] = (uint32_t)(U + e.off);
                s.spt_resident += 1;
                continue;
            }
        }
        const size_t per = c->train ? 3 * rec + 4 : rec;    // bytes a record streams
        // slab space for `len` records, evicting least recently used SPTs (never this view's)
        auto alloc = [&](uint64_t len, uint64_t *at) -> int {
            while (!range_alloc(c, len, at)) {
                if (c->lru.empty() || c->entry[c->lru.back()].used == c->view) {
                    set_error("stream_nodes: the view's SPT records exceed the cache capacity");
                    return LODGS_E_CAPACITY;
                }
                evict(c, c->lru.back(), &s.bytes_written_back);
                s.evictions += 1;
            }
            return LODGS_OK;
        };
        if (e.valid) {
            // a longer prefix of a cached SPT: keep the cached records (trained
            // or not) and stream only the tail, in place when the slab after the
            // prefix is free, else after moving the prefix on the device
            const uint64_t grow = need - e.h;
            touch(c, j);
            if (!range_take_at(c, e.off + e.h, grow)) {
                uint64_t off = 0;
                if (int rc = alloc(need, &off)) return rc;
                add_move(c, U + e.off, U + off, e.h);
                moved_from.emplace_back(e.off, e.h);      // freed once the batch is queued
                e.off = off;
            }
            add_rows(c, PH_LOAD, U + e.off + e.h, c->spt_base[j] + e.h, grow, false);
            c->cached_records += grow;
            e.h = need;
            e.x = x;
            s.bytes_streamed += (int64_t)(grow * per);
            s.spt_loaded += 1;
            c->h_x_used[q] = x;
            c->h_src[q] = (uint32_t)(U + e.off);
            continue;
        }
        uint64_t off = 0;
        if (int rc = alloc(need, &off)) return rc;
        e.valid = true;
        e.dirty = false;
        e.x = x;
        e.h = need;
        e.off = off;
        c->lru.push_front(j);
        e.lru = c->lru.begin();
        e.used = c->view;
        c->cached_records += need;
        c->cached_spts += 1;
        add_rows(c, PH_LOAD, U + off, c->spt_base[j], need, false);
        s.bytes_streamed += (int64_t)(need * per);
        s.spt_loaded += 1;
        c->h_x_used[q] = x;
        c->h_src[q] = (uint32_t)(U + off);
    }
    // the batch: write-backs, then moves, then loads, all on the copy stream
    if (int rc = issue_pieces(c, cs)) return rc;
    for (auto &r : moved_from) range_free(c, r.first, r.second);
    LODGS_CUDA(cudaEventRecord(c->copies_done, cs));
    // 3. SPT cut at the chosen distances, with the slab slot of every record
    if (n_emit) {
        LODGS_CUDA(cudaMemcpyAsync(f.emit_x, c->h_x_used, n_emit * 4, cudaMemcpyHostToDevice, st));
        LODGS_CUDA(cudaMemcpyAsync(f.emit_src, c->h_src, n_emit * 4, cudaMemcpyHostToDevice, st));
    }
    if (int rc = launch_spt_high(sc, f, st)) return rc;
    if (int rc = launch_select_spt(sc, f, true, st)) return rc;
    LODGS_CUDA(cudaStreamWaitEvent(st, c->copies_done, 0));   // the render reads the streamed records
    fr->mark(LODGS_STAGE_SELECT, 1, st);
    f.use_src = true;
    fr->cache = c;
    fr->cache_view = c->view;
    fr->selected = true;
    fr->rendered = false;
    s.cached_spts = (int64_t)c->cached_spts;
    s.cached_records = (int64_t)c->cached_records;
    if (stats) *stats = s;
    return LODGS_OK;
}

}  // extern "C"
