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
//             least-recently-used SPTs not used by this view) and cut at x_j.
// The reuse ratio is taken on x = tau d / f, i.e. on the focal-normalised
// distance, so cameras with different focal lengths share cached cuts.
#include <string.h>

#include <list>
#include <map>
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
    std::list<uint32_t>::iterator lru;
};

}  // namespace

struct lodgs_cache {
    lodgs_scene *scene = nullptr;
    uint32_t layout_version = 0;      // the scene layout the host copy and slab follow
    float d_min = 1.f, d_max = 1.f;
    uint64_t slab_records = 0;
    float *h_rows = nullptr;          // pinned, n_nodes x stride
    float *d_records = nullptr;       // device: upper rows then the slab
    std::vector<uint32_t> spt_base;   // host copy (n_spt + 1)
    std::vector<Entry> entry;
    std::list<uint32_t> lru;          // front = most recently used
    std::map<uint64_t, uint64_t> free_ranges;   // offset -> length
    uint64_t view = 0, cached_records = 0, cached_spts = 0;
    // pinned staging for the per-view decisions
    uint32_t *h_cnt = nullptr, *h_emit_j = nullptr, *h_high = nullptr, *h_src = nullptr;
    float *h_emit_x = nullptr, *h_x_used = nullptr;
    cudaEvent_t copies_done = nullptr;
};

namespace {

void range_free(lodgs_cache *c, uint64_t off, uint64_t len) {
    auto it = c->free_ranges.emplace(off, len).first;
    if (it != c->free_ranges.begin()) {                       // merge with the previous range
        auto p = std::prev(it);
        if (p->first + p->second == it->first) { p->second += it->second; c->free_ranges.erase(it); it = p; }
    }
    auto n = std::next(it);
    if (n != c->free_ranges.end() && it->first + it->second == n->first) {
        it->second += n->second;
        c->free_ranges.erase(n);
    }
}

bool range_alloc(lodgs_cache *c, uint64_t len, uint64_t *off) {
    for (auto it = c->free_ranges.begin(); it != c->free_ranges.end(); ++it)
        if (it->second >= len) {                              // first fit
            *off = it->first;
            uint64_t rest = it->second - len, at = it->first + len;
            c->free_ranges.erase(it);
            if (rest) c->free_ranges.emplace(at, rest);
            return true;
        }
    return false;
}

void evict(lodgs_cache *c, uint32_t j) {
    Entry &e = c->entry[j];
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
    c->free_ranges.emplace(0, c->slab_records);
    const size_t n = (size_t)std::max<int64_t>(S, 1);
    if ((e = cudaMallocHost((void **)&c->h_cnt, C_COUNT * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_emit_j, n * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_emit_x, n * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_high, n * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_x_used, n * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&c->h_src, n * 4)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->copies_done, cudaEventDisableTiming)) != cudaSuccess)
        return fail(cuda_fail(e, "cache_create: staging"));
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
    if (c->copies_done) cudaEventDestroy(c->copies_done);
    delete c;
}

int lodgs_cache_flush(lodgs_cache *c) {
    if (!c) { set_error("cache_flush: NULL cache"); return LODGS_E_INVALID; }
    for (Entry &e : c->entry) e.valid = false;
    c->lru.clear();
    c->free_ranges.clear();
    c->free_ranges.emplace(0, c->slab_records);
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
    if (c->layout_version != sc->layout_version) {
        set_error("stream_nodes: the cache was created before the scene was densified; create a new cache");
        return LODGS_E_STATE;
    }
    if (!(cam->width > 0 && cam->height > 0 && cam->fx > 0 && cam->fy > 0 && cam->tau > 0 && cam->znear > 0)) {
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
    // 2. cache decisions (host)
    c->view += 1;
    lodgs_stream_stats s{};
    const uint32_t n_emit = c->h_cnt[C_NEMIT];
    const size_t rec = (size_t)sc->stride * sizeof(float);
    const uint64_t U = (uint64_t)sc->n_upper_rows;
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
            evict(c, j);
        }
        uint64_t off = 0;
        while (!range_alloc(c, need, &off)) {                 // evict least recently used, never this view's
            if (c->lru.empty() || c->entry[c->lru.back()].used == c->view) {
                set_error("stream_nodes: the view's SPT records exceed the cache capacity");
                return LODGS_E_CAPACITY;
            }
            evict(c, c->lru.back());
            s.evictions += 1;
        }
        e.valid = true;
        e.x = x;
        e.h = need;
        e.off = off;
        c->lru.push_front(j);
        e.lru = c->lru.begin();
        e.used = c->view;
        c->cached_records += need;
        c->cached_spts += 1;
        const size_t bytes = (size_t)need * rec;
        LODGS_CUDA(cudaMemcpyAsync(c->d_records + (U + off) * sc->stride, c->h_rows + (size_t)c->spt_base[j] * sc->stride,
                                   bytes, cudaMemcpyHostToDevice, cs));
        s.bytes_streamed += (int64_t)bytes;
        s.spt_loaded += 1;
        c->h_x_used[q] = x;
        c->h_src[q] = (uint32_t)(U + off);
    }
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
    fr->selected = true;
    fr->rendered = false;
    s.cached_spts = (int64_t)c->cached_spts;
    s.cached_records = (int64_t)c->cached_records;
    if (stats) *stats = s;
    return LODGS_OK;
}

}  // extern "C"
