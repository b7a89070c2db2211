// C ABI of liblodgs: argument checks, scene and frame lifetime, workspace
// growth, and the order of the per-view stages.  No exception crosses the ABI.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lodgs_internal.cuh"

namespace lodgs {

static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// host-side fault injection (tests of the error paths; nothing faults on the device)
static std::atomic<int64_t> g_fault[LODGS_FAULT_SITES + 1];
static struct FaultInit {
    FaultInit() { for (auto &f : g_fault) f.store(-1); }
} g_fault_init;

bool fault_hit(int site) {
    int64_t c = g_fault[site].load();
    while (c >= 0) {
        const int64_t next = c == 0 ? -1 : c - 1;
        if (g_fault[site].compare_exchange_weak(c, next)) return c == 0;
    }
    return false;
}

void set_error(const std::string &msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LODGS_E_OOM : LODGS_E_CUDA;
}

int launch_priority_high() {
    static const int prio = [] {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
        return greatest;
    }();
    return prio;
}

static int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        dev = 0;
    }
    return dev;
}

int device_sms() {
    static std::mutex mu;
    static std::map<int, int> cache;
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(mu);
    const auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 148;
    }
    cache.emplace(dev, sms);
    return sms;
}

int resident_blocks(const void *kern, int threads) {
    static std::mutex mu;
    static std::map<std::pair<int, std::pair<const void *, int>>, int> cache;
    const int dev = current_device();
    const int sms = device_sms();
    const auto key = std::make_pair(dev, std::make_pair(kern, threads));
    std::lock_guard<std::mutex> lock(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();   // a grid of one block per SM is still correct
        per_sm = 1;
    }
    cache.emplace(key, sms * per_sm);
    return sms * per_sm;
}

// Camera constants in float32 (host).  The LoD test compares tau*d/f with the
// node size; culling uses the four side planes through the camera centre and
// the near plane; the EWA Jacobian is clamped at 1.3x the half field of view.
CamK make_camk(const lodgs_camera &c) {
    CamK k;
    memcpy(k.R, c.R, sizeof(k.R));
    memcpy(k.pos, c.pos, sizeof(k.pos));
    k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy;
    k.W = c.width; k.H = c.height;
    k.TX = (c.width + TILE - 1) / TILE;
    k.TY = (c.height + TILE - 1) / TILE;
    k.znear = c.znear;
    k.inv_k = c.tau / c.fx;
    k.spt_scale = c.spt_scale > 0.0f ? c.spt_scale : 1.0f;
    float fW = (float)c.width, fH = (float)c.height;
    k.limx = 1.3f * ((0.5f * fW) / c.fx);
    k.limy = 1.3f * ((0.5f * fH) / c.fy);
    float l = sqrtf(c.fx * c.fx + c.cx * c.cx);
    k.plane[0][0] = c.fx / l; k.plane[0][1] = 0.0f; k.plane[0][2] = c.cx / l;
    float wr = fW - c.cx;
    l = sqrtf(c.fx * c.fx + wr * wr);
    k.plane[1][0] = -c.fx / l; k.plane[1][1] = 0.0f; k.plane[1][2] = wr / l;
    l = sqrtf(c.fy * c.fy + c.cy * c.cy);
    k.plane[2][0] = 0.0f; k.plane[2][1] = c.fy / l; k.plane[2][2] = c.cy / l;
    float hb = fH - c.cy;
    l = sqrtf(c.fy * c.fy + hb * hb);
    k.plane[3][0] = 0.0f; k.plane[3][1] = -c.fy / l; k.plane[3][2] = hb / l;
    return k;
}

}  // namespace lodgs

using namespace lodgs;


namespace lodgs {
bool camera_ok(const lodgs_camera *c) {
    return c && c->width > 0 && c->height > 0 && c->width <= 65535 * TILE && c->height <= 65535 * TILE &&
           c->fx > 0 && c->fy > 0 && c->tau > 0 && c->znear > 0 && isfinite(c->fx) && isfinite(c->fy) &&
           isfinite(c->cx) && isfinite(c->cy) && isfinite(c->tau) && isfinite(c->spt_scale) && c->spt_scale >= 0;
}
}  // namespace lodgs

namespace {

template <typename T>
int grow(T *&p, uint64_t &cap, uint64_t want, size_t elem_per = 1) {
    if (want <= cap && p) return LODGS_OK;
    if (fault_hit(LODGS_FAULT_ALLOC)) {                     // before the old buffer is released
        set_error("frame workspace: injected allocation failure");
        return LODGS_E_OOM;
    }
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    LODGS_CUDA(cudaMalloc((void **)&p, std::max<uint64_t>(want, 1) * elem_per * sizeof(T)));
    cap = want;
    return LODGS_OK;
}

int ensure_sel(lodgs_frame *fr, uint64_t want) {
    FrameBufs &f = fr->f;
    if (want <= f.cap_sel && f.sp_a) return LODGS_OK;
    want = std::min<uint64_t>(std::max<uint64_t>(want, 1024), (uint64_t)fr->scene->n_nodes);
    uint64_t c;
#define G1(ptr, per)                                  \
    c = f.cap_sel;                                    \
    if (int r_ = grow(ptr, c, want, per)) return r_;
    G1(f.sp_a, 1) G1(f.sp_b, 1) G1(f.sp_c, 1) G1(f.dkey, 1) G1(f.dval, 1) G1(f.dkey_alt, 1) G1(f.dval_alt, 1)
    G1(f.rect, 1) G1(f.ntiles, 1) G1(f.pair_off, 1) G1(f.g2d, G2D_STRIDE)
#undef G1
    f.cap_sel = want;
    return LODGS_OK;
}

int ensure_pairs(lodgs_frame *fr, uint64_t want) {
    FrameBufs &f = fr->f;
    if (want <= f.cap_pairs && f.pkey) return LODGS_OK;
    want = std::max<uint64_t>(want, 1 << 16);
    if (want > 0xffffffffull) { set_error("render: more than 2^32 (Gaussian, tile) pairs"); return LODGS_E_INVALID; }
    uint64_t c;
    c = f.cap_pairs; if (int r = grow(f.pkey, c, want)) return r;
    c = f.cap_pairs; if (int r = grow(f.pval, c, want)) return r;
    c = f.cap_pairs; if (int r = grow(f.pscratch, c, want)) return r;
    c = f.cap_pairs; if (int r = grow(f.pkey_alt, c, want)) return r;
    c = f.cap_pairs; if (int r = grow(f.pval_alt, c, want)) return r;
    c = f.cap_keep; if (int r = grow(f.keep, c, want / 16 + 1)) return r;   // rectangle pairs up to 2x kept
    f.cap_keep = c;
    f.cap_pairs = want;
    return LODGS_OK;
}

void free_frame_bufs(FrameBufs &f) {
    void *ps[] = {f.cnt, f.d_view, f.sel_rows, f.emit_j, f.high, f.work_off, f.emit_x, f.block_counts, f.scan_bsum,
                  f.sort_hist, f.sp_a, f.sp_b, f.sp_c, f.dkey, f.dval, f.dkey_alt, f.dval_alt, f.rect, f.ntiles,
                  f.pair_off, f.g2d, f.pkey, f.pval, f.pscratch, f.pkey_alt, f.pval_alt, f.ranges, f.tile_cnt,
                  f.tile_order, f.keep, f.work,
                  f.sel_src, f.emit_src, f.up_out, f.up_x};
    for (void *p : ps)
        if (p) cudaFree(p);
    f = FrameBufs();
}

}  // namespace

namespace {

// Upload the frame's view (camera constants and background) on `st`.
int set_view(lodgs_frame *fr, const lodgs_camera *cam, const float *bg, cudaStream_t st, bool zero_counters = false) {
    if (cam) fr->k = make_camk(*cam);
    if (bg) { fr->bg[0] = bg[0]; fr->bg[1] = bg[1]; fr->bg[2] = bg[2]; }
    View v;
    v.k = fr->k;
    v.bg[0] = fr->bg[0]; v.bg[1] = fr->bg[1]; v.bg[2] = fr->bg[2]; v.bg[3] = 0.f;
    int rc = launch_set_view(v, fr->f.d_view, st, zero_counters ? fr->f.cnt : nullptr);
    if (!rc) fr->have_view = true;
    return rc;
}

}  // namespace

namespace lodgs {
int check_frame(const lodgs_scene *sc, const lodgs_frame *fr, const char *who) {
    if (!sc || !fr || fr->scene != sc) {
        set_error(std::string(who) + ": frame does not belong to scene");
        return LODGS_E_INVALID;
    }
    if (fr->layout_version != sc->layout_version) {
        set_error(std::string(who) + ": the frame was created before the scene was densified; create a new frame");
        return LODGS_E_STATE;
    }
    return LODGS_OK;
}
}  // namespace lodgs

extern "C" {

const char *lodgs_last_error(void) { return g_err.c_str(); }

int lodgs_debug_inject_fault(int site, int64_t after) {
    if (site < 1 || site > LODGS_FAULT_SITES) { set_error("debug_inject_fault: unknown site"); return LODGS_E_INVALID; }
    g_fault[site].store(after < 0 ? -1 : after);
    return LODGS_OK;
}
const char *lodgs_version(void) { return "lodgs 0.1 (sm_103a)"; }
uint64_t lodgs_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int lodgs_build_hierarchy(const float *leaves, int64_t n, int sh_degree, int leaves_on_device,
                          const lodgs_build_params *params, lodgs_scene **out) {
    if (!out) { set_error("build_hierarchy: out is NULL"); return LODGS_E_INVALID; }
    *out = nullptr;
    if (!leaves || n < 1 || sh_degree < 0 || sh_degree > 3 || !params) {
        set_error("build_hierarchy: need leaves, n >= 1, 0 <= sh_degree <= 3, params");
        return LODGS_E_INVALID;
    }
    if (!(params->spt_volume > 0) || !(params->kappa > 0)) {
        set_error("build_hierarchy: spt_volume and kappa must be > 0");
        return LODGS_E_INVALID;
    }
    lodgs_scene *sc = new (std::nothrow) lodgs_scene();
    if (!sc) { set_error("build_hierarchy: host allocation failed"); return LODGS_E_OOM; }
    int rc = build_scene(leaves, n, sh_degree, leaves_on_device, *params, sc);
    if (rc) {
        free_scene(sc);
        delete sc;
        return rc;
    }
    *out = sc;
    return LODGS_OK;
}

void lodgs_scene_free(lodgs_scene *scene) {
    if (!scene) return;
    free_scene(scene);
    delete scene;
}

int lodgs_scene_get_info(const lodgs_scene *sc, lodgs_scene_info *info) {
    if (!sc || !info) { set_error("scene_get_info: NULL argument"); return LODGS_E_INVALID; }
    info->n_leaves = sc->n_leaves; info->n_nodes = sc->n_nodes; info->n_upper = sc->n_upper;
    info->n_upper_rows = sc->n_upper_rows; info->n_spt = sc->n_spt;
    info->sh_degree = sc->sh_degree; info->stride = sc->stride; info->d_rows = sc->d_rows;
    info->root = sc->root; info->layout_version = sc->layout_version;
    return LODGS_OK;
}

int lodgs_scene_save(const lodgs_scene *sc, const char *path) {
    if (!sc || !path) { set_error("scene_save: NULL argument"); return LODGS_E_INVALID; }
    return save_scene(sc, path);
}

int lodgs_scene_load(const char *path, lodgs_scene **out) {
    if (!path || !out) { set_error("scene_load: NULL argument"); return LODGS_E_INVALID; }
    *out = nullptr;
    lodgs_scene *sc = new (std::nothrow) lodgs_scene();
    if (!sc) { set_error("scene_load: host allocation failed"); return LODGS_E_OOM; }
    int rc = load_scene(path, sc);
    if (rc) {
        free_scene(sc);
        delete sc;
        return rc;
    }
    *out = sc;
    return LODGS_OK;
}

int lodgs_scene_densify(lodgs_scene *sc, const lodgs_densify_op *ops, int64_t n_ops, int32_t *old_row_of_new_row,
                        int64_t capacity) {
    if (!sc || (n_ops > 0 && !ops) || n_ops < 0 || !old_row_of_new_row) {
        set_error("scene_densify: NULL or negative argument");
        return LODGS_E_INVALID;
    }
    return densify_scene(sc, ops, n_ops, old_row_of_new_row, capacity);
}


int lodgs_scene_export(const lodgs_scene *sc, float *node_rec, int64_t *left, int64_t *right, int64_t *up_node,
                       int32_t *up_kind, int64_t *up_parent, int64_t *up_ref, int64_t *spt_root, int64_t *spt_base,
                       int64_t *spt_count, int64_t *node_of_row, float *lo_row, float *hi_row) {
    if (!sc) { set_error("scene_export: NULL scene"); return LODGS_E_INVALID; }
    const int64_t M = sc->n_nodes, U = sc->n_upper, S = sc->n_spt;
    std::vector<int32_t> t32(std::max<int64_t>(M, 1));
    if (node_rec) {      // canonical order = render rows scattered through node_of_row
        if (!sc->d_rows) { set_error("scene_export: the scene's records are not on the device"); return LODGS_E_STATE; }
        const size_t st = (size_t)sc->stride;
        std::vector<float> rows((size_t)M * st);
        LODGS_CUDA(cudaMemcpy(rows.data(), sc->d_rows, rows.size() * 4, cudaMemcpyDeviceToHost));
        LODGS_CUDA(cudaMemcpy(t32.data(), sc->d_node_of_row, M * 4, cudaMemcpyDeviceToHost));
        for (int64_t r = 0; r < M; ++r) memcpy(node_rec + (size_t)t32[r] * st, rows.data() + (size_t)r * st, st * 4);
    }
    auto widen = [&](int64_t *dst, const int32_t *src, int64_t n) -> int {
        if (!dst) return LODGS_OK;
        LODGS_CUDA(cudaMemcpy(t32.data(), src, n * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; ++i) dst[i] = t32[i];
        return LODGS_OK;
    };
    if (int r = widen(left, sc->d_left, M)) return r;
    if (int r = widen(right, sc->d_right, M)) return r;
    if (int r = widen(up_node, sc->d_up_node, U)) return r;
    if (int r = widen(spt_root, sc->d_spt_root, S)) return r;
    if (int r = widen(node_of_row, sc->d_node_of_row, M)) return r;
    if (up_kind || up_parent || up_ref) {
        std::vector<UpperEntry> ue(std::max<int64_t>(U, 1));
        LODGS_CUDA(cudaMemcpy(ue.data(), sc->d_upper, U * sizeof(UpperEntry), cudaMemcpyDeviceToHost));
        for (int64_t u = 0; u < U; ++u) {
            if (up_kind) up_kind[u] = ue[u].kind;
            if (up_parent) up_parent[u] = ue[u].parent;
            if (up_ref) up_ref[u] = ue[u].ref;
        }
    }
    if (spt_base || spt_count) {
        std::vector<uint32_t> b(S + 1);
        LODGS_CUDA(cudaMemcpy(b.data(), sc->d_spt_base, (S + 1) * 4, cudaMemcpyDeviceToHost));
        for (int64_t j = 0; j < S; ++j) {
            if (spt_base) spt_base[j] = b[j];
            if (spt_count) spt_count[j] = (int64_t)b[j + 1] - b[j];
        }
    }
    if (lo_row) LODGS_CUDA(cudaMemcpy(lo_row, sc->d_lo, M * 4, cudaMemcpyDeviceToHost));
    if (hi_row) LODGS_CUDA(cudaMemcpy(hi_row, sc->d_hi, M * 4, cudaMemcpyDeviceToHost));
    return LODGS_OK;
}

int lodgs_frame_create(lodgs_scene *sc, lodgs_frame **out) {
    if (!sc || !out) { set_error("frame_create: NULL argument"); return LODGS_E_INVALID; }
    *out = nullptr;
    lodgs_frame *fr = new (std::nothrow) lodgs_frame();
    if (!fr) { set_error("frame_create: host allocation failed"); return LODGS_E_OOM; }
    fr->scene = sc;
    fr->layout_version = sc->layout_version;
    FrameBufs &f = fr->f;
    const int64_t M = sc->n_nodes, S = sc->n_spt;
    cudaError_t e = cudaSuccess;
#define AL(p, n)                                                                  \
    if (e == cudaSuccess) e = cudaMalloc((void **)&p, std::max<size_t>((size_t)(n), 1) * sizeof(*p));
    AL(f.cnt, C_COUNT) AL(f.d_view, 1) AL(f.sel_rows, M) AL(f.emit_j, S) AL(f.emit_x, S) AL(f.high, S + 1) AL(f.work_off, S + 1)
    AL(f.block_counts, SEL_BLOCK_COUNTS) AL(f.scan_bsum, SCAN_GRID_MAX) AL(f.sort_hist, SORT_HIST) AL(f.work, 4)
    AL(f.up_out, sc->n_upper) AL(f.up_x, sc->n_upper)
#undef AL
    if (e == cudaSuccess) e = cudaMallocHost((void **)&fr->h_cnt, C_COUNT * sizeof(uint32_t));
    if (e != cudaSuccess) {
        free_frame_bufs(f);
        if (fr->h_cnt) cudaFreeHost(fr->h_cnt);
        delete fr;
        return cuda_fail(e, "frame_create");
    }
    memset(fr->h_cnt, 0, C_COUNT * sizeof(uint32_t));
    // small initial per-view buffers: they grow to what the views need (a
    // render that overflows reports LODGS_E_CAPACITY and the next one is sized)
    int rc = ensure_sel(fr, std::min<int64_t>(M, 1 << 12));
    if (!rc) rc = ensure_pairs(fr, 1 << 16);
    if (rc) { lodgs_frame_free(fr); return rc; }
    *out = fr;
    return LODGS_OK;
}

void lodgs_frame_free(lodgs_frame *fr) {
    if (!fr) return;
    cudaStreamSynchronize(fr->stream);
    for (cudaEvent_t &e : fr->ev)
        if (e) cudaEventDestroy(e);
    free_frame_bufs(fr->f);
    if (fr->h_cnt) cudaFreeHost(fr->h_cnt);
    delete fr;
}

int lodgs_frame_set_view(lodgs_frame *fr, const lodgs_camera *cam, const float *bg, void *stream) {
    if (!fr) { set_error("frame_set_view: NULL frame"); return LODGS_E_INVALID; }
    if (cam && !camera_ok(cam)) { set_error("frame_set_view: invalid camera"); return LODGS_E_INVALID; }
    if (cam) fr->rendered = fr->blend_bwd_done = false;   // the last render belongs to the old camera
    return set_view(fr, cam, bg, (cudaStream_t)stream);
}

int lodgs_select_lod(lodgs_scene *sc, const lodgs_camera *cam, lodgs_frame *fr, void *stream) {
    if (int rc = check_frame(sc, fr, "select_lod")) return rc;
    if (cam ? !camera_ok(cam) : !fr->have_view) {
        set_error(cam ? "select_lod: invalid camera" : "select_lod: no camera given and none set on the frame");
        return LODGS_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    fr->stream = st;
    fr->f.use_src = false;
    fr->cache = nullptr;                 // no longer a cache view
    for (bool &r : fr->ran) r = false;
    fr->mark(LODGS_STAGE_SELECT, 0, st);
    if (cam) {
        if (int rc = set_view(fr, cam, nullptr, st, true)) return rc;    // uploads the view, clears the counters
    } else {
        LODGS_CUDA(cudaMemsetAsync(fr->f.cnt, 0, C_COUNT * sizeof(uint32_t), st));
    }
    int rc = launch_select(sc, fr->f, st);
    if (rc) return rc;
    fr->counters_fresh = true;
    fr->mark(LODGS_STAGE_SELECT, 1, st);
    fr->selected = true;
    fr->rendered = false;
    fr->blend_bwd_done = false;
    return LODGS_OK;
}

int lodgs_frame_selection(lodgs_frame *fr, const uint32_t **d_rows, int64_t *n_selected) {
    if (!fr || !fr->selected) { set_error("frame_selection: no selection"); return LODGS_E_STATE; }
    if (d_rows) *d_rows = fr->f.sel_rows;
    if (n_selected) {
        LODGS_CUDA(cudaMemcpyAsync(fr->h_cnt, fr->f.cnt, C_COUNT * 4, cudaMemcpyDeviceToHost, fr->stream));
        LODGS_CUDA(cudaStreamSynchronize(fr->stream));
        *n_selected = fr->h_cnt[C_NSEL];
    }
    return LODGS_OK;
}

int lodgs_render(lodgs_scene *sc, lodgs_frame *fr, const float *rows, const float *bg, float *image, void *stream) {
    if (int rc = check_frame(sc, fr, "render")) return rc;
    if (!image) { set_error("render: NULL image"); return LODGS_E_INVALID; }
    if (fault_hit(LODGS_FAULT_RENDER)) { set_error("render: injected out of device memory"); return LODGS_E_OOM; }
    if (!fr->selected) { set_error("render: select_lod was not called on this frame"); return LODGS_E_STATE; }
    cudaStream_t st = (cudaStream_t)stream;
    if (st != fr->stream) {       // order after the selection's stream
        cudaEvent_t ev;
        LODGS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaEventRecord(ev, fr->stream);
        cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
        fr->stream = st;
    }
    if (int r = ensure_sel(fr, fr->want_sel)) return r;
    if (int r = ensure_pairs(fr, fr->want_pairs)) return r;
    uint64_t n_tiles = (uint64_t)fr->k.TX * fr->k.TY;
    if (n_tiles > fr->f.cap_tiles || !fr->f.ranges) {
        uint64_t c = fr->f.cap_tiles, c2 = fr->f.cap_tiles, c3 = fr->f.cap_tiles;
        if (int r = grow(fr->f.ranges, c, n_tiles)) return r;
        if (int r = grow(fr->f.tile_cnt, c2, n_tiles)) return r;
        if (int r = grow(fr->f.tile_order, c3, n_tiles)) return r;
        LODGS_CUDA(cudaMemsetAsync(fr->f.tile_cnt, 0, n_tiles * sizeof(uint32_t), st));   // zero between renders
        fr->f.cap_tiles = c;
    }
    if (bg && (bg[0] != fr->bg[0] || bg[1] != fr->bg[1] || bg[2] != fr->bg[2]))
        if (int r = set_view(fr, nullptr, bg, st)) return r;
    fr->f.count_work = fr->prof_mask != 0;
    // reset the render's counters and status (the selection's counters stay);
    // right after a selection they are still zero
    if (!fr->counters_fresh)
        LODGS_CUDA(cudaMemsetAsync(fr->f.cnt + C_NSEL_EFF, 0, (C_COUNT - C_NSEL_EFF) * sizeof(uint32_t), st));
    fr->counters_fresh = false;
    fr->mark(LODGS_STAGE_PROJECT, 0, st);
    if (!rows && !sc->d_rows) {
        set_error("render: the scene's records live in host memory; pass the cache's device records");
        return LODGS_E_INVALID;
    }
    int rc = launch_project(sc, rows ? rows : sc->d_rows, fr->f, st);
    if (rc) return rc;
    fr->mark(LODGS_STAGE_PROJECT, 1, st);
    StageMarks sm{fr->prof_mask ? fr->ev : nullptr, fr->prof_mask};
    rc = launch_raster(fr->k, fr->f, image, st, sm);
    if (rc) return rc;
    for (int s2 = LODGS_STAGE_COUNT; s2 <= LODGS_STAGE_BLEND; ++s2)
        if (fr->prof_mask >> s2 & 1u) fr->ran[s2] = true;
    LODGS_CUDA(cudaMemcpyAsync(fr->h_cnt, fr->f.cnt, C_COUNT * 4, cudaMemcpyDeviceToHost, st));
    fr->rendered = true;
    fr->blend_bwd_done = false;
    return LODGS_OK;
}

namespace {
int backward_blend(lodgs_scene *sc, lodgs_frame *fr, const float *image, const float *dL_dimage,
                   const void *target, bool target_u8, float l1_scale, float *loss_sum, void *stream,
                   const char *who) {
    if (int rc = check_frame(sc, fr, who)) return rc;
    if (!image || (!dL_dimage && !(target && loss_sum))) {
        set_error(std::string(who) + ": NULL argument");
        return LODGS_E_INVALID;
    }
    if (!fr->rendered) { set_error("render_backward: render was not called on this frame"); return LODGS_E_STATE; }
    if ((uint64_t)fr->k.TX * fr->k.TY > fr->f.cap_tiles) {
        set_error("render_backward: the frame's camera is larger than the one it was rendered with");
        return LODGS_E_STATE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (st != fr->stream) {
        cudaEvent_t ev;
        LODGS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaEventRecord(ev, fr->stream);
        cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
        fr->stream = st;
    }
    fr->mark(LODGS_STAGE_BLEND_BWD, 0, st);
    int rc = launch_raster_backward(fr->k, fr->f, image, dL_dimage, target, target_u8, l1_scale, loss_sum,
                                    fr->blend_bwd_done, st);
    if (rc) return rc;
    fr->mark(LODGS_STAGE_BLEND_BWD, 1, st);
    fr->blend_bwd_done = true;
    return LODGS_OK;
}
}  // namespace

int lodgs_render_backward_blend(lodgs_scene *sc, lodgs_frame *fr, const float *image, const float *dL_dimage,
                                void *stream) {
    if (!dL_dimage) { set_error("render_backward_blend: NULL dL_dimage"); return LODGS_E_INVALID; }
    return backward_blend(sc, fr, image, dL_dimage, nullptr, false, 0.f, nullptr, stream, "render_backward_blend");
}

int lodgs_render_backward_blend_l1(lodgs_scene *sc, lodgs_frame *fr, const float *image, const float *target,
                                   float grad_scale, float *loss_sum, void *stream) {
    if (!target || !loss_sum) { set_error("render_backward_blend_l1: NULL argument"); return LODGS_E_INVALID; }
    return backward_blend(sc, fr, image, nullptr, target, false, grad_scale, loss_sum, stream,
                          "render_backward_blend_l1");
}

int lodgs_render_backward_blend_l1_u8(lodgs_scene *sc, lodgs_frame *fr, const float *image, const uint8_t *target,
                                      float grad_scale, float *loss_sum, void *stream) {
    if (!target || !loss_sum) { set_error("render_backward_blend_l1_u8: NULL argument"); return LODGS_E_INVALID; }
    return backward_blend(sc, fr, image, nullptr, target, true, grad_scale, loss_sum, stream,
                          "render_backward_blend_l1_u8");
}

int lodgs_render_backward_project(lodgs_scene *sc, lodgs_frame *fr, const float *rows, float *grad_rows,
                                  int64_t grad_capacity, int dense,
                                  void *stream) {
    if (int rc = check_frame(sc, fr, "render_backward_project")) return rc;
    if (!grad_rows) {
        set_error("render_backward_project: NULL argument");
        return LODGS_E_INVALID;
    }
    if (!fr->blend_bwd_done) { set_error("render_backward_project: the blend backward has not run"); return LODGS_E_STATE; }
    if (!rows && !sc->d_rows) {
        set_error("render_backward: the scene's records live in host memory; pass the cache's device records");
        return LODGS_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (st != fr->stream) {
        cudaEvent_t ev;
        LODGS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaEventRecord(ev, fr->stream);
        cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
        fr->stream = st;
    }
    fr->mark(LODGS_STAGE_PROJECT_BWD, 0, st);
    int rc = launch_project_backward(sc, rows ? rows : sc->d_rows, fr->f, grad_rows, grad_capacity, dense, st);
    if (rc) return rc;
    fr->mark(LODGS_STAGE_PROJECT_BWD, 1, st);
    return LODGS_OK;
}

int lodgs_render_backward(lodgs_scene *sc, lodgs_frame *fr, const float *rows, const float *bg,
                          const float *image, const float *dL_dimage, float *grad_rows, int64_t grad_capacity, int dense,
                          void *stream) {
    if (int rc = check_frame(sc, fr, "render_backward")) return rc;
    if (!image || !dL_dimage || !grad_rows) {
        set_error("render_backward: NULL argument");
        return LODGS_E_INVALID;
    }
    if (bg && (bg[0] != fr->bg[0] || bg[1] != fr->bg[1] || bg[2] != fr->bg[2])) {
        set_error("render_backward: background differs from the one the frame was rendered with");
        return LODGS_E_STATE;
    }
    int rc = lodgs_render_backward_blend(sc, fr, image, dL_dimage, stream);
    if (!rc) rc = lodgs_render_backward_project(sc, fr, rows, grad_rows, grad_capacity, dense, stream);
    return rc;
}

int lodgs_select_lod_batch(lodgs_scene *sc, const lodgs_camera *cams, lodgs_frame *const *frames, int n,
                           void *stream) {
    static_assert(LODGS_SELECT_BATCH_MAX <= SCAN_BATCH_MAX, "batch bound");
    if (!sc || !cams || !frames || n < 1 || n > LODGS_SELECT_BATCH_MAX) {
        set_error("select_lod_batch: NULL argument or n not in 1..LODGS_SELECT_BATCH_MAX");
        return LODGS_E_INVALID;
    }
    for (int i = 0; i < n; ++i) {
        if (int rc = check_frame(sc, frames[i], "select_lod_batch")) return rc;
        if (!camera_ok(&cams[i])) { set_error("select_lod_batch: invalid camera"); return LODGS_E_INVALID; }
        for (int j = 0; j < i; ++j)
            if (frames[j] == frames[i]) { set_error("select_lod_batch: a frame appears twice"); return LODGS_E_INVALID; }
    }
    cudaStream_t st = (cudaStream_t)stream;
    View views[LODGS_SELECT_BATCH_MAX];
    FrameBufs *fs[LODGS_SELECT_BATCH_MAX];
    for (int i = 0; i < n; ++i) {
        lodgs_frame *fr = frames[i];
        fr->stream = st;
        fr->f.use_src = false;
        fr->cache = nullptr;
        for (bool &r : fr->ran) r = false;
        fr->mark(LODGS_STAGE_SELECT, 0, st);
        fr->k = make_camk(cams[i]);
        views[i].k = fr->k;
        views[i].bg[0] = fr->bg[0]; views[i].bg[1] = fr->bg[1]; views[i].bg[2] = fr->bg[2]; views[i].bg[3] = 0.f;
        fs[i] = &fr->f;
    }
    if (int rc = launch_select_batch(sc, fs, views, n, st)) return rc;
    for (int i = 0; i < n; ++i) {
        lodgs_frame *fr = frames[i];
        fr->have_view = true;
        fr->counters_fresh = true;
        fr->mark(LODGS_STAGE_SELECT, 1, st);
        fr->selected = true;
        fr->rendered = false;
        fr->blend_bwd_done = false;
    }
    return LODGS_OK;
}

int lodgs_frame_get_stats(lodgs_frame *fr, lodgs_frame_stats *s) {
    if (!fr || !s) { set_error("frame_get_stats: NULL argument"); return LODGS_E_INVALID; }
    LODGS_CUDA(cudaStreamSynchronize(fr->stream));
    // the render leaves a copy of its counters; a backward since may have set a status bit
    if (!fr->rendered || fr->blend_bwd_done)
        LODGS_CUDA(cudaMemcpy(fr->h_cnt, fr->f.cnt, C_COUNT * 4, cudaMemcpyDeviceToHost));
    const uint32_t *h = fr->h_cnt;
    s->n_selected = h[C_NSEL];
    s->n_upper_selected = h[C_NUP];
    s->n_spt_cut = h[C_NEMIT];
    s->n_spt_scanned = h[C_WORK];
    s->n_visible = h[C_NVIS];
    s->n_pairs = h[C_NKEPT];
    s->width = fr->k.W;
    s->height = fr->k.H;
    s->status = LODGS_OK;
    if (h[C_STATUS] & ST_TIMEOUT) s->status = LODGS_E_TIMEOUT;
    if (h[C_STATUS] & ST_GRAD_CAPACITY) {
        s->status = LODGS_E_CAPACITY;
        set_error("render_backward: the gradient rows were fewer than the selected nodes; nothing was written");
    }
    if (h[C_STATUS] & ST_CAPACITY) {
        s->status = LODGS_E_CAPACITY;
        uint64_t ns = h[C_NSEL], np = h[C_NKEPT_WANT];
        if (ns > fr->f.cap_sel) fr->want_sel = std::max<uint64_t>(fr->want_sel, ns + ns / 4);
        else if (np > fr->f.cap_pairs) fr->want_pairs = std::max<uint64_t>(fr->want_pairs, np + np / 4);
    }
    return LODGS_OK;
}

int lodgs_frame_memory(lodgs_frame *fr, int64_t *held, int64_t *needed) {
    if (!fr) { set_error("frame_memory: NULL frame"); return LODGS_E_INVALID; }
    const FrameBufs &f = fr->f;
    const lodgs_scene *sc = fr->scene;
    const uint64_t M = (uint64_t)sc->n_nodes, S = (uint64_t)sc->n_spt, U = (uint64_t)sc->n_upper;
    // bytes per selected node, per pair and per tile of the grown buffers
    constexpr uint64_t per_sel = 3 * sizeof(float4) + 4 * sizeof(uint32_t) + sizeof(uint2) + 2 * sizeof(uint32_t) +
                                 G2D_STRIDE * sizeof(float);
    constexpr uint64_t per_pair = 4 * sizeof(uint32_t) + sizeof(unsigned long long);
    constexpr uint64_t per_tile = sizeof(uint2) + 2 * sizeof(uint32_t);
    const uint64_t fixed = C_COUNT * 4 + sizeof(View) + M * 4 + S * 8 + (S + 1) * 8 + SEL_BLOCK_COUNTS * 4 +
                           SCAN_GRID_MAX * 4 + SORT_HIST * 4 + 4 * sizeof(unsigned long long) + U * 5 +
                           (f.sel_src ? M * 4 : 0) + (f.emit_src ? std::max<uint64_t>(S, 1) * 4 : 0);
    if (held)
        *held = (int64_t)(fixed + f.cap_sel * per_sel + f.cap_pairs * per_pair + f.cap_keep * 4 +
                          f.cap_tiles * per_tile);
    if (needed) {
        LODGS_CUDA(cudaStreamSynchronize(fr->stream));
        LODGS_CUDA(cudaMemcpy(fr->h_cnt, f.cnt, C_COUNT * 4, cudaMemcpyDeviceToHost));
        const uint64_t ns = fr->selected ? fr->h_cnt[C_NSEL] : 0;
        const uint64_t np = fr->rendered ? std::max(fr->h_cnt[C_NKEPT], fr->h_cnt[C_NKEPT_WANT]) : 0;
        const uint64_t nt = fr->rendered ? (uint64_t)fr->k.TX * fr->k.TY : 0;
        *needed = (int64_t)(fixed + std::max<uint64_t>(ns, 1) * per_sel + np * per_pair +
                            (np ? np / 16 + 1 : 0) * 4 + nt * per_tile);
    }
    return LODGS_OK;
}

int lodgs_frame_reserve(lodgs_frame *fr, int64_t n_sel, int64_t n_pairs) {
    if (!fr || n_sel < 0 || n_pairs < 0) { set_error("frame_reserve: NULL frame or negative count"); return LODGS_E_INVALID; }
    LODGS_CUDA(cudaStreamSynchronize(fr->stream));        // no render of this frame is reading the buffers
    fr->want_sel = std::max<uint64_t>((uint64_t)n_sel, fr->f.cap_sel);
    fr->want_pairs = std::max<uint64_t>((uint64_t)n_pairs, fr->f.cap_pairs);
    if (int r = ensure_sel(fr, fr->want_sel)) return r;
    if (int r = ensure_pairs(fr, fr->want_pairs)) return r;
    fr->want_sel = fr->f.cap_sel;
    fr->want_pairs = fr->f.cap_pairs;
    return LODGS_OK;
}

int lodgs_frame_set_ordering(lodgs_frame *fr, int mode) {
    if (!fr || mode < ORDER_AUTO || mode > ORDER_GLOBAL) {
        set_error("frame_set_ordering: NULL frame or mode not in 0..2");
        return LODGS_E_INVALID;
    }
    fr->f.ordering = mode;
    return LODGS_OK;
}

int lodgs_frame_set_profiling(lodgs_frame *fr, int on) {
    if (!fr) { set_error("frame_set_profiling: NULL frame"); return LODGS_E_INVALID; }
    if (on)
        for (cudaEvent_t &e : fr->ev)
            if (!e) LODGS_CUDA(cudaEventCreate(&e));
    fr->prof_mask = on < 0 ? (1u << LODGS_NUM_STAGES) - 1u : (uint32_t)on;
    return LODGS_OK;
}

int lodgs_frame_stage_ms(lodgs_frame *fr, float *ms) {
    if (!fr || !ms) { set_error("frame_stage_ms: NULL argument"); return LODGS_E_INVALID; }
    if (!fr->prof_mask) { set_error("frame_stage_ms: profiling is off"); return LODGS_E_STATE; }
    LODGS_CUDA(cudaStreamSynchronize(fr->stream));
    for (int s2 = 0; s2 < LODGS_NUM_STAGES; ++s2) {
        ms[s2] = 0.f;
        if (fr->ran[s2]) LODGS_CUDA(cudaEventElapsedTime(&ms[s2], fr->ev[2 * s2], fr->ev[2 * s2 + 1]));
    }
    return LODGS_OK;
}

int lodgs_frame_work(lodgs_frame *fr, uint64_t *work) {
    if (!fr || !work) { set_error("frame_work: NULL argument"); return LODGS_E_INVALID; }
    LODGS_CUDA(cudaStreamSynchronize(fr->stream));
    unsigned long long w[4] = {0, 0, 0, 0};
    if (fr->f.count_work)           // the last render was a profiling one (the only kind that tallies)
        LODGS_CUDA(cudaMemcpy(w, fr->f.work, sizeof(w), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 4; ++i) work[i] = w[i];
    return LODGS_OK;
}

int lodgs_frame_export(lodgs_frame *fr, uint32_t *pair_index, int64_t cap_pairs, uint32_t *ranges, float *splats,
                       uint32_t *depth_key) {
    if (!fr || !fr->rendered) { set_error("frame_export: render was not called on this frame"); return LODGS_E_STATE; }
    LODGS_CUDA(cudaStreamSynchronize(fr->stream));
    LODGS_CUDA(cudaMemcpy(fr->h_cnt, fr->f.cnt, C_COUNT * 4, cudaMemcpyDeviceToHost));
    if (fr->h_cnt[C_STATUS] & ST_CAPACITY) { set_error("frame_export: last render overflowed"); return LODGS_E_CAPACITY; }
    const uint64_t np = fr->h_cnt[C_NKEPT], ns = fr->h_cnt[C_NSEL_EFF];
    const uint64_t nt = (uint64_t)fr->k.TX * fr->k.TY;
    if (pair_index) {
        if ((int64_t)np > cap_pairs) { set_error("frame_export: pair buffer too small"); return LODGS_E_INVALID; }
        if (np) LODGS_CUDA(cudaMemcpy(pair_index, fr->f.sorted_pval, np * 4, cudaMemcpyDeviceToHost));
    }
    if (ranges) LODGS_CUDA(cudaMemcpy(ranges, fr->f.ranges, nt * 8, cudaMemcpyDeviceToHost));
    if (splats && ns) {
        std::vector<float4> a(ns), b(ns), c(ns);
        LODGS_CUDA(cudaMemcpy(a.data(), fr->f.sp_a, ns * 16, cudaMemcpyDeviceToHost));
        LODGS_CUDA(cudaMemcpy(b.data(), fr->f.sp_b, ns * 16, cudaMemcpyDeviceToHost));
        LODGS_CUDA(cudaMemcpy(c.data(), fr->f.sp_c, ns * 16, cudaMemcpyDeviceToHost));
        for (uint64_t i = 0; i < ns; ++i) {
            float *o = splats + LODGS_SPLAT_FLOATS * i;
            o[0] = a[i].x; o[1] = a[i].y; o[2] = -2.0f * a[i].z; o[3] = -a[i].w; o[4] = -2.0f * b[i].x;
            o[5] = b[i].y; o[6] = b[i].z; o[7] = b[i].w; o[8] = c[i].x; o[9] = c[i].y; o[10] = c[i].z;
        }
    }
    if (depth_key && ns) {
        if (!fr->f.order) {
            LODGS_CUDA(cudaMemcpy(depth_key, fr->f.dkey, ns * 4, cudaMemcpyDeviceToHost));
        } else {     // the global ordering's depth sort permuted the keys: undo it with the sorted order
            const uint32_t *skeys = fr->f.order == fr->f.dval ? fr->f.dkey : fr->f.dkey_alt;
            std::vector<uint32_t> o(ns), kk(ns);
            LODGS_CUDA(cudaMemcpy(o.data(), fr->f.order, ns * 4, cudaMemcpyDeviceToHost));
            LODGS_CUDA(cudaMemcpy(kk.data(), skeys, ns * 4, cudaMemcpyDeviceToHost));
            for (uint64_t r = 0; r < ns; ++r) depth_key[o[r]] = kk[r];
        }
    }
    return LODGS_OK;
}

}  // extern "C"
