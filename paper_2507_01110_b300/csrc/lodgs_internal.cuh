// Internal declarations shared by the CUDA translation units of liblodgs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "../../include/lodgs.h"

namespace lodgs {

// ---- record layout (see include/lodgs.h) ----------------------------------
constexpr int REC_MU = 0, REC_S = 3, REC_Q = 6, REC_OP = 10, REC_B = 11, REC_F = 14;
constexpr int KIND_INTERNAL = 0, KIND_LEAF = 1, KIND_SPT = 2;
constexpr int TILE = 16;
constexpr int TILE_PIX = TILE * TILE;

inline int sh_count(int degree) { return (degree + 1) * (degree + 1) - 1; }
inline int record_stride(int degree) { return (14 + 3 * sh_count(degree) + 7) / 8 * 8; }

// ---- per-camera constants, float32 (same expressions as the decisions they feed)
struct CamK {
    float R[9];
    float pos[3];
    float fx, fy, cx, cy;
    float inv_k;           // tau / fx
    float spt_scale;       // factor on the SPT root distances (training LoD noise; 1 = none)
    float limx, limy;      // 1.3 * tan(half fov)
    float plane[4][3];     // unit inward normals of the 4 side planes (camera space)
    float znear;
    int W, H, TX, TY;
};

CamK make_camk(const lodgs_camera &c);

// Per-view parameters read by the kernels from device memory, so that a
// captured CUDA graph of a view's step can be replayed for any camera of the
// same resolution (the view is uploaded outside the graph).
struct View {
    CamK k;
    float bg[4];
};

// view-space position and camera distance of a world point (float32, evaluated
// exactly as written; translation units using it are compiled without FMA
// contraction)
__device__ __forceinline__ void cam_view(const CamK &k, float mx, float my, float mz, float t[3], float *dist) {
    float dx = mx - k.pos[0], dy = my - k.pos[1], dz = mz - k.pos[2];
    *dist = sqrtf((dx * dx + dy * dy) + dz * dz);
    t[0] = (k.R[0] * dx + k.R[1] * dy) + k.R[2] * dz;
    t[1] = (k.R[3] * dx + k.R[4] * dy) + k.R[5] * dz;
    t[2] = (k.R[6] * dx + k.R[7] * dy) + k.R[8] * dz;
}

// sphere (centre t, radius 3 * maxs) entirely outside the near plane or one of
// the four side planes
__device__ __forceinline__ bool cam_culled(const CamK &k, const float t[3], float maxs) {
    float r = 3.0f * maxs;
    if (t[2] + r < k.znear) return true;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        float s = (k.plane[p][0] * t[0] + k.plane[p][1] * t[1]) + k.plane[p][2] * t[2];
        if (s < -r) return true;
    }
    return false;
}

// ---- device status words and counters --------------------------------------
enum : uint32_t {
    ST_CAPACITY = 1u,       // a frame workspace buffer was too small
    ST_TIMEOUT = 2u,        // a bounded device wait ran out
    ST_GRAD_CAPACITY = 4u,  // the caller's gradient rows were fewer than the selection
};
enum {
    C_NSEL = 0,      // selected nodes (a1 + a2)
    C_NUP = 1,       // of which upper-hierarchy nodes
    C_NEMIT = 2,     // SPT roots handed to the SPT cut
    C_WORK = 3,      // SPT entries scanned (sum of the prefixes)
    C_NSPTSEL = 4,   // SPT entries selected
    C_NSEL_EFF = 5,  // selected nodes processed by the render (0 on overflow)
    C_NPAIR = 6,     // (Gaussian, tile) rectangle pairs
    C_NPAIR_EFF = 7, // rectangle pairs emitted by the global ordering (0 on overflow)
    C_NVIS = 8,      // visible Gaussians
    C_STATUS = 9,    // ST_* bits
    C_NKEPT = 10,    // pairs kept by the tile support test
    C_NKEPT_WANT = 11, // kept pairs counted before the capacity check (workspace growth)
    C_NPAIR64 = 12,  // words 12-13: rectangle pairs as a 64-bit sum (32-bit index guard)
    C_COUNT = 16
};

// ---- scene -----------------------------------------------------------------
struct UpperEntry {        // 32 bytes, one per upper-hierarchy BFS entry
    float mu[3];
    float S;               // size term S_i (float32 decision D3)
    float maxs;            // max scale (culling sphere radius / 3)
    int32_t parent;        // upper index of the parent, -1 for the root
    int32_t kind;          // KIND_*
    int32_t ref;           // render row (internal/leaf) or SPT index
};

}  // namespace lodgs

struct lodgs_scene {
    int64_t n_leaves = 0, n_nodes = 0, n_upper = 0, n_upper_rows = 0, n_spt = 0;
    int sh_degree = 0, stride = 0;
    float spt_volume = 0.f, kappa = 0.f;
    int upper_depth = 0;                         // max depth of the upper hierarchy
    uint32_t layout_version = 0;                 // bumped by each densification (rows renumbered)
    int32_t root = -1;                           // canonical id of the root
    // device
    float *d_rows = nullptr;                     // n_nodes x stride, render-row order
    lodgs::UpperEntry *d_upper = nullptr;        // n_upper
    uint32_t *d_spt_base = nullptr;              // n_spt + 1
    float *d_lo = nullptr, *d_hi = nullptr;      // n_nodes (render rows)
    // canonical structure (device), kept for export and rebuilds
    float *d_node_rec = nullptr;                 // n_nodes x stride, canonical id order
    int32_t *d_left = nullptr, *d_right = nullptr;
    int32_t *d_node_of_row = nullptr;
    int32_t *d_up_node = nullptr;
    int32_t *d_spt_root = nullptr;
};

namespace lodgs {

// Device buffers of one frame (one view).  Capacities are element counts.
enum : int { ORDER_AUTO = 0, ORDER_PER_TILE = 1, ORDER_GLOBAL = 2 };

// floats per Gaussian of the 2D gradient rows (9 used; 16-byte aligned rows)
constexpr int G2D_STRIDE = 12;

struct FrameBufs {
    uint32_t *cnt = nullptr;         // C_COUNT device counters
    View *d_view = nullptr;          // camera constants and background of the current view
    // selection (capacity n_nodes / n_spt)
    uint32_t *sel_rows = nullptr, *emit_j = nullptr, *high = nullptr, *work_off = nullptr;
    uint32_t *sel_src = nullptr;      // record slot of each selected node (out-of-core renders)
    uint8_t *up_out = nullptr;        // per upper entry: its Algorithm 1 outcome (optional cache)
    float *up_x = nullptr;            // per upper entry: tau * d / f (with up_out)
    uint32_t *emit_src = nullptr;     // slot of entry 0 of each emitted SPT (out-of-core renders)
    bool use_src = false;             // project through sel_src instead of sel_rows
    float *emit_x = nullptr;
    uint32_t *block_counts = nullptr, *scan_bsum = nullptr, *sort_hist = nullptr;
    // per selected node (capacity cap_sel)
    float4 *sp_a = nullptr;          // u, v, -A/2, -B        (mean in pixels, scaled conic)
    float4 *sp_b = nullptr;          // -C/2, opacity, r, g
    float4 *sp_c = nullptr;          // b, rx, ry, 0   (rx, ry: support half extents, block test)
    uint32_t *dkey = nullptr;        // float32 bits of the view depth (0xffffffff if invisible)
    uint32_t *dval = nullptr, *dkey_alt = nullptr, *dval_alt = nullptr;   // global ordering: depth sort
    uint2 *rect = nullptr;           // x0 | y0 << 16, x1 | y1 << 16
    uint32_t *ntiles = nullptr, *pair_off = nullptr;
    float *g2d = nullptr;            // G2D_STRIDE per selected: d/d(u, v, A, B, C, opacity, r, g, b), 3 unused
    // pairs (capacity cap_pairs)
    uint32_t *pkey = nullptr, *pval = nullptr;   // pairs: depth key / tile key, selected index
    uint32_t *pkey_alt = nullptr, *pval_alt = nullptr;   // global ordering: tile sort
    unsigned long long *pscratch = nullptr;      // merge scratch of the per-tile sort (long lists)
    uint32_t *keep = nullptr;        // per 32 rectangle pairs: kept lanes (per-tile ordering), cap_keep words
    uint64_t cap_keep = 0;
    // tiles (capacity cap_tiles)
    uint2 *ranges = nullptr;
    uint32_t *tile_cnt = nullptr;     // kept pairs per tile, then scatter cursors; zero between renders
    uint32_t *tile_order = nullptr;   // tiles by pair count, largest first: the blends' block -> tile map
    unsigned long long *work = nullptr;   // 4 counters, see lodgs_frame_work
    bool count_work = false;              // blends tally the work counters (profiling frames)
    int ordering = 0;                     // ORDER_*: how pairs are put in (tile, depth, index) order
    const uint32_t *order = nullptr;      // global ordering: selected indices by depth
    const uint32_t *sorted_pval = nullptr;   // selected index of each ordered pair
    uint64_t cap_sel = 0, cap_pairs = 0, cap_tiles = 0;
};

void set_error(const std::string &msg);
void count_launches(int n);     // process-wide tally of this library's kernel launches

// Programmatic dependent launch.  A kernel launched through pdl_launch may be
// scheduled while the kernel before it on the stream is still draining its
// last blocks; it calls pdl_wait() as its first statement, which returns once
// that kernel has completed and its memory operations are visible.  So only
// the launch latency overlaps the predecessor's tail: every global read and
// write still follows it.  (After a copy, a memset or an event wait the launch
// is ordered as usual; without a programmatic predecessor pdl_wait returns at
// once.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

//
// Launch priority (LODGS_PRIO_SPLIT): every kernel but the two blends is
// launched at the device's greatest priority, so that when several views are
// in flight the short memory- and latency-bound kernels of one view take SMs
// as the issue-bound blend CTAs of another retire, instead of waiting behind
// the blend's remaining waves.  The blends use pdl_launch_p with priority 0
// (the default, lowest).  Measured with three views in flight: fwd+bwd step
// 0.2836 -> 0.2790 ms, forward with two views in flight 0.140 -> 0.132 ms per
// view; 0 launches everything at the default priority.
#ifndef LODGS_PRIO_SPLIT
#define LODGS_PRIO_SPLIT 1
#endif
int launch_priority_high();     // the device's greatest stream priority (cached)

// Blocks of `kern` (with `threads` threads and its static shared memory) that
// are resident on the current device at once: the SM count times the
// occupancy calculator's blocks per SM, cached per kernel and device.  Kernels
// whose blocks split the work evenly (grid-stride loops, even chunks) are
// launched with a whole number of such waves: a partial last wave would run a
// few blocks per SM while the rest of the device idles.
int resident_blocks(const void *kern, int threads);
int device_sms();   // SM count of the current device (cached per device)
template <typename... KArgs>
inline int resident_grid(void (*kern)(KArgs...), int threads, int waves = 1) {
    return waves * resident_blocks(reinterpret_cast<const void *>(kern), threads);
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch_p(int prio, void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                                Args &&...args) {
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributePriority;
    attr[1].val.priority = prio;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = prio != 0 ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args &&...args) {
    return pdl_launch_p(LODGS_PRIO_SPLIT ? launch_priority_high() : 0, kern, grid, block, st,
                        std::forward<Args>(args)...);
}
bool fault_hit(int site);       // an armed injected fault at `site` fires (host side only)
int cuda_fail(cudaError_t e, const char *what);
#define LODGS_CUDA(call)                                       \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return lodgs::cuda_fail(_e, #call); \
    } while (0)

// hierarchy construction (scene.cu)
int build_scene(const float *leaves, int64_t n, int degree, int on_device, const lodgs_build_params &p,
                lodgs_scene *sc);
void free_scene(lodgs_scene *sc);
int densify_scene(lodgs_scene *sc, const lodgs_densify_op *ops, int64_t n_ops, int32_t *old_row_of_new_row,
                  int64_t capacity);
int save_scene(const lodgs_scene *sc, const char *path);
int load_scene(const char *path, lodgs_scene *sc);
// 0 if `fr` belongs to `sc` and was created for its current layout, else an
// error code (with the message set, prefixed by `who`)
int check_frame(const lodgs_scene *sc, const lodgs_frame *fr, const char *who);
bool camera_ok(const lodgs_camera *c);   // the camera checks every entry point applies
// sparse Adam over `rows` of params/m/v/t (lodgs_adam_step's contract); dirty[row] = 1 if given
int launch_adam(const lodgs_scene *sc, float *params, float *m, float *v, uint32_t *t, const uint32_t *rows,
                const float *grads, const uint32_t *d_n, int64_t max_n, const float *lr, float b1, float b2,
                float eps, cudaStream_t st, uint32_t *dirty = nullptr);

// radix sort and scans (sort.cu).  All take element counts from device memory so
// that no host synchronisation is needed between stages.
struct SortWork {
    uint32_t *hist = nullptr;       // RADIX * grid
    size_t hist_cap = 0;
};
#ifndef LODGS_SORT_GRID
#define LODGS_SORT_GRID 296
#endif
constexpr int SORT_GRID = LODGS_SORT_GRID;   // radix sort blocks for short sorts (2 per SM on 148 SMs)
constexpr int SORT_GRID_MAX = 148 * 8;       // ... growing with the element count up to 8 per SM
constexpr int SORT_HIST = 256 * (SORT_GRID_MAX + 1);   // histogram table + digit totals
int radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                     const uint32_t *d_n, uint32_t max_n, int begin_bit, int end_bit, uint32_t *hist,
                     cudaStream_t st, bool *result_in_alt);
// exclusive scan of n (device count) uint32 values in[idx[i]] (idx null: in[i]);
// total written to *d_total
constexpr int SEL_BLOCK_COUNTS = 1024;        // per-block counts of the selection passes (buffer entries)
constexpr int SCAN_GRID = 148;                // scan blocks for short scans
constexpr int SCAN_GRID_MAX = 148 * 8;        // ... growing with the element count (block-sum buffers)
// Exclusive scans of k arrays at once (one grid row each), each as
// scan_exclusive with no index array; the same max_n bounds every array.
constexpr int SCAN_BATCH_MAX = 8;
struct ScanBatch {
    const uint32_t *in[SCAN_BATCH_MAX];
    uint32_t *out[SCAN_BATCH_MAX];
    const uint32_t *d_n[SCAN_BATCH_MAX];
    uint32_t *block_sums[SCAN_BATCH_MAX];
    uint32_t *d_total[SCAN_BATCH_MAX];
};
int scan_exclusive_batch(const ScanBatch &b, int k, uint32_t max_n, cudaStream_t st);
int scan_exclusive(const uint32_t *in, uint32_t *out, const uint32_t *d_n, uint32_t max_n,
                   uint32_t *block_sums, uint32_t *d_total, cudaStream_t st, const uint32_t *idx = nullptr);
// optional CUDA events bracketing stages (ev[2s], ev[2s+1]) of the stages in `mask`
struct StageMarks {
    cudaEvent_t *ev = nullptr;
    uint32_t mask = 0;
    void mark(int stage, int end, cudaStream_t st) const {
        if (ev && (mask >> stage & 1u)) cudaEventRecord(ev[2 * stage + end], st);
    }
};

// per-view stages (select.cu, project.cu, raster.cu)
// zero_cnt: also clear C_COUNT counters there (the start of a selection)
int launch_set_view(const View &v, View *dst, cudaStream_t st, uint32_t *zero_cnt = nullptr);
int launch_select(const lodgs_scene *sc, FrameBufs &f, cudaStream_t st);
// the selection of k <= SCAN_BATCH_MAX views in one launch of each pass (views
// given: uploaded to each frame, its counters cleared)
int launch_select_batch(const lodgs_scene *sc, FrameBufs *const *fs, const View *views, int k, cudaStream_t st);
int launch_select_upper(const lodgs_scene *sc, FrameBufs &f, bool with_src, cudaStream_t st);
int launch_spt_high(const lodgs_scene *sc, FrameBufs &f, cudaStream_t st);
int launch_select_spt(const lodgs_scene *sc, FrameBufs &f, bool with_src, cudaStream_t st);
// `k` is the host copy of the view (resolution, grid sizes); kernels read f.d_view
int launch_project(const lodgs_scene *sc, const float *rows, FrameBufs &f, cudaStream_t st);
int launch_raster(const CamK &k, FrameBufs &f, float *image, cudaStream_t st, const StageMarks &sm);
// target (with loss_sum): the L1 loss's gradient formed in the kernel from a
// float32 or (target_u8) 8-bit H x W x 3 target; else dL/dC read from dL_dimage
// zero_g2d: clear the 2D gradient rows first (the projection of the render
// cleared those of its selection; set it for a second backward of one render)
int launch_raster_backward(const CamK &k, FrameBufs &f, const float *image, const float *dL_dimage,
                           const void *target, bool target_u8, float l1_scale, float *loss_sum, bool zero_g2d,
                           cudaStream_t st);
int launch_project_backward(const lodgs_scene *sc, const float *rows, FrameBufs &f, float *grad_rows,
                            int64_t grad_capacity, int dense, cudaStream_t st);
}  // namespace lodgs

struct lodgs_frame {
    lodgs_scene *scene = nullptr;
    uint32_t layout_version = 0;        // the scene layout the buffers were sized for
    const void *cache = nullptr;        // the cache of the last lodgs_stream_nodes, and its view number
    uint64_t cache_view = 0;
    lodgs::FrameBufs f;
    uint32_t *h_cnt = nullptr;          // pinned mirror of the device counters
    cudaStream_t stream = 0;
    lodgs::CamK k{};
    bool selected = false, rendered = false, have_view = false, blend_bwd_done = false;
    bool counters_fresh = false;      // every counter is zero since the last selection: no render reset
    float bg[3] = {0.f, 0.f, 0.f};
    uint64_t want_sel = 0, want_pairs = 0;
    // stage timing: ev[2s] / ev[2s+1] bracket stage s, for the stages in prof_mask
    uint32_t prof_mask = 0;
    cudaEvent_t ev[2 * LODGS_NUM_STAGES] = {};
    bool ran[LODGS_NUM_STAGES] = {};
    void mark(int stage, int end, cudaStream_t st) {
        if (!(prof_mask >> stage & 1u)) return;
        cudaEventRecord(ev[2 * stage + end], st);
        if (end) ran[stage] = true;
    }
};

