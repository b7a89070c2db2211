// LoD cut into caller-owned buffers with no device allocation.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// all handed to its own arena or pool (a renderer or game engine that budgets
// every byte itself), and latency-critical loops where cudaMalloc's implicit
// device synchronisation would stall other work on the GPU.  This variant of
// lodgs_select_lod keeps its scratch (counters, per-SPT lists, block counts) in
// one file-scope __device__ array instead of a frame's workspace.
//
// The array lives in every GPU that loads the library until the process exits
// and is shared by all calls on that GPU: calls that overlap on the device
// (concurrent streams, threads) race on it and must be serialised by the
// caller.  Its counters are cleared at the start of every call.  The array's
// device address is looked up once per device, on the first call there, and
// kept for the life of the process: after cudaDeviceReset the kept address is
// stale, so a process that resets a device must not call this entry point on
// it again.
#include <mutex>

#include "lodgs_internal.cuh"

namespace lodgs {
namespace {

constexpr int64_t NA_MAX_SPT = LODGS_NOALLOC_MAX_SPT;
// word offsets inside the scratch array
constexpr size_t NA_CNT = 0;                                  // C_COUNT counters
constexpr size_t NA_VIEW = 64;                                // the view (camera constants)
constexpr size_t NA_BLOCK = 256;                              // 1024 block counts
static_assert(sizeof(View) <= (NA_BLOCK - NA_VIEW) * 4, "the view must fit its slot");
constexpr size_t NA_BSUM = NA_BLOCK + SEL_BLOCK_COUNTS;       // scan block sums
constexpr size_t NA_EMIT_J = NA_BSUM + 256;                   // n_spt SPT indices
constexpr size_t NA_EMIT_X = NA_EMIT_J + NA_MAX_SPT;          // n_spt query values
constexpr size_t NA_HIGH = NA_EMIT_X + NA_MAX_SPT;            // n_spt + 1 prefix lengths
constexpr size_t NA_WORK = NA_HIGH + NA_MAX_SPT + 64;         // n_spt + 1 prefix offsets
constexpr size_t NA_WORDS = NA_WORK + NA_MAX_SPT + 64;        // ~16 MiB in total
// the scans of this path cover at most NA_MAX_SPT values, which take the
// short-scan grid (SCAN_GRID blocks)
static_assert(SCAN_GRID <= 256, "scan block sums must fit their slot");

static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

std::mutex g_mu;
uint32_t *g_scratch_ptr[256] = {};     // device address of the array, per device

// Host code may not use the array's name as a device address: fetch the real
// address once per device, with that device current.
int scratch_for_current_device(uint32_t **out) {
    int dev = 0;
    LODGS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) { set_error("select_lod_noalloc: device index out of range"); return LODGS_E_INVALID; }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "select_lod_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return LODGS_OK;
}

}  // namespace
}  // namespace lodgs

using namespace lodgs;

extern "C" int lodgs_select_lod_noalloc(lodgs_scene *scene, const lodgs_camera *cam, uint32_t *d_rows,
                                        int64_t capacity, uint32_t *d_count, void *stream) {
    if (!scene || !cam || !d_rows || !d_count) {
        set_error("select_lod_noalloc: NULL argument");
        return LODGS_E_INVALID;
    }
    if (capacity < scene->n_nodes) {
        set_error("select_lod_noalloc: capacity must be at least the scene's node count (" +
                  std::to_string(scene->n_nodes) + ")");
        return LODGS_E_INVALID;
    }
    if (scene->n_spt > NA_MAX_SPT) {
        set_error("select_lod_noalloc: the scene has " + std::to_string(scene->n_spt) +
                  " SPTs, more than the static scratch holds (" + std::to_string(NA_MAX_SPT) + ")");
        return LODGS_E_INVALID;
    }
    if (!camera_ok(cam)) {
        set_error("select_lod_noalloc: invalid camera");
        return LODGS_E_INVALID;
    }
    uint32_t *s = nullptr;
    if (int rc = scratch_for_current_device(&s)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    FrameBufs f;
    f.cnt = s + NA_CNT;
    f.d_view = reinterpret_cast<View *>(s + NA_VIEW);
    f.block_counts = s + NA_BLOCK;
    f.scan_bsum = s + NA_BSUM;
    f.emit_j = s + NA_EMIT_J;
    f.emit_x = reinterpret_cast<float *>(s + NA_EMIT_X);
    f.high = s + NA_HIGH;
    f.work_off = s + NA_WORK;
    f.sel_rows = d_rows;
    LODGS_CUDA(cudaMemsetAsync(f.cnt, 0, C_COUNT * sizeof(uint32_t), st));
    View v{};
    v.k = make_camk(*cam);
    if (int rc = launch_set_view(v, f.d_view, st)) return rc;   // a kernel argument: no staging buffer
    if (int rc = launch_select(scene, f, st)) return rc;
    LODGS_CUDA(cudaMemcpyAsync(d_count, f.cnt + C_NSEL, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    return LODGS_OK;
}
