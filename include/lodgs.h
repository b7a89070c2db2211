/*
 * lodgs.h -- C ABI of the B300-native LoD Gaussian render path.
 *
 * Method: "A LoD of Gaussians" (arxiv 2507.01110).  Given Gaussians and their
 * hierarchy, a camera and an LoD threshold, select a proper cut of the
 * hierarchical SPT (Sec. 4.3, Algorithms 1-2, Eq. 4/6), render it with the 3DGS
 * tile rasterizer (Sec. 3, Eq. 1-2) and return gradients for the cut's
 * parameters (Appendix "Implementation Details"; only cut-set nodes receive
 * gradients).
 *
 * Conventions
 *  - Every call returns a status code (LODGS_OK = 0, negative on error) and
 *    never throws or aborts; lodgs_last_error() gives a message for the calling
 *    thread.
 *  - Pointers are plain host or device pointers; sizes are element counts.
 *    Streams are cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Calls that take a stream only enqueue work; results are valid once that
 *    stream has been synchronised.  They do not synchronise the device.
 *  - Node records are float32 rows of `stride` floats (stride = 14 + 3K rounded
 *    up to a multiple of 8, K = (D+1)^2 - 1 SH coefficients per channel):
 *      [0:3] mean, [3:6] scales (linear), [6:10] quaternion (w,x,y,z, need not
 *      be normalised), [10] opacity in [0,1], [11:14] base colour,
 *      [14:14+3K] SH coefficients of degrees 1..D, coefficient-major, RGB-minor.
 *  - Cameras: world->camera rotation R (row-major; rows = right, down,
 *    forward), camera centre `pos` in world units, pinhole intrinsics in
 *    pixels; pixel (x, y) covers [x, x+1) x [y, y+1), its centre is +0.5.
 *  - Images are float32 H x W x 3 (row-major, RGB interleaved), device memory
 *    owned by the caller.
 */
#ifndef LODGS_H
#define LODGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LODGS_OK 0
#define LODGS_E_INVALID (-1)   /* bad argument or size */
#define LODGS_E_OOM (-2)       /* device or pinned allocation failed */
#define LODGS_E_CUDA (-3)      /* a CUDA runtime call failed */
#define LODGS_E_TIMEOUT (-4)   /* a bounded device wait ran out */
#define LODGS_E_STATE (-5)     /* call out of order (e.g. backward before render) */
#define LODGS_E_CAPACITY (-6)  /* a frame buffer was too small; grown, re-run the frame */

typedef struct lodgs_scene lodgs_scene; /* opaque, library-owned */
typedef struct lodgs_frame lodgs_frame; /* opaque per-view state and workspace, library-owned */

typedef struct {
    float R[9];        /* world->camera rotation, row-major */
    float pos[3];      /* camera centre, world */
    float fx, fy, cx, cy;
    int32_t width, height;
    float tau;         /* LoD threshold in pixels (projected size of a node, Eq. 6 reading) */
    float znear;       /* near plane, > 0 */
    float spt_scale;   /* factor on the distances to the SPT roots (training LoD noise, 1 + 5 r^4 with
                          r ~ U(0, 1), appendix "Varying level of detail"); 1 = none, 0 is read as 1 */
} lodgs_camera;

typedef struct {
    float spt_volume;  /* HSPT volume threshold `size` of Sec. 4.3: s1*s2*s3 < size roots an SPT */
    float kappa;       /* smallest focal/tau (pixels per world unit) the scene will be cut for;
                          folds the focal normalisation of the appendix into the SPT intervals */
} lodgs_build_params;

typedef struct {
    int64_t n_leaves, n_nodes;       /* n_nodes = 2 n_leaves - 1 (every internal node has two children) */
    int64_t n_upper;                 /* entries of the upper hierarchy (BFS order), SPT roots included */
    int64_t n_upper_rows;            /* upper nodes that are not SPT roots (render rows 0..n_upper_rows-1) */
    int64_t n_spt;                   /* number of SPTs */
    int32_t sh_degree, stride;
    float *d_rows;                   /* device, library-owned: n_nodes x stride records in render-row order */
    int64_t root;                    /* canonical id of the root (n_nodes-1 until a densification moves it) */
    int64_t layout_version;          /* 0 after the build, +1 per lodgs_scene_densify */
} lodgs_scene_info;

typedef struct {
    int64_t n_selected;              /* cut size (Algorithms 1-2) */
    int64_t n_upper_selected;        /* of which upper-hierarchy nodes */
    int64_t n_spt_cut;               /* SPTs handed to Algorithm 2 */
    int64_t n_spt_scanned;           /* SPT entries tested, sum of the binary-search prefixes */
    int64_t n_visible;               /* selected nodes in front of the near plane with a non-empty tile rect */
    int64_t n_pairs;                 /* (Gaussian, tile) pairs whose support reaches the tile (blended) */
    int32_t status;                  /* LODGS_OK, or LODGS_E_CAPACITY / LODGS_E_TIMEOUT from the device */
    int32_t width, height;
} lodgs_frame_stats;

/* Number of kernels this library has launched in this process (all streams). */
uint64_t lodgs_kernel_launches(void);

/* Thread-local message for the last failing call of this thread. */
const char *lodgs_last_error(void);

/*
 * Host-side fault injection, for tests of the error paths (nothing faults,
 * traps or hangs on the device): the call at `site` after `after` more
 * successful ones fails as documented, once; after < 0 disarms.  Sites:
 *   LODGS_FAULT_STREAM  lodgs_stream_nodes returns LODGS_E_CUDA before it
 *                       changes any cache or frame state (a failed copy);
 *   LODGS_FAULT_ALLOC   a frame workspace allocation (lodgs_frame_create or a
 *                       growth) returns LODGS_E_OOM before releasing the old
 *                       buffer (device memory exhausted);
 *   LODGS_FAULT_RENDER  lodgs_render returns LODGS_E_OOM before enqueuing
 *                       anything (a render whose workspace cannot grow).
 * Process-wide; LODGS_E_INVALID for an unknown site.
 */
#define LODGS_FAULT_STREAM 1
#define LODGS_FAULT_ALLOC 2
#define LODGS_FAULT_RENDER 3
#define LODGS_FAULT_SITES 3
int lodgs_debug_inject_fault(int site, int64_t after);
/* Library version string. */
const char *lodgs_version(void);

/*
 * Build the scene from leaf Gaussians (Sec. 3 "Gaussian Hierarchies"; Sec. 4.3
 * HSPT construction).  Leaves are merged pairwise, level by level, in Morton
 * order (moment-matched mean and covariance, weights opacity x surface term);
 * the hierarchy is cut by a BFS on the volume test into the upper hierarchy and
 * SPT roots; each SPT's nodes are laid out by descending parent bound (Eq. 4)
 * with the conservative spread term of Sec. 4.1 and top-down clamping
 * (appendix "Unreachable Gaussians").
 *   leaves: n x stride float32 records (layout above), host or device
 *           (leaves_on_device != 0); read only during the call.
 *   n >= 1, 0 <= sh_degree <= 3.  Synchronous.  *out is owned by the caller
 *   and released with lodgs_scene_free.
 */
int lodgs_build_hierarchy(const float *leaves, int64_t n, int sh_degree, int leaves_on_device,
                          const lodgs_build_params *params, lodgs_scene **out);
void lodgs_scene_free(lodgs_scene *scene);
int lodgs_scene_get_info(const lodgs_scene *scene, lodgs_scene_info *info);

/*
 * Copy the scene structure to host buffers (any pointer may be NULL to skip).
 * Canonical node ids: leaves 0..n-1 in input order, internal nodes n.. in merge
 * order, root n_nodes-1; after lodgs_scene_densify the ids it documents.
 *   node_rec   n_nodes x stride   records by canonical id
 *   left,right n_nodes            children (-1 for leaves)
 *   up_node, up_kind (0 internal, 1 leaf, 2 SPT root), up_parent, up_ref
 *              n_upper            upper hierarchy in BFS order; ref = render row or SPT index
 *   spt_root, spt_base, spt_count n_spt
 *   node_of_row n_nodes; lo_row, hi_row n_nodes (NaN for upper rows)
 * Synchronous.
 */
int lodgs_scene_export(const lodgs_scene *scene, float *node_rec, int64_t *left, int64_t *right,
                       int64_t *up_node, int32_t *up_kind, int64_t *up_parent, int64_t *up_ref,
                       int64_t *spt_root, int64_t *spt_base, int64_t *spt_count,
                       int64_t *node_of_row, float *lo_row, float *hi_row);

/*
 * Checkpoint of a scene (training resumes from it): the canonical node records,
 * the children of every node, the root, the SH degree and the build parameters,
 * with a checksum.  lodgs_scene_load validates the file (magic, header,
 * checksum, one full binary tree over all nodes: LODGS_E_INVALID otherwise) and
 * rebuilds the HSPT and SPT layout, which is deterministic: the loaded scene's
 * render rows, intervals and upper hierarchy equal the saved scene's, so per-row
 * state saved beside it (Adam moments) stays valid.  Synchronous.  Save needs
 * the scene's records on the device (LODGS_E_STATE after a cache released them).
 */
int lodgs_scene_save(const lodgs_scene *scene, const char *path);
int lodgs_scene_load(const char *path, lodgs_scene **out);

/*
 * Densification by moving Gaussians (Sec. 3 "Densification"): a batch of
 * operations on leaves, after which the HSPT and SPT layout are rebuilt
 * (Sec. 4.3, Algorithm 1 split and Sec. 4.1 intervals) with the scene's
 * build parameters.
 *   LODGS_DENSIFY_SPAWN    leaf `target` becomes an internal node with two new
 *                          leaf children (canonical ids n_nodes, n_nodes+1 in
 *                          operation order); n_nodes grows by 2.
 *   LODGS_DENSIFY_RESPAWN  leaf `dead` and its parent P leave their places: the
 *                          sibling of `dead` takes P's place under P's parent
 *                          (or becomes the root), and P and `dead` become the
 *                          two children of leaf `target`; n_nodes is unchanged.
 * In both, the two children carry the split of the target's record (the
 * 3DGS-MCMC split with two copies): its mean, rotation and colour; opacity
 * o' = 1 - sqrt(1 - o); scales times o / (2 o' - o'^2 / sqrt 2) (float32 as
 * written, sqrt 2 rounded to float32); the target keeps its own record and
 * becomes their parent.  `target` and `dead` are render rows of the
 * layout before the call and must be leaves of it; a node made by an earlier
 * operation of the same batch cannot be a target or dead, and `dead` != `target`.
 * ops[i].dead is ignored for SPAWN.
 *   old_row_of_new_row  device int32, capacity >= the new n_nodes: for each render
 *                       row of the new layout, the row the node held before the
 *                       call, or -1 for a node whose record is new (the
 *                       children).  Per-row state follows it through
 *                       lodgs_gather_rows.
 * The host edits only the nodes the operations touch (values gathered on the
 * device, changes scattered back); records, layout and row map are built on the
 * device.
 * Render rows are renumbered: frames and caches created before the call are
 * rejected afterwards (LODGS_E_STATE) and must be recreated.  Requires the
 * scene's records on the device (LODGS_E_STATE after a cache released them).
 * Invalid operations leave the scene unchanged (LODGS_E_INVALID).  Synchronous.
 */
#define LODGS_DENSIFY_SPAWN 0
#define LODGS_DENSIFY_RESPAWN 1
typedef struct {
    int32_t kind;      /* LODGS_DENSIFY_SPAWN or LODGS_DENSIFY_RESPAWN */
    int32_t pad_;
    int64_t target;    /* render row of a leaf to split */
    int64_t dead;      /* RESPAWN: render row of the leaf that is moved */
} lodgs_densify_op;
int lodgs_scene_densify(lodgs_scene *scene, const lodgs_densify_op *ops, int64_t n_ops,
                        int32_t *old_row_of_new_row, int64_t capacity);

/*
 * The operations of one densification step, planned on the device (Sec. 3
 * "Densification": candidates by maximal screen-space gradient, the
 * hierarchical 3DGS criterion; dead leaves respawned; appendix edge cases):
 *   dead:      leaves with a parent whose opacity (record column 10 of `rows`)
 *              is below min_opacity or whose stale flag is set, except the
 *              left child of a node whose two children are dead;
 *   candidate: leaves that are neither transparent nor stale, with
 *              grad_max >= grad_threshold, largest first, ties by row.
 * The i-th dead row is respawned under the i-th candidate; the remaining
 * candidates spawn while n_nodes + 2 * spawns <= max_nodes (max_nodes < 0:
 * no budget).  ops receives the spawns, then the respawns, in the order
 * lodgs_scene_densify applies them.
 *   rows:      device records in render-row order (NULL = the scene's own)
 *   grad_max:  device float per render row (lodgs_frame_screen_grad_max)
 *   stale:     device uint8 per render row, nonzero = stale, or NULL
 *   ops:       host, `capacity` entries; *n_ops = operations planned (also
 *              when capacity is too small: LODGS_E_INVALID), *n_spawn of them
 *              spawns.
 * Synchronises `stream`.
 */
int lodgs_densify_plan(lodgs_scene *scene, const float *rows, const float *grad_max, const uint8_t *stale,
                       float grad_threshold, float min_opacity, int64_t max_nodes, lodgs_densify_op *ops,
                       int64_t capacity, int64_t *n_ops, int64_t *n_spawn, void *stream);

/* Per-view state: selection, projected splats, sorted pairs and workspace.
 * Buffers grow on demand; a frame may be reused for any camera and resolution
 * of its scene.  A frame must not be used by two streams at once. */
int lodgs_frame_create(lodgs_scene *scene, lodgs_frame **out);
void lodgs_frame_free(lodgs_frame *frame);

/*
 * Set the frame's view: the camera (if cam != NULL) and the background (if
 * bg != NULL, host RGB).  The view is uploaded on `stream` and read by the
 * kernels from device memory, so a CUDA graph captured from
 * lodgs_select_lod(scene, NULL, ...) + lodgs_render(..., bg = NULL, ...) +
 * lodgs_render_backward can be replayed for any camera of the same resolution
 * after a lodgs_frame_set_view outside the graph.  Asynchronous.
 */
int lodgs_frame_set_view(lodgs_frame *frame, const lodgs_camera *cam, const float *bg, void *stream);

/*
 * LoD cut for one camera (Algorithm 1 on the upper hierarchy with frustum
 * culling, Sec. 4.3; Algorithm 2 per SPT at the shared root distance, Eq. 4).
 * A node is fine enough when its projected size f*S/d <= tau.  The selected
 * render rows (ascending) stay in the frame.  cam == NULL uses the view set on
 * the frame (lodgs_frame_set_view).  Asynchronous on `stream`.
 */
int lodgs_select_lod(lodgs_scene *scene, const lodgs_camera *cam, lodgs_frame *frame, void *stream);

/*
 * The LoD cuts of n views at once (Algorithms 1-2, as lodgs_select_lod for
 * each): cams[i] is cut into frames[i], with one launch of each selection pass
 * serving all n views (a view index in the grid), so n short, latency-bound
 * selections cost about as many launches as one.  Afterwards each frame is
 * exactly as lodgs_select_lod(scene, &cams[i], frames[i], stream) leaves it;
 * its render may run on another stream (it is ordered after the selection).
 *   cams:   host array of n cameras
 *   frames: host array of n distinct frames of this scene
 *   n:      1 <= n <= LODGS_SELECT_BATCH_MAX
 * LODGS_E_INVALID for a bad n, camera or repeated frame, with nothing
 * enqueued.  Asynchronous on `stream`.  Interface addition for serving and
 * multi-view batches; the paper selects one camera at a time.
 */
#define LODGS_SELECT_BATCH_MAX 8
int lodgs_select_lod_batch(lodgs_scene *scene, const lodgs_camera *cams, lodgs_frame *const *frames, int n,
                           void *stream);

/*
 * The same LoD cut as lodgs_select_lod, written to caller-owned device buffers,
 * for callers that cannot allocate device memory: an application whose device
 * memory all belongs to its own arena or pool, or a loop that cannot afford
 * cudaMalloc's device synchronisation.  The paper has no counterpart; this is
 * an interface variant only.  It allocates nothing: its scratch is a static
 * device array of about 16 MiB that every GPU loading the library keeps until
 * the process exits.
 *   d_rows:   device uint32 buffer, capacity >= the scene's n_nodes; receives
 *             the selected render rows, ascending
 *   d_count:  device uint32; receives the number of selected rows
 * Scenes with more than LODGS_NOALLOC_MAX_SPT SPTs, a smaller capacity, or a
 * camera lodgs_select_lod would refuse, are rejected with LODGS_E_INVALID.
 * All calls on a GPU share the scratch and each call clears it first: calls
 * that overlap on the device race, so serialise them.  The first call on a
 * device looks up the scratch address (cudaGetSymbolAddress) and keeps it for
 * the life of the process; make that first call before any stream capture,
 * and do not call this entry point again on a device after cudaDeviceReset.
 * Asynchronous.
 */
#define LODGS_NOALLOC_MAX_SPT (1 << 20)
int lodgs_select_lod_noalloc(lodgs_scene *scene, const lodgs_camera *cam, uint32_t *d_rows, int64_t capacity,
                             uint32_t *d_count, void *stream);

/*
 * Out-of-core mode (Sec. 4.4 "Caching on the GPU", Eq. 7, Algorithm 3): all
 * records in pinned host memory, the scene structure and the upper
 * hierarchy's records on the device, and a device slab of SPT records managed
 * LRU.  A miss streams the contiguous prefix of the SPT's records that the cut
 * can select (one cudaMemcpyAsync per SPT on a copy stream).
 */
typedef struct lodgs_cache lodgs_cache; /* opaque, library-owned */

typedef struct {
    int64_t capacity_bytes;  /* device slab for SPT records (the upper rows are extra) */
    float d_min, d_max;      /* reuse window of Eq. 7 on x_now / x_cached, x = tau d / f; [1,1] = exact */
    int32_t release_scene_rows; /* free the scene's device copy of the records after copying them to host */
    int32_t train;           /* keep Adam state (m, v, step counts) beside the records: pinned host arrays
                                and device slabs mirroring the record slab (3x the slab plus 4 B a record) */
} lodgs_cache_params;

typedef struct {
    int64_t spt_hits;        /* SPTs whose cached cut was reused (inside the Eq. 7 window) */
    int64_t spt_resident;    /* SPTs cut at the current distance from records already on the device */
    int64_t spt_loaded;      /* SPTs whose record prefix was copied from host memory */
    int64_t bytes_streamed;  /* host-to-device bytes issued for this view */
    int64_t evictions;       /* cached SPTs evicted (least recently used) for this view */
    int64_t cached_spts, cached_records;  /* cache contents after this view */
    int64_t bytes_written_back;  /* training caches: bytes of the trained SPT prefixes this view evicted; an
                                    upper bound, only rows trained since their load are copied
                                    (lodgs_cache_written_bytes) */
} lodgs_stream_stats;

/* Create the cache: copies the scene's records to pinned host memory (the
 * scene's device copy is freed if release_scene_rows), allocates the device
 * slab and copies the upper hierarchy's records.  Synchronous. */
int lodgs_cache_create(lodgs_scene *scene, const lodgs_cache_params *params, lodgs_cache **out);
void lodgs_cache_free(lodgs_cache *cache);
/* Drop every cached SPT (Sec. 4.4: the paper flushes the whole cache
 * periodically during training).  A training cache first writes its trained
 * rows and Adam state back to host memory (synchronous, after a device
 * synchronisation); otherwise host-side only. */
int lodgs_cache_flush(lodgs_cache *cache);

/*
 * Out-of-core training (Algorithm 3: optimise the cached nodes, write them back
 * when the LRU evicts them; Adam state in host memory beside the records).
 * lodgs_cache_adam_step: sparse Adam (lodgs_adam_step's update, hyper-parameters
 * and per-column lr[stride]) over the frame's selected rows in the cache's
 * device slabs.  `frame` must hold this cache's latest lodgs_stream_nodes view,
 * rendered with the cache's records and back-propagated (lodgs_render_backward,
 * sparse gradient rows `grads` in selection order, grad_capacity rows
 * allocated; no row at or past it is read).  Marks the view's SPTs
 * and the upper rows as trained.  Asynchronous on `stream`; the next
 * lodgs_stream_nodes orders its write-backs after it.  LODGS_E_STATE for a
 * cache created without `train`.
 * The rows of a trained SPT prefix that Adam updated since the prefix was loaded
 * are copied back to host memory (records, m, v, step counts) when it is
 * evicted, on the copy stream, ahead of any load into its range.
 * lodgs_cache_written_bytes: the bytes write-backs have copied to host memory
 * since the cache was created (synchronises the device).
 * lodgs_cache_writeback: copies every trained SPT prefix and the upper rows
 * back to host memory on `stream` (the cache keeps them); the host arrays are
 * current once `stream` has completed.
 * lodgs_cache_host_state: the pinned host arrays in render-row order: records
 * (n_nodes x stride), m, v (n_nodes x stride; NULL unless training), step
 * counts (n_nodes; NULL unless training).  Library-owned.
 */
int lodgs_cache_adam_step(lodgs_cache *cache, lodgs_frame *frame, const float *grads, int64_t grad_capacity,
                          const float *lr, float b1, float b2, float eps, void *stream);
int lodgs_cache_writeback(lodgs_cache *cache, void *stream);
int lodgs_cache_host_state(lodgs_cache *cache, float **h_rows, float **h_m, float **h_v, uint32_t **h_t);
int lodgs_cache_written_bytes(lodgs_cache *cache, int64_t *bytes);
/* Device records to pass as `rows` to lodgs_render / lodgs_render_backward for
 * frames selected with lodgs_stream_nodes (upper rows, then the slab). */
int lodgs_cache_records(lodgs_cache *cache, float **d_records);

/*
 * LoD cut of one camera through the cache, replacing lodgs_select_lod for
 * out-of-core scenes: upper cut on `stream`, one host synchronisation to take
 * the per-SPT cache decisions (hit / resident / load), copies of missing
 * prefixes on `copy_stream`, then the SPT cut on `stream`, which is made to
 * wait for the copies.  Renders that read the cache must run on `stream` (or
 * be complete) before the next call, because evicted slab ranges are reused.
 * Returns LODGS_E_CAPACITY if one view's SPT records do not fit the slab.
 */
int lodgs_stream_nodes(lodgs_scene *scene, lodgs_cache *cache, const lodgs_camera *cam, lodgs_frame *frame,
                       void *stream, void *copy_stream, lodgs_stream_stats *stats);

/* Device pointer to the frame's selected rows (uint32, ascending) and, after a
 * stream sync, their count. */
int lodgs_frame_selection(lodgs_frame *frame, const uint32_t **d_rows, int64_t *n_selected);

/*
 * Render the frame's selection (Eq. 1-2): EWA projection with SH colour, tile x
 * depth sort, front-to-back blending per 16x16 tile with early stop at
 * transmittance 1e-4.
 *   rows:  device records in render-row order (NULL = the scene's own)
 *   bg:    host RGB background (NULL = the frame's current background, black
 *          unless set)
 *   image: device float32 H x W x 3, caller-owned
 * Asynchronous.  If a workspace buffer was too small the frame records
 * LODGS_E_CAPACITY in its status (lodgs_frame_get_stats), grows the buffer at
 * the next call, and the image must be rendered again.
 */
int lodgs_render(lodgs_scene *scene, lodgs_frame *frame, const float *rows, const float *bg,
                 float *image, void *stream);

/*
 * Backward of lodgs_render for the same frame, rows and bg (Eq. 1-2
 * differentiated): each tile's list is walked front to back again,
 * recomputing transmittance per tile (nothing per pixel is stored by the
 * forward); the colour behind each Gaussian is the forward's output minus the
 * colour composited in front of it.
 *   image:     device H x W x 3, the image the frame's last lodgs_render wrote,
 *              unchanged since
 *   dL_dimage: device H x W x 3
 *   grad_rows: device, caller-owned.  dense == 0: n_selected x stride rows, row i
 *              for the i-th selected node (lodgs_frame_selection order);
 *              dense != 0: n_nodes x stride by render row, only selected rows
 *              are written (the caller zeroes the rest).
 *   grad_capacity: rows allocated at grad_rows.  Dense needs n_nodes
 *              (LODGS_E_INVALID otherwise).  Sparse rows are checked on the
 *              device against the selection count: if they do not fit, nothing
 *              is written, the frame records LODGS_E_CAPACITY
 *              (lodgs_frame_get_stats) and its device row count
 *              (lodgs_frame_device_count) becomes 0.
 * Gradients are w.r.t. the stored record values (quaternion normalisation
 * included).  Asynchronous.
 */
int lodgs_render_backward(lodgs_scene *scene, lodgs_frame *frame, const float *rows, const float *bg,
                          const float *image, const float *dL_dimage, float *grad_rows, int64_t grad_capacity,
                          int dense, void *stream);

/*
 * Gradient of a multi-view batch loss: sums the per-view sparse gradient rows
 * (lodgs_render_backward with dense = 0) into one row per node of the union of
 * the views' cuts; only cut-set nodes receive gradients (appendix,
 * Implementation Details).  Deterministic: rows of a node are summed in view
 * order, without atomics.
 *   frames[v], grads[v]  the n_views rendered frames and their device gradient rows
 *              (NULL allowed for a view that selected nothing); rows of at
 *              most 64 floats (SH degree <= 3), read as float2 when every
 *              array is 8-byte aligned
 *   out_rows   device uint32, capacity >= sum of the views' selections: union rows, ascending
 *   out_grads  device float32, capacity x stride: the summed rows, in out_rows order
 *   d_count    device uint32: the union size
 * Temporary device memory (allocated and released in stream order): up to 8 views,
 * about 5 bytes per scene node plus 16 per entry (entries grouped by a byte of
 * view bits per node); for more views about 36 bytes per entry (a radix sort).
 * Synchronises the frames' streams, then runs asynchronously on `stream`.
 */
int lodgs_accumulate_grads(lodgs_scene *scene, lodgs_frame *const *frames, const float *const *grads, int n_views,
                           uint32_t *out_rows, float *out_grads, int64_t capacity, uint32_t *d_count, void *stream);

/*
 * Row gather for per-row state across a densification (its old_row_of_new_row):
 * dst[r] = src[src_row[r]] for r < n_rows, each row `row_words` 32-bit words
 * (floats or step counts alike); rows whose src_row is -1 (or >= n_src) are
 * zero, the fresh state of a new node.  src (n_src rows), dst (n_rows rows) and
 * src_row (n_rows int32) are device pointers; src and dst must not overlap.
 * Asynchronous on `stream`.
 */
int lodgs_gather_rows(const void *src, int64_t n_src, void *dst, const int32_t *src_row, int64_t n_rows,
                      int32_t row_words, void *stream);

/*
 * Sparse Adam step over the cut set (appendix "Implementation Details": only
 * the nodes of the cut are optimised; Adam after Kingma and Ba).  For each of
 * the n listed rows r = rows[i] (unique) with gradient row grads[i] (stride
 * floats, the layout of lodgs_render_backward's sparse rows or of
 * lodgs_accumulate_grads' output), t[r] += 1 and for every record column c that
 * the SH degree uses:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   p -= lr[c] (m / (1 - b1^t[r])) / (sqrt(v / (1 - b2^t[r])) + eps)
 * so each row's bias correction counts the steps it took part in.
 *   params, m, v: device float32 n_nodes x stride (render-row order, e.g. the
 *                 scene's own records); m, v, t zeroed by the caller before the
 *                 first step
 *   t:            device uint32 n_nodes
 *   d_n:          device uint32 count of rows (NULL: exactly max_n rows);
 *                 max_n bounds it (grid sizing)
 *   lr:           host float[stride] per-column learning rates
 * Asynchronous.  The update is w.r.t. the stored values (activations are the
 * caller's, as for the gradients).
 */
int lodgs_adam_step(lodgs_scene *scene, float *params, float *m, float *v, uint32_t *t, const uint32_t *rows,
                    const float *grads, const uint32_t *d_n, int64_t max_n, const float *lr, float b1, float b2,
                    float eps, void *stream);

/*
 * Densification criterion (Sec. 3: nodes are split where the screen-space
 * gradient is largest): after lodgs_render_backward on `frame`, for every
 * selected node max_per_node[row] = max(max_per_node[row], |dL/d(u, v)|), the
 * norm of the gradient w.r.t. the projected mean.  max_per_node: device float
 * n_nodes, zeroed by the caller.  Asynchronous on `stream`.
 */
int lodgs_frame_screen_grad_max(lodgs_frame *frame, float *max_per_node, void *stream);

/* Device pointer to the frame's count of selected nodes as its last render
 * processed them (uint32, valid while the frame lives): the row count of its
 * sparse gradient rows, for lodgs_adam_step without a host synchronisation. */
int lodgs_frame_device_count(lodgs_frame *frame, const uint32_t **d_n_selected);

/*
 * Photometric L1 loss of a rendered image against a target (the training loss
 * of the benchmark step) fused with its gradient, in one pass over device
 * buffers of n floats (16-byte aligned): dL[i] = grad_scale * sign(image[i] -
 * target[i]) and *loss_sum = sum |image[i] - target[i]| (device float,
 * overwritten).  For the mean loss pass grad_scale = 1/n and divide the sum by n.
 * Not part of the paper's method: its loss is the training objective around it.
 */
int lodgs_l1_loss_grad(const float *image, const float *target, int64_t n, float grad_scale, float *dL,
                       float *loss_sum, void *stream);

/* The two halves of lodgs_render_backward, for callers that schedule them
 * separately (e.g. as separate CUDA graphs): the blend backward (per-pixel
 * recomputation, 2D gradients kept in the frame), then the projection backward
 * into gradient rows (same meaning of rows, grad_rows, grad_capacity, dense). */
int lodgs_render_backward_blend(lodgs_scene *scene, lodgs_frame *frame, const float *image, const float *dL_dimage,
                                void *stream);
int lodgs_render_backward_project(lodgs_scene *scene, lodgs_frame *frame, const float *rows, float *grad_rows,
                                  int64_t grad_capacity, int dense, void *stream);

/*
 * The blend backward of the mean-L1 training step with the loss folded in:
 * dL/dC = grad_scale * sign(image - target) is formed per pixel inside the
 * backward (no dL/dC buffer, no separate pass over the image), and
 * *loss_sum = sum |image - target| over the image (device float, overwritten;
 * grad_scale = 1/n and loss_sum / n give the mean).  target: device H x W x 3
 * float32.  The same results as lodgs_l1_loss_grad followed by
 * lodgs_render_backward_blend, up to the order of float atomic sums.
 * Not part of the paper's method: its loss is the training objective around it.
 */
int lodgs_render_backward_blend_l1(lodgs_scene *scene, lodgs_frame *frame, const float *image, const float *target,
                                   float grad_scale, float *loss_sum, void *stream);

/*
 * lodgs_render_backward_blend_l1 with an 8-bit target (device H x W x 3
 * uint8, the format training photographs are stored in): each byte t is read
 * as t / 255, correctly rounded to float32, so the results equal those of
 * lodgs_render_backward_blend_l1 on that float32 target, up to the order of
 * float atomic sums.  A quarter of the float target's bytes to upload.
 */
int lodgs_render_backward_blend_l1_u8(lodgs_scene *scene, lodgs_frame *frame, const float *image,
                                      const uint8_t *target, float grad_scale, float *loss_sum, void *stream);

/* Counters of the last select/render on this frame (blocks until `stream`,
 * the stream the frame last ran on, is idle). */
int lodgs_frame_get_stats(lodgs_frame *frame, lodgs_frame_stats *stats);

/*
 * Device memory of a frame, for callers that budget it (a render server that
 * admits requests by memory).  The paper has no counterpart; this is an
 * interface addition only.
 *   held_bytes:   what the frame's workspace holds now: the buffers sized by
 *                 the scene at creation plus the per-selected-node, per-pair
 *                 and per-tile buffers as grown so far (they never shrink)
 *   needed_bytes: what the same buffers take when sized exactly for the
 *                 frame's last view (its selection, and its kept pairs and
 *                 tiles if it was rendered)
 * Either pointer may be NULL.  Synchronises the frame's stream.
 */
int lodgs_frame_memory(lodgs_frame *frame, int64_t *held_bytes, int64_t *needed_bytes);

/*
 * Sizes a frame's per-view buffers for a view of n_selected selected nodes and
 * n_pairs kept (Gaussian, tile) pairs: grows them now where they are smaller
 * (they never shrink), and makes this the size the next render grows to,
 * replacing any growth that a capacity overflow (LODGS_E_CAPACITY) queued.
 * (0, 0) keeps the current size and cancels queued growth: a caller that
 * budgets device memory can then move the overflowing view to a larger frame
 * instead of letting this one grow.  Interface addition; the paper has no
 * counterpart.  LODGS_E_OOM if an allocation fails.
 */
int lodgs_frame_reserve(lodgs_frame *frame, int64_t n_selected, int64_t n_pairs);

/* Stages timed by lodgs_frame_stage_ms, in order. */
#define LODGS_STAGE_SELECT 0      /* upper-hierarchy BFS cut + SPT interval test and compaction */
#define LODGS_STAGE_PROJECT 1     /* gather + EWA projection + SH colour */
#define LODGS_STAGE_COUNT 2       /* per tile: pair scan, tile test, counts, ranges; global: depth sort */
#define LODGS_STAGE_EMIT 3        /* per tile: scatter into tiles; global: pair emission in depth order */
#define LODGS_STAGE_TILE_SORT 4   /* per tile: sort of each tile's list; global: radix sort by tile + ranges */
#define LODGS_STAGE_BLEND 5       /* front-to-back blending */
#define LODGS_STAGE_BLEND_BWD 6   /* backward of the blend (per-tile recomputation) */
#define LODGS_STAGE_PROJECT_BWD 7 /* backward of the projection + gradient rows */
#define LODGS_NUM_STAGES 8

/* Record CUDA events around the stages of this frame: on < 0 all stages, 0
 * none, > 0 a bit mask of LODGS_STAGE_* bits (1 << stage). */
int lodgs_frame_set_profiling(lodgs_frame *frame, int on);
/* Device time in milliseconds of each stage of the last select/render/backward
 * on this frame (LODGS_NUM_STAGES floats; 0 for stages that did not run since
 * the last select).  Blocks until the frame's stream is idle. */
int lodgs_frame_stage_ms(lodgs_frame *frame, float *ms);

/*
 * How lodgs_render puts the (tile, Gaussian) pairs in (tile, depth key,
 * selected index) order -- the result is the same either way:
 *   LODGS_ORDER_PER_TILE  pairs counted and scattered per tile, each tile's list
 *                         sorted by one block (few launches; best for short lists)
 *   LODGS_ORDER_GLOBAL    stable radix sort of the selection by depth, pairs
 *                         emitted in that order, stable radix sort by tile
 *                         (best for long tile lists)
 *   LODGS_ORDER_AUTO      per tile while the frame's pair workspace averages at
 *                         most 1024 pairs per tile, global beyond (default)
 */
#define LODGS_ORDER_AUTO 0
#define LODGS_ORDER_PER_TILE 1
#define LODGS_ORDER_GLOBAL 2
int lodgs_frame_set_ordering(lodgs_frame *frame, int mode);

/* Pixel-Gaussian work of the last render/backward on this frame (4 uint64):
 * [0] forward support tests evaluated, [1] forward blends (alpha composited),
 * [2] backward support tests, [3] backward contributions.  Tests skipped by
 * the 8x8-block support test are not counted; [2] and [3] are 0 after a render
 * until the backward runs.  The counters are tallied only while the frame's
 * profiling is on (lodgs_frame_set_profiling); otherwise they read 0.
 * Blocks until the frame's stream is idle. */
int lodgs_frame_work(lodgs_frame *frame, uint64_t *work);

/*
 * Copy the frame's last render products to host buffers (inspection and
 * tests; any pointer may be NULL to skip).  Blocks until the frame's stream is
 * idle.
 *   pair_index  n_pairs uint32: selected index of each (tile, depth)-sorted pair
 *   ranges      2 x n_tiles uint32: [start, end) of each tile's pairs
 *   splats      n_selected x LODGS_SPLAT_FLOATS float32: u, v, A, B, C (conic of Eq. 2),
 *               opacity, r, g, b, rx, ry (support half extents of the 8x8-block test)
 *   depth_key   n_selected uint32: float32 bits of the view depth (0xffffffff if invisible)
 *   cap_pairs   capacity of pair_index in elements (LODGS_E_INVALID if too small)
 */
#define LODGS_SPLAT_FLOATS 11
int lodgs_frame_export(lodgs_frame *frame, uint32_t *pair_index, int64_t cap_pairs, uint32_t *ranges,
                       float *splats, uint32_t *depth_key);

#ifdef __cplusplus
}
#endif
#endif /* LODGS_H */
