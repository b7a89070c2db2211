"""Python binding of the C ABI (include/lodgs.h), same names, torch for memory.

Every step of the render path runs in liblodgs.so; this module only converts
arguments (torch tensors -> device pointers, cameras -> structs) and retries a
frame once its workspace has grown (LODGS_E_CAPACITY).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import Camera as _Cam, check, lib


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous() and t.dtype == torch.float32, "need a contiguous float32 CUDA tensor"
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class _DeviceArray:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3, "strides": None}


def _device_view(ptr: int, shape, typestr: str) -> torch.Tensor:
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")


def camera_struct(cam) -> _Cam:
    """Convert a synth.Camera-like object (R, pos, fx, fy, cx, cy, width, height, tau, znear[, spt_scale])."""
    c = _Cam()
    R = np.asarray(cam.R, dtype=np.float32).reshape(9)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.pos[i] = float(np.float32(cam.pos[i]))
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    c.tau, c.znear = float(np.float32(cam.tau)), float(np.float32(cam.znear))
    c.spt_scale = float(np.float32(getattr(cam, "spt_scale", 1.0)))
    return c


# numpy mirror of lodgs_densify_op (int32 kind, int32 padding, int64 target, int64 dead)
_OP_DTYPE = np.dtype([("kind", np.int32), ("pad_", np.int32), ("target", np.int64), ("dead", np.int64)])
assert _OP_DTYPE.itemsize == C.sizeof(_lib.DensifyOp)


class Scene:
    """A built scene (library-owned device memory)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle
        self._refresh()

    def _refresh(self):
        info = _lib.SceneInfo()
        check(lib().lodgs_scene_get_info(self._h, C.byref(info)))
        self.n_leaves, self.n_nodes = info.n_leaves, info.n_nodes
        self.n_upper, self.n_upper_rows, self.n_spt = info.n_upper, info.n_upper_rows, info.n_spt
        self.sh_degree, self.stride = info.sh_degree, info.stride
        self.root, self.layout_version = info.root, info.layout_version
        self._rows_ptr = info.d_rows

    def densify(self, spawn=(), respawn=()) -> np.ndarray:
        """Densification by moving Gaussians (Sec. 3): `spawn` lists render rows of
        leaves that each get two new children; `respawn` lists (target, dead)
        pairs of leaf rows, where the dead leaf and its parent become the target's
        children.  Both carry the split of the target's record.  Operations run
        spawn first, then respawn, in list order.  Rebuilds the HSPT/SPT layout;
        frames and caches made earlier must be recreated.  Returns, per new
        render row, the row the node held before (-1 for the new children), as
        an int32 CUDA tensor, to carry per-row state such as Adam moments
        across (gather_rows)."""
        sp = np.asarray(spawn, dtype=np.int64).reshape(-1)
        rs = np.asarray(respawn, dtype=np.int64).reshape(-1, 2)
        n_ops = sp.size + rs.shape[0]
        arr = np.zeros(max(n_ops, 1), _OP_DTYPE)             # the layout of lodgs_densify_op
        arr["kind"][:sp.size] = _lib.DENSIFY_SPAWN
        arr["target"][:sp.size] = sp
        arr["dead"][:sp.size] = -1
        arr["kind"][sp.size:n_ops] = _lib.DENSIFY_RESPAWN
        arr["target"][sp.size:n_ops] = rs[:, 0]
        arr["dead"][sp.size:n_ops] = rs[:, 1]
        cap = self.n_nodes + 2 * sp.size
        out = torch.empty(cap, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        rc = lib().lodgs_scene_densify(self._h, C.c_void_p(arr.ctypes.data), n_ops, C.c_void_p(out.data_ptr()), cap)
        self._refresh()
        check(rc)
        return out[:self.n_nodes]

    @property
    def handle(self):
        return self._h

    def rows(self) -> torch.Tensor:
        """The scene's node records in render-row order (n_nodes x stride), a
        zero-copy view of library-owned device memory valid while the scene lives."""
        return _device_view(self._rows_ptr, (self.n_nodes, self.stride), "<f4")

    def plan_densify(self, grad_max: torch.Tensor, grad_threshold: float, min_opacity: float = 0.005,
                     max_nodes: int | None = None, stale: torch.Tensor | None = None,
                     rows: torch.Tensor | None = None, stream=None) -> tuple[list, list]:
        """The operations of one densification step, planned on the device
        (candidates by maximal screen-space gradient, dead leaves by opacity or
        the stale flag, the appendix's two-dead-siblings rule): (spawn rows,
        [(target row, dead row)]) for densify()."""
        assert grad_max.is_cuda and grad_max.dtype == torch.float32 and grad_max.numel() == self.n_nodes
        if stale is not None:
            stale = stale.to(device="cuda", dtype=torch.uint8).contiguous()
        n_ops, n_sp = C.c_int64(), C.c_int64()

        def run(cap):
            arr = np.zeros(max(cap, 1), _OP_DTYPE)
            rc = lib().lodgs_densify_plan(self._h, _ptr(rows), _ptr(grad_max.contiguous()),
                                          C.c_void_p(stale.data_ptr()) if stale is not None else None,
                                          C.c_float(grad_threshold), C.c_float(min_opacity),
                                          C.c_int64(-1 if max_nodes is None else int(max_nodes)),
                                          C.c_void_p(arr.ctypes.data), C.c_int64(cap), C.byref(n_ops),
                                          C.byref(n_sp), _stream_ptr(stream))
            return rc, arr

        rc, arr = run(1 << 16)
        if rc == _lib.LODGS_E_INVALID and n_ops.value > (1 << 16):
            rc, arr = run(n_ops.value)                 # more operations than the first buffer held
        check(rc)
        ns, n = n_sp.value, n_ops.value                # spawns first, then respawns
        spawn = arr["target"][:ns].tolist()
        respawn = list(zip(arr["target"][ns:n].tolist(), arr["dead"][ns:n].tolist()))
        return spawn, respawn

    def save(self, path) -> None:
        """Checkpoint: records, tree and build parameters (lodgs_scene_save)."""
        check(lib().lodgs_scene_save(self._h, str(path).encode()))

    def topology(self) -> dict:
        """Children (canonical ids, -1 for leaves), node_of_row and the root, copied
        to the host; what densification planning needs without the records."""
        M = self.n_nodes
        a = {"left": np.zeros(M, np.int64), "right": np.zeros(M, np.int64), "node_of_row": np.zeros(M, np.int64)}
        ptr = {k: C.c_void_p(v.ctypes.data) for k, v in a.items()}
        check(lib().lodgs_scene_export(self._h, None, ptr["left"], ptr["right"], None, None, None, None, None, None,
                                       None, ptr["node_of_row"], None, None))
        a["root"] = self.root
        return a

    def export(self) -> dict:
        M, U, S, st = self.n_nodes, self.n_upper, self.n_spt, self.stride
        a = {
            "node_rec": np.zeros((M, st), np.float32), "left": np.zeros(M, np.int64), "right": np.zeros(M, np.int64),
            "up_node": np.zeros(U, np.int64), "up_kind": np.zeros(U, np.int32), "up_parent": np.zeros(U, np.int64),
            "up_ref": np.zeros(U, np.int64), "spt_root": np.zeros(max(S, 1), np.int64),
            "spt_base": np.zeros(max(S, 1), np.int64), "spt_count": np.zeros(max(S, 1), np.int64),
            "node_of_row": np.zeros(M, np.int64), "lo_row": np.zeros(M, np.float32), "hi_row": np.zeros(M, np.float32),
        }
        order = ["node_rec", "left", "right", "up_node", "up_kind", "up_parent", "up_ref", "spt_root", "spt_base",
                 "spt_count", "node_of_row", "lo_row", "hi_row"]
        check(lib().lodgs_scene_export(self._h, *[C.c_void_p(a[k].ctypes.data) for k in order]))
        for k in ("spt_root", "spt_base", "spt_count"):
            a[k] = a[k][:S]
        a.update({"n_upper": U, "n_spt": S, "n_upper_rows": self.n_upper_rows, "stride": st,
                  "degree": self.sh_degree, "n_leaves": self.n_leaves, "root": self.root})
        return a

    def close(self):
        if self._h:
            lib().lodgs_scene_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Frame:
    """Per-view state of a scene (selection, splats, sorted pairs)."""

    def __init__(self, scene: Scene):
        self.scene = scene
        h = C.c_void_p()
        check(lib().lodgs_frame_create(scene.handle, C.byref(h)))
        self._h = h
        self.camera = None
        self.bg = (0.0, 0.0, 0.0)
        self.image = None           # tensor the last render wrote (read by render_backward)

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        s = _lib.FrameStats()
        check(lib().lodgs_frame_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _lib.FrameStats._fields_}

    def selection(self) -> torch.Tensor:
        """Selected render rows (int64, ascending) copied from the device."""
        p = C.c_void_p()
        n = C.c_int64()
        check(lib().lodgs_frame_selection(self._h, C.byref(p), C.byref(n)))
        if n.value == 0:
            return torch.zeros(0, dtype=torch.int64, device="cuda")
        return _device_view(p.value, (int(n.value),), "<u4").to(torch.int64)

    def selection_device(self) -> tuple:
        """(device address of the selected rows (uint32), device address of their count)
        -- the rows of the frame's sparse gradient rows, for adam_step without a copy."""
        p = C.c_void_p()
        n = C.c_int64()
        check(lib().lodgs_frame_selection(self._h, C.byref(p), C.byref(n)))
        return p.value, frame_device_count(self)

    ORDER_AUTO, ORDER_PER_TILE, ORDER_GLOBAL = 0, 1, 2

    def set_ordering(self, mode: int) -> None:
        """How renders order the (tile, Gaussian) pairs: Frame.ORDER_* (same result)."""
        check(lib().lodgs_frame_set_ordering(self._h, C.c_int(int(mode))))

    def set_profiling(self, on=True) -> None:
        """True: time every stage; False: none; a list of stage names: those."""
        if on is True:
            mask = -1
        elif not on:
            mask = 0
        else:
            mask = sum(1 << _lib.STAGES.index(s) for s in on)
        check(lib().lodgs_frame_set_profiling(self._h, C.c_int(mask)))

    def stage_ms(self) -> dict:
        """Device milliseconds per stage of the last select/render/backward."""
        ms = (C.c_float * len(_lib.STAGES))()
        check(lib().lodgs_frame_stage_ms(self._h, ms))
        return dict(zip(_lib.STAGES, [float(v) for v in ms]))

    def memory(self) -> tuple[int, int]:
        """(held, needed) device bytes: what the frame's workspace holds now, and
        what it takes sized exactly for the frame's last view (lodgs_frame_memory)."""
        held, needed = C.c_int64(), C.c_int64()
        check(lib().lodgs_frame_memory(self._h, C.byref(held), C.byref(needed)))
        return held.value, needed.value

    def reserve(self, n_selected: int = 0, n_pairs: int = 0) -> None:
        """Size the per-view buffers for n_selected nodes and n_pairs pairs (grow
        now, never shrink) and cancel growth a capacity overflow queued."""
        check(lib().lodgs_frame_reserve(self._h, C.c_int64(int(n_selected)), C.c_int64(int(n_pairs))))

    def work(self) -> dict:
        """Pixel-Gaussian work counters of the last render/backward."""
        w = (C.c_uint64 * 4)()
        check(lib().lodgs_frame_work(self._h, w))
        return {"fwd_eval": w[0], "fwd_blend": w[1], "bwd_eval": w[2], "bwd_contrib": w[3]}

    def export(self) -> dict:
        """Sorted pair order, tile ranges, splats and depth keys of the last render."""
        st = self.stats()
        cam = self.camera
        n_tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
        pairs = np.zeros(max(st["n_pairs"], 1), np.uint32)
        ranges = np.zeros((n_tiles, 2), np.uint32)
        spl = np.zeros((max(st["n_selected"], 1), 11), np.float32)   # u v A B C opacity r g b rx ry
        keys = np.zeros(max(st["n_selected"], 1), np.uint32)
        check(lib().lodgs_frame_export(self._h, C.c_void_p(pairs.ctypes.data), C.c_int64(pairs.size),
                                       C.c_void_p(ranges.ctypes.data), C.c_void_p(spl.ctypes.data),
                                       C.c_void_p(keys.ctypes.data)))
        return {"pair_i": pairs[: st["n_pairs"]], "ranges": ranges, "splats": spl[: st["n_selected"]],
                "depth_key": keys[: st["n_selected"]], "stats": st}

    def close(self):
        if self._h:
            lib().lodgs_frame_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cache:
    """Out-of-core node cache of a scene (records in pinned host memory)."""

    def __init__(self, scene: Scene, capacity_bytes: int, d_min: float = 0.9, d_max: float = 1.1,
                 release_scene_rows: bool = False, train: bool = False):
        self.scene = scene
        self.train = bool(train)
        p = _lib.CacheParams(int(capacity_bytes), float(d_min), float(d_max), int(release_scene_rows), int(train))
        h = C.c_void_p()
        check(lib().lodgs_cache_create(scene.handle, C.byref(p), C.byref(h)))
        self._h = h
        ptr = C.c_void_p()
        check(lib().lodgs_cache_records(self._h, C.byref(ptr)))
        rec = scene.stride * 4
        n = scene.n_upper_rows + int(capacity_bytes) // rec
        self.records = _device_view(ptr.value, (n, scene.stride), "<f4")

    @property
    def handle(self):
        return self._h

    def flush(self):
        """Drop every cached SPT (the paper's periodic cache flush); a training
        cache writes its trained rows and Adam state back first."""
        check(lib().lodgs_cache_flush(self._h))

    def adam_step(self, frame: Frame, grads: torch.Tensor, lr, b1: float = 0.9, b2: float = 0.999,
                  eps: float = 1e-15, stream=None) -> None:
        """Sparse Adam on the cached rows of the frame's view (after
        render_backward with rows=cache.records); lr: float or per-column."""
        lrv = np.broadcast_to(np.asarray(lr, dtype=np.float32), (self.scene.stride,)).copy()
        check(lib().lodgs_cache_adam_step(self._h, frame.handle, _ptr(grads),
                                          C.c_int64(_grad_rows_capacity(self.scene, grads)),
                                          lrv.ctypes.data_as(C.c_void_p),
                                          C.c_float(b1), C.c_float(b2), C.c_float(eps), _stream_ptr(stream)))

    def written_bytes(self) -> int:
        """Bytes the write-backs have copied to host memory since creation (only
        rows trained since their load are copied)."""
        b = C.c_int64()
        check(lib().lodgs_cache_written_bytes(self._h, C.byref(b)))
        return b.value

    def writeback(self, stream=None) -> None:
        """Copy every trained row (records and Adam state) back to host memory."""
        check(lib().lodgs_cache_writeback(self._h, _stream_ptr(stream)))

    def host_state(self) -> dict:
        """numpy views of the pinned host arrays (render-row order): rows, and
        for training caches m, v, t.  Current after writeback() and a sync."""
        ptrs = [C.c_void_p() for _ in range(4)]
        check(lib().lodgs_cache_host_state(self._h, *[C.byref(p) for p in ptrs]))
        M, st = self.scene.n_nodes, self.scene.stride
        out = {}
        for name, p, shape, ct in (("rows", ptrs[0], (M, st), C.c_float), ("m", ptrs[1], (M, st), C.c_float),
                                   ("v", ptrs[2], (M, st), C.c_float), ("t", ptrs[3], (M,), C.c_uint32)):
            if p.value:
                n = int(np.prod(shape))
                out[name] = np.ctypeslib.as_array((ct * n).from_address(p.value)).reshape(shape)
        return out

    def close(self):
        if self._h:
            lib().lodgs_cache_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stream_nodes(scene: Scene, cache: Cache, camera, frame: Frame | None = None, stream=None,
                 copy_stream=None) -> tuple[Frame, dict]:
    """LoD cut through the out-of-core cache; returns the frame and the view's
    streaming statistics.  Render it with rows=cache.records."""
    fr = frame if frame is not None else Frame(scene)
    cs = camera_struct(camera)
    st = _lib.StreamStats()
    cpy = copy_stream if copy_stream is not None else (stream or torch.cuda.current_stream())
    check(lib().lodgs_stream_nodes(scene.handle, cache.handle, C.byref(cs), fr.handle, _stream_ptr(stream),
                                   C.c_void_p(cpy.cuda_stream), C.byref(st)))
    fr.camera = camera
    return fr, {k: getattr(st, k) for k, _ in _lib.StreamStats._fields_}


def accumulate_grads(scene: Scene, frames: list, grads: list, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
    """Sum per-view sparse gradient rows over the union of the views' cuts.
    Returns (rows int64 ascending, summed gradient rows)."""
    n = len(frames)
    total = sum(int(g.shape[0]) for g in grads)
    out_rows = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    out_grads = torch.empty((max(total, 1), scene.stride), dtype=torch.float32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    fr_arr = (C.c_void_p * n)(*[f.handle.value for f in frames])
    g_arr = (C.c_void_p * n)(*[g.data_ptr() for g in grads])
    check(lib().lodgs_accumulate_grads(scene.handle, fr_arr, g_arr, C.c_int(n), C.c_void_p(out_rows.data_ptr()),
                                       C.c_void_p(out_grads.data_ptr()), C.c_int64(max(total, 1)),
                                       C.c_void_p(count.data_ptr()), _stream_ptr(stream)))
    k = int(count.item())
    return out_rows[:k].to(torch.int64), out_grads[:k]


def gather_rows(src: torch.Tensor, src_row, stream=None) -> torch.Tensor:
    """New tensor whose row r is src[src_row[r]], zeros where src_row[r] is -1
    (a densification's old_row_of_new_row; the gather runs in the library's
    kernel).  src: CUDA tensor of a 4-byte dtype, rows along dim 0."""
    assert src.is_cuda and src.element_size() == 4 and src.is_contiguous()
    if isinstance(src_row, torch.Tensor):
        idx = src_row.to(device="cuda", dtype=torch.int32).contiguous()
    else:
        idx = torch.as_tensor(np.ascontiguousarray(src_row, dtype=np.int32)).to("cuda", non_blocking=False)
    n = idx.numel()
    words = int(np.prod(src.shape[1:])) if src.dim() > 1 else 1
    out = torch.empty((n,) + tuple(src.shape[1:]), dtype=src.dtype, device="cuda")
    check(lib().lodgs_gather_rows(C.c_void_p(src.data_ptr()), C.c_int64(src.shape[0]), C.c_void_p(out.data_ptr()),
                                  C.c_void_p(idx.data_ptr()), C.c_int64(n), C.c_int32(words), _stream_ptr(stream)))
    if stream is not None:
        idx.record_stream(stream)        # freed on return: keep it until `stream` is done with it
    return out


class AdamState:
    """Sparse Adam state of a scene's records (device float32 m, v; uint32 step counts)."""

    def __init__(self, scene: Scene):
        self.m = torch.zeros((scene.n_nodes, scene.stride), dtype=torch.float32, device="cuda")
        self.v = torch.zeros_like(self.m)
        self.t = torch.zeros(scene.n_nodes, dtype=torch.int32, device="cuda")

    def remap(self, old_row_of_new_row) -> None:
        """Carry the state across a densification: each node keeps its moments
        and step count, new nodes start from zero (as 3DGS-MCMC resets the
        state of relocated Gaussians)."""
        self.m = gather_rows(self.m, old_row_of_new_row)
        self.v = gather_rows(self.v, old_row_of_new_row)
        self.t = gather_rows(self.t, old_row_of_new_row)


def adam_step(scene: Scene, params: torch.Tensor, state: AdamState, rows: torch.Tensor, grads: torch.Tensor, lr,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15, d_n=None, stream=None) -> None:
    """Sparse Adam step of the listed rows (uint32/int32 device tensor or a raw device
    pointer with d_n): params -= lr m_hat / (sqrt(v_hat) + eps), per-row step counts.
    lr: a float or a per-column sequence of `stride` floats."""
    lrv = np.broadcast_to(np.asarray(lr, dtype=np.float32), (scene.stride,)).copy()
    if isinstance(rows, torch.Tensor):
        n = rows.numel()
        rows = rows.to(torch.int32).contiguous()
        assert rows.is_cuda, "rows must be a CUDA tensor"
        rows_p = C.c_void_p(rows.data_ptr())
    else:
        rows_p, n = rows
    assert state.t.is_cuda and state.t.dtype == torch.int32
    check(lib().lodgs_adam_step(scene.handle, _ptr(params), _ptr(state.m), _ptr(state.v),
                                C.c_void_p(state.t.data_ptr()), rows_p,
                                _ptr(grads), C.c_void_p(d_n) if d_n else None, C.c_int64(int(n)),
                                lrv.ctypes.data_as(C.c_void_p), C.c_float(b1), C.c_float(b2), C.c_float(eps),
                                _stream_ptr(stream)))


def screen_grad_max(frame: Frame, max_per_node: torch.Tensor, stream=None) -> torch.Tensor:
    """max_per_node[row] = max(.., |dL/d(u, v)|) over the frame's selected nodes (after render_backward)."""
    check(lib().lodgs_frame_screen_grad_max(frame.handle, _ptr(max_per_node), _stream_ptr(stream)))
    return max_per_node


def frame_device_count(frame: Frame) -> int:
    """Device address of the frame's selected-node count (uint32)."""
    p = C.c_void_p()
    check(lib().lodgs_frame_device_count(frame.handle, C.byref(p)))
    return p.value


def l1_loss_grad(image: torch.Tensor, target: torch.Tensor, dL: torch.Tensor | None = None,
                 loss_sum: torch.Tensor | None = None, stream=None):
    """Mean L1 loss and its gradient in one pass; returns (dL, loss_sum) where
    loss_sum / image.numel() is the mean (a device scalar, not synchronised)."""
    n = image.numel()
    if dL is None:
        dL = torch.empty_like(image)
    if loss_sum is None:
        loss_sum = torch.empty(1, dtype=torch.float32, device=image.device)
    check(lib().lodgs_l1_loss_grad(_ptr(image), _ptr(target), C.c_int64(n), C.c_float(1.0 / max(n, 1)),
                                   _ptr(dL), _ptr(loss_sum), _stream_ptr(stream)))
    return dL, loss_sum


def inject_fault(site: int, after: int = 0) -> None:
    """Test hook: the call at `site` (_lib.FAULT_STREAM, _lib.FAULT_ALLOC) after
    `after` more successful ones fails once, on the host (after < 0 disarms)."""
    check(lib().lodgs_debug_inject_fault(int(site), int(after)))


def load_scene(path) -> Scene:
    """A scene from a checkpoint written by Scene.save; the layout is rebuilt
    and equals the saved scene's."""
    h = C.c_void_p()
    check(lib().lodgs_scene_load(str(path).encode(), C.byref(h)))
    return Scene(h)


def build_hierarchy(leaves, sh_degree: int, spt_volume: float, kappa: float) -> Scene:
    """Leaves (n x stride float32, numpy or torch) -> Scene.  See lodgs_build_hierarchy."""
    lib()
    if isinstance(leaves, torch.Tensor):
        t = leaves.contiguous().to(torch.float32)
        on_dev = int(t.is_cuda)
        ptr = C.c_void_p(t.data_ptr())
        keep = t
        n = t.shape[0]
    else:
        a = np.ascontiguousarray(leaves, dtype=np.float32)
        on_dev, ptr, keep, n = 0, C.c_void_p(a.ctypes.data), a, a.shape[0]
    p = _lib.BuildParams(float(spt_volume), float(kappa))
    h = C.c_void_p()
    check(lib().lodgs_build_hierarchy(ptr, C.c_int64(n), C.c_int(sh_degree), C.c_int(on_dev), C.byref(p), C.byref(h)))
    del keep
    return Scene(h)


def render_backward_blend(scene: Scene, frame: Frame, dL_dimage: torch.Tensor, stream=None,
                          image: torch.Tensor | None = None) -> None:
    """First half of render_backward: the blend backward (2D gradients stay in the frame)."""
    check(lib().lodgs_render_backward_blend(scene.handle, frame.handle, _ptr(_rendered_image(frame, image)),
                                            _ptr(dL_dimage.contiguous()), _stream_ptr(stream)))


def render_backward_blend_l1(scene: Scene, frame: Frame, target: torch.Tensor, loss_sum: torch.Tensor | None = None,
                             grad_scale: float | None = None, stream=None, image: torch.Tensor | None = None
                             ) -> torch.Tensor:
    """Blend backward of the mean-L1 loss against `target`, the loss folded in:
    dL/dC = grad_scale * sign(image - target) (default scale 1/numel) is formed
    in the kernel; returns loss_sum (device, sum |image - target|).  `target`
    is float32, or uint8 read as byte / 255 (lodgs_render_backward_blend_l1_u8)."""
    img = _rendered_image(frame, image)
    if loss_sum is None:
        loss_sum = torch.empty(1, dtype=torch.float32, device="cuda")
    if target.shape != img.shape or not target.is_cuda:
        raise ValueError(f"target must be a CUDA tensor of the image's shape {tuple(img.shape)}")
    fn = {torch.float32: lib().lodgs_render_backward_blend_l1,
          torch.uint8: lib().lodgs_render_backward_blend_l1_u8}.get(target.dtype)
    if fn is None:
        raise TypeError(f"target must be float32 or uint8, not {target.dtype}")
    scale = 1.0 / max(img.numel(), 1) if grad_scale is None else grad_scale
    target = target.contiguous()
    check(fn(scene.handle, frame.handle, _ptr(img), C.c_void_p(target.data_ptr()), C.c_float(scale), _ptr(loss_sum),
             _stream_ptr(stream)))
    return loss_sum


def render_backward_project(scene: Scene, frame: Frame, grad: torch.Tensor, rows: torch.Tensor | None = None,
                            dense: bool = False, stream=None) -> torch.Tensor:
    """Second half of render_backward: the projection backward into `grad`."""
    check(lib().lodgs_render_backward_project(scene.handle, frame.handle, _ptr(rows), _ptr(grad),
                                              C.c_int64(_grad_rows_capacity(scene, grad)), C.c_int(int(dense)),
                                              _stream_ptr(stream)))
    return grad


def set_view(frame: Frame, camera=None, bg=None, stream=None) -> None:
    """Set the frame's camera and/or background on the device (outside any
    captured graph); later select_lod(scene, None, frame) and render(...) use it."""
    cs = C.byref(camera_struct(camera)) if camera is not None else None
    bgv = (C.c_float * 3)(*[float(b) for b in bg]) if bg is not None else None
    check(lib().lodgs_frame_set_view(frame.handle, cs, bgv, _stream_ptr(stream)))
    if camera is not None:
        frame.camera = camera
    if bg is not None:
        frame.bg = tuple(float(b) for b in bg)


def select_lod(scene: Scene, camera, frame: Frame | None = None, stream=None) -> Frame:
    """LoD cut for one camera; the selection stays in the returned frame.
    camera=None uses the view set on the frame (graph-capturable form)."""
    fr = frame if frame is not None else Frame(scene)
    cs = C.byref(camera_struct(camera)) if camera is not None else None
    check(lib().lodgs_select_lod(scene.handle, cs, fr.handle, _stream_ptr(stream)))
    if camera is not None:
        fr.camera = camera
    return fr


def select_lod_batch(scene: Scene, cameras, frames: list, stream=None) -> list:
    """LoD cuts of up to LODGS_SELECT_BATCH_MAX views in one launch of each
    selection pass; frames[i] ends as select_lod(scene, cameras[i], frames[i])
    leaves it (its render may run on another stream)."""
    n = len(cameras)
    if n != len(frames):
        raise ValueError("one frame per camera")
    cs = (_lib.Camera * n)(*[camera_struct(c) for c in cameras])
    hs = (C.c_void_p * n)(*[f.handle.value for f in frames])
    check(lib().lodgs_select_lod_batch(scene.handle, C.cast(cs, C.c_void_p), C.cast(hs, C.c_void_p), C.c_int(n),
                                       _stream_ptr(stream)))
    for f, c in zip(frames, cameras):
        f.camera = c
    return frames


def render(scene: Scene, frame: Frame, rows: torch.Tensor | None = None, bg=(0.0, 0.0, 0.0),
           image: torch.Tensor | None = None, stream=None, check_capacity: bool = True) -> torch.Tensor:
    """Render the frame's selection into an H x W x 3 float32 CUDA tensor.

    With check_capacity the call synchronises the stream, and if a workspace
    buffer was too small (the buffers then grow) renders again."""
    cam = frame.camera
    if image is None:
        image = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    if bg is None:
        bgv = None
    else:
        bgv = (C.c_float * 3)(*[float(b) for b in bg])
        frame.bg = tuple(float(b) for b in bg)
    frame.image = image             # what render_backward reads by default
    for _ in range(4):
        check(lib().lodgs_render(scene.handle, frame.handle, _ptr(rows), bgv, _ptr(image), _stream_ptr(stream)))
        if not check_capacity:
            return image
        st = frame.stats()
        if st["status"] != _lib.LODGS_E_CAPACITY:
            check(st["status"])
            return image
    raise _lib.LodgsError(_lib.LODGS_E_CAPACITY, "workspace did not converge")


def _rendered_image(frame: Frame, image: torch.Tensor | None) -> torch.Tensor:
    img = image if image is not None else getattr(frame, "image", None)
    if img is None:
        raise _lib.LodgsError(_lib.LODGS_E_STATE, "render_backward: no image rendered on this frame")
    return img.contiguous()


def render_backward(scene: Scene, frame: Frame, dL_dimage: torch.Tensor, rows: torch.Tensor | None = None,
                    grad: torch.Tensor | None = None, dense: bool = False, n_selected: int | None = None,
                    stream=None, image: torch.Tensor | None = None) -> torch.Tensor:
    """Gradients of the frame's last render w.r.t. the records.  Sparse: one row per
    selected node (selection order); dense: n_nodes x stride with selected rows written.
    `image` is the frame's last rendered image (default: the tensor render wrote)."""
    if grad is None:
        if dense:
            grad = torch.zeros((scene.n_nodes, scene.stride), dtype=torch.float32, device="cuda")
        else:
            if n_selected is None:
                n_selected = frame.stats()["n_selected"]
            grad = torch.empty((max(n_selected, 1), scene.stride), dtype=torch.float32, device="cuda")
    bgv = (C.c_float * 3)(*frame.bg)
    dL = dL_dimage.contiguous()
    img = _rendered_image(frame, image)
    check(lib().lodgs_render_backward(scene.handle, frame.handle, _ptr(rows), bgv, _ptr(img), _ptr(dL), _ptr(grad),
                                      C.c_int64(_grad_rows_capacity(scene, grad)), C.c_int(int(dense)),
                                      _stream_ptr(stream)))
    return grad


def _grad_rows_capacity(scene: Scene, grad: torch.Tensor) -> int:
    """Whole gradient rows the tensor holds (the library checks the selection
    against it on the device)."""
    assert grad.is_cuda and grad.dtype == torch.float32 and grad.is_contiguous()
    return grad.numel() // scene.stride
