"""lodgs_select_lod_noalloc: the LoD cut for callers that cannot allocate device
memory (for example code running under CUDA graph capture or inside its own
memory pool).  Its scratch is a static device array, so it must give exactly
the selection of the allocating entry point, on consecutive calls that reuse
that array.  Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


def test_select_noalloc_matches_select_lod_on_consecutive_calls():
    from paper_2507_01110_b300 import _lib, api, build
    build.build()
    cfg = synth.config1_scene()
    scene = api.build_hierarchy(cfg["leaves"], 0, cfg["spt_volume"], cfg["kappa"])
    cams = [cfg["cameras"][0],
            synth.camera_look([80.0, -60.0, 40.0], [-1.0, 0.7, -0.3], [0.0, 0.0, 1.0], 200, 120, tau=2.0),
            synth.camera_look([10.0, 5.0, -70.0], [0.0, 0.05, 1.0], [1.0, 0.0, 0.0], 333, 190, tau=1.0)]
    frame = api.Frame(scene)
    out = torch.empty(scene.n_nodes, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = _lib.lib()
    stream = torch.cuda.current_stream()
    for cam in cams:                                  # consecutive calls share the static scratch
        api.select_lod(scene, cam, frame)
        ref = frame.selection().cpu().numpy()
        out.fill_(-1)
        cs = api.camera_struct(cam)
        rc = L.lodgs_select_lod_noalloc(scene.handle, C.byref(cs), C.c_void_p(out.data_ptr()),
                                        C.c_int64(scene.n_nodes), C.c_void_p(count.data_ptr()),
                                        C.c_void_p(stream.cuda_stream))
        assert rc == _lib.LODGS_OK, L.lodgs_last_error()
        torch.cuda.synchronize()
        n = int(count.item())
        assert n == len(ref) > 0
        got = out[:n].cpu().numpy().view(np.uint32).astype(np.int64)
        assert np.array_equal(got, ref)


def test_select_noalloc_rejects_small_capacity():
    from paper_2507_01110_b300 import _lib, api, build
    build.build()
    leaves = synth.leaves_uniform_cube(1000, seed=3, half_extent=5.0)
    scene = api.build_hierarchy(leaves, 0, 2.0, 150.0)
    cam = synth.camera_look([0.0, 0.0, -20.0], [0, 0, 1], [1, 0, 0], 64, 64)
    out = torch.empty(scene.n_nodes, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    cs = api.camera_struct(cam)
    L = _lib.lib()
    rc = L.lodgs_select_lod_noalloc(scene.handle, C.byref(cs), C.c_void_p(out.data_ptr()),
                                    C.c_int64(scene.n_nodes - 1), C.c_void_p(count.data_ptr()), None)
    assert rc == _lib.LODGS_E_INVALID and b"capacity" in L.lodgs_last_error()
