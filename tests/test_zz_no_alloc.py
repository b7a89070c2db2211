"""lodgs_select_lod_noalloc: the LoD cut for callers that cannot allocate device
memory (an application that hands all device memory to its own pool, or a loop
that cannot take cudaMalloc's device synchronisation).  Its scratch is a static
device array, so it must give exactly the selection of the allocating entry
point, on consecutive calls that reuse that array.  Kept in its own file,
collected last."""
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


def _noalloc(L, scene, cam, out, count, stream=None):
    cs = api_camera(cam)
    return L.lodgs_select_lod_noalloc(scene.handle, C.byref(cs), C.c_void_p(out.data_ptr()),
                                      C.c_int64(scene.n_nodes), C.c_void_p(count.data_ptr()),
                                      C.c_void_p(stream.cuda_stream) if stream is not None else None)


def api_camera(cam):
    from paper_2507_01110_b300 import api
    return api.camera_struct(cam)


def test_select_noalloc_matches_on_a_scene_with_a_multi_block_spt_scan():
    """A scene with more than 16384 SPTs: the per-SPT prefix scan then takes its
    multi-block path, whose block sums live in the static scratch too."""
    from paper_2507_01110_b300 import _lib, api, build
    build.build()
    leaves = synth.leaves_ground_and_boxes(60_000, seed=44, degree=0, extent=300.0, n_boxes=40)
    cam0 = synth.camera_look([0.0, -80.0, 40.0], [0.0, 1.0, -0.5], [1.0, 0.0, 0.0], 320, 180, tau=1.0)
    scene = api.build_hierarchy(leaves, 0, 0.05, float(cam0.fx))
    assert scene.n_spt > 16384
    cams = [cam0, synth.camera_look([30.0, -20.0, 10.0], [-0.2, 1.0, -0.3], [1.0, 0.2, 0.0], 256, 200, tau=0.5)]
    frame = api.Frame(scene)
    out = torch.empty(scene.n_nodes, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = _lib.lib()
    for cam in cams:
        api.select_lod(scene, cam, frame)
        ref = frame.selection().cpu().numpy()
        out.fill_(-1)
        assert _noalloc(L, scene, cam, out, count, torch.cuda.current_stream()) == _lib.LODGS_OK
        torch.cuda.synchronize()
        n = int(count.item())
        assert n == len(ref) > 0 and frame.stats()["n_spt_cut"] > 3000
        assert np.array_equal(out[:n].cpu().numpy().view(np.uint32).astype(np.int64), ref)


def test_select_noalloc_refuses_the_cameras_select_lod_refuses():
    import dataclasses
    from paper_2507_01110_b300 import _lib, api, build
    build.build()
    leaves = synth.leaves_uniform_cube(1000, seed=3, half_extent=5.0)
    scene = api.build_hierarchy(leaves, 0, 2.0, 150.0)
    cam = synth.camera_look([0.0, 0.0, -20.0], [0, 0, 1], [1, 0, 0], 64, 64)
    out = torch.empty(scene.n_nodes, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = _lib.lib()
    for bad in (dataclasses.replace(cam, spt_scale=-1.0), dataclasses.replace(cam, cx=float("nan")),
                dataclasses.replace(cam, width=65535 * 16 + 1)):
        with pytest.raises(_lib.LodgsError):
            api.select_lod(scene, bad)
        assert _noalloc(L, scene, bad, out, count) == _lib.LODGS_E_INVALID
        assert b"camera" in L.lodgs_last_error()


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
