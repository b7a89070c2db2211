"""Sparse Adam over the cut set and the per-node screen-space gradient maximum,
through the C ABI, against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("deg,n_leaves", [(0, 700), (1, 700), (1, 6000), (3, 3000)])
def test_adam_matches_oracle_over_changing_row_sets(deg, n_leaves):
    """Rows of 4, 6 and 15 quarters (SH 0, 1, 3): with 6 and 15 a warp holds
    whole rows only, so the step count of a row is read by all its quarters
    before it is written."""
    from paper_2507_01110_b300 import api, build
    build.build()
    leaves = synth.leaves_uniform_cube(n_leaves, seed=51, half_extent=10.0, degree=deg)
    scene = api.build_hierarchy(leaves, deg, 0.5, 300.0)
    n, stride = scene.n_nodes, scene.stride
    used = 14 + 3 * ((deg + 1) ** 2 - 1)
    params = scene.rows().clone()
    p0 = params.cpu().numpy().astype(np.float64)
    state = api.AdamState(scene)
    po, mo, vo = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    to = np.zeros(n, np.uint32)
    rng = np.random.default_rng(52)
    lr = rng.uniform(1e-4, 1e-2, stride).astype(np.float32)
    touched = np.zeros(n, bool)
    for step in range(5):
        rows = np.sort(rng.choice(n, size=rng.integers(n // 20, n // 2), replace=False)).astype(np.int32)
        g = rng.standard_normal((len(rows), stride)).astype(np.float32)
        api.adam_step(scene, params, state, torch.from_numpy(rows).cuda(), torch.from_numpy(g).cuda(), lr,
                      eps=1e-8)
        # the ABI takes float32 hyper-parameters: give the oracle the same values
        oracle.adam_sparse(po, mo, vo, to, rows, g.astype(np.float64), lr.astype(np.float64),
                           b1=float(np.float32(0.9)), b2=float(np.float32(0.999)), eps=float(np.float32(1e-8)),
                           used=used)
        touched[rows] = True
    torch.cuda.synchronize()
    pg = params.cpu().numpy()
    assert np.array_equal(state.t.cpu().numpy().view(np.uint32), to)
    assert np.allclose(pg, po, rtol=1e-6, atol=1e-6)
    assert np.allclose(state.m.cpu().numpy(), mo, rtol=1e-5, atol=1e-7)
    assert np.allclose(state.v.cpu().numpy(), vo, rtol=1e-5, atol=1e-9)
    # untouched rows and the unused padding columns keep their bits
    assert np.array_equal(pg[~touched], p0[~touched].astype(np.float32))
    assert np.array_equal(pg[:, used:], p0[:, used:].astype(np.float32))
    assert np.abs(pg[touched, :used] - p0[touched, :used]).max() > 1e-4


def test_screen_gradient_max_over_two_views_matches_oracle():
    from paper_2507_01110_b300 import api, build
    build.build()
    leaves = synth.leaves_uniform_cube(6000, seed=53, half_extent=15.0, degree=0)
    cams = [synth.camera_look([1.0, 0.0, -45.0], [0.0, 0.02, 1.0], [1.0, 0.0, 0.0], 120, 88),
            synth.camera_look([40.0, 5.0, 0.0], [-1.0, 0.0, 0.1], [0.0, 0.0, 1.0], 96, 96, tau=1.5)]
    kappa = float(cams[0].fx)
    sc_o = oracle.build_scene(leaves, 0, 1.0, kappa)
    scene = api.build_hierarchy(leaves, 0, 1.0, kappa)
    gmax = torch.zeros(scene.n_nodes, device="cuda")
    views = []
    rng = np.random.default_rng(54)
    for cam in cams:
        fr = api.select_lod(scene, cam)
        img = api.render(scene, fr)
        w = rng.uniform(-1, 1, img.shape).astype(np.float32)
        api.render_backward(scene, fr, torch.from_numpy(w).cuda())
        api.screen_grad_max(fr, gmax)
        out = oracle.render(sc_o, cam)
        g = oracle.render_backward(sc_o, cam, out, w.astype(np.float64))["g2d"]
        views.append((out["sel"], g))
    torch.cuda.synchronize()
    # both sides index nodes by render row (the oracle's selection is in render rows)
    ref = oracle.screen_grad_max(scene.n_nodes, views)
    got = gmax.cpu().numpy().astype(np.float64)
    assert (ref > 0).sum() > 100
    big = ref > 1e-3 * ref.max()
    assert np.all(np.abs(got[big] - ref[big]) <= 1e-3 * ref[big] + 1e-6 * ref.max())
    assert np.all(got[ref == 0] == 0)
