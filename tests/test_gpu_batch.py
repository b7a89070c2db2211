"""Batch gradient over several views: the union of the cuts, summed rows."""
import numpy as np
import pytest
import torch

from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("degree", [1, 3])
def test_accumulate_grads_equals_scatter_add(degree):
    """The union of the cuts, and each node's rows summed in view order: bit
    for bit the float32 sum in view order, with the rows 16-byte aligned
    (float4 lane groups), 8-byte aligned (float2) and 4-byte aligned (floats),
    and with a view that selects nothing."""
    from paper_2507_01110_b300 import api, build
    build.build()
    leaves = synth.leaves_uniform_cube(20000, seed=61, half_extent=20.0, degree=degree)
    cams = [synth.camera_look([0.0, 0.0, -70.0], [0, 0, 1], [1, 0, 0], 96, 80),
            synth.camera_look([10.0, 2.0, -60.0], [-0.1, 0.0, 1.0], [1, 0, 0], 96, 80, tau=2.0),
            synth.camera_look([0.0, 0.0, -300.0], [0, 0, -1], [1, 0, 0], 64, 64),          # looks away
            synth.camera_look([60.0, 0.0, 0.0], [-1, 0, 0], [0, 0, 1], 120, 64)]
    scene = api.build_hierarchy(leaves, degree, 2.0, float(cams[0].fx))
    frames, grads, sels = [], [], []
    rng = np.random.default_rng(3)
    for cam in cams:
        fr = api.select_lod(scene, cam)
        img = api.render(scene, fr)
        w = torch.from_numpy(rng.uniform(-1, 1, img.shape).astype(np.float32)).cuda()
        g = api.render_backward(scene, fr, w)
        sel = fr.selection()
        frames.append(fr)
        grads.append(g[: sel.numel()].contiguous())
        sels.append(sel.cpu().numpy())
    assert min(len(x) for x in sels) == 0 and max(len(x) for x in sels) > 100
    union = np.unique(np.concatenate(sels))
    ref = np.zeros((scene.n_nodes, scene.stride), np.float32)     # float32, in view order
    for sl, g in zip(sels, grads):
        ref[sl] += g.cpu().numpy()
    for shift in (0, 2, 1):                       # floats past a 16-byte boundary
        gs = grads
        if shift:
            gs = []
            for g in grads:
                buf = torch.empty(g.numel() + shift, device="cuda")
                buf[shift:] = g.reshape(-1)
                gs.append(buf[shift:].view(g.shape))
            assert all(g.data_ptr() % 16 == 4 * shift for g in gs if g.numel())
        rows, summed = api.accumulate_grads(scene, frames, gs)
        rows, summed = rows.cpu().numpy(), summed.cpu().numpy()
        assert np.array_equal(rows, union)
        assert np.array_equal(summed, ref[union]), shift


def test_fused_l1_loss_grad_matches_torch():
    from paper_2507_01110_b300 import api, build
    build.build()
    g = torch.Generator(device="cuda").manual_seed(7)
    for shape in ((1080, 1920, 3), (37, 41, 3)):
        img = torch.rand(shape, device="cuda", generator=g)
        tgt = torch.rand(shape, device="cuda", generator=g)
        tgt.view(-1)[:5] = img.view(-1)[:5]                      # sign(0) = 0
        dL, s = api.l1_loss_grad(img, tgt)
        n = img.numel()
        assert torch.equal(dL, torch.sign(img - tgt) * (1.0 / n))
        assert abs(s.item() / n - (img - tgt).abs().mean().item()) < 1e-6
