"""A CUDA graph captured from select(None) + render + loss + backward on one
camera, replayed after lodgs_frame_set_view for another camera, gives the same
image as rendering that camera eagerly."""
import pytest
import torch

from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


def test_captured_step_replays_for_a_new_camera():
    from paper_2507_01110_b300 import api, build
    build.build()
    leaves = synth.leaves_uniform_cube(30000, seed=71, half_extent=20.0, degree=1)
    camA = synth.camera_look([0.0, 0.0, -70.0], [0, 0, 1], [1, 0, 0], 200, 120)
    camB = synth.camera_look([8.0, -3.0, -55.0], [-0.1, 0.05, 1.0], [1, 0, 0], 200, 120, tau=1.5)
    scene = api.build_hierarchy(leaves, 1, 2.0, float(camA.fx))
    # eager references
    ref = {}
    for name, cam in (("A", camA), ("B", camB)):
        fr = api.select_lod(scene, cam)
        ref[name] = api.render(scene, fr, bg=(0.1, 0.2, 0.3)).clone()
    fr = api.Frame(scene)
    img = torch.empty((120, 200, 3), device="cuda")
    tgt = torch.rand((120, 200, 3), device="cuda")
    dL = torch.empty_like(img)
    loss = torch.empty(1, device="cuda")
    # grow the workspace on both cameras before capturing (no allocation during capture)
    for cam in (camA, camB):
        api.select_lod(scene, cam, fr)
        api.render(scene, fr, image=img, bg=(0.1, 0.2, 0.3))
    n_max = fr.stats()["n_selected"]
    api.select_lod(scene, camA, fr)
    api.render(scene, fr, image=img, bg=(0.1, 0.2, 0.3))
    n_max = max(n_max, fr.stats()["n_selected"])
    grad = torch.empty((n_max, scene.stride), device="cuda")
    api.set_view(fr, camA, bg=(0.1, 0.2, 0.3))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            api.select_lod(scene, None, fr)
            api.render(scene, fr, image=img, bg=None, check_capacity=False)
            api.l1_loss_grad(img, tgt, dL=dL, loss_sum=loss)
            api.render_backward(scene, fr, dL, grad=grad)
    torch.cuda.synchronize()
    for name, cam in (("B", camB), ("A", camA), ("B", camB)):
        api.set_view(fr, cam)
        g.replay()
        torch.cuda.synchronize()
        assert fr.stats()["status"] == 0
        assert torch.equal(img, ref[name]), name


def test_split_backward_matches_the_combined_call():
    from paper_2507_01110_b300 import api, build
    build.build()
    leaves = synth.leaves_uniform_cube(20000, seed=72, half_extent=15.0, degree=2)
    cam = synth.camera_look([0.0, 0.0, -50.0], [0, 0, 1], [1, 0, 0], 160, 96)
    scene = api.build_hierarchy(leaves, 2, 2.0, float(cam.fx))
    fr = api.select_lod(scene, cam)
    img = api.render(scene, fr)
    dL = torch.rand_like(img) - 0.5
    n = fr.stats()["n_selected"]
    g1 = torch.zeros((n, scene.stride), device="cuda")
    api.render_backward(scene, fr, dL, grad=g1)
    g2 = torch.zeros_like(g1)
    api.render_backward_blend(scene, fr, dL)
    api.render_backward_project(scene, fr, g2)
    torch.cuda.synchronize()
    # per-Gaussian 2D gradients are summed across tiles with float atomics, so
    # two backward passes agree up to summation order
    scale = g1.abs().amax(dim=0, keepdim=True).clamp_min(1e-12)
    assert ((g1 - g2).abs() / scale).max().item() < 1e-4
    # the projection half refuses to run before a blend backward on a new render
    api.render(scene, fr)
    with pytest.raises(Exception):
        api.render_backward_project(scene, fr, g2)


def test_fused_l1_backward_matches_loss_then_backward():
    """lodgs_render_backward_blend_l1 (the mean-L1 gradient formed inside the
    blend backward) against lodgs_l1_loss_grad followed by the plain blend
    backward: the same loss sum and the same gradient rows, up to the order of
    float atomic sums."""
    from paper_2507_01110_b300 import api, build
    build.build()
    cfg = synth.config2_scene(n=200_000)
    scene = api.build_hierarchy(cfg["leaves"], 3, cfg["spt_volume"], cfg["kappa"])
    cam = synth.camera_look(cfg["cameras"][12].pos, cfg["cameras"][12].R[2], cfg["cameras"][12].R[0], 333, 190)
    gen = torch.Generator(device="cuda").manual_seed(8)
    target = torch.rand((cam.height, cam.width, 3), device="cuda", generator=gen)
    fr = api.select_lod(scene, cam)
    img = api.render(scene, fr)
    n = fr.stats()["n_selected"]
    dL, loss_a = api.l1_loss_grad(img, target)
    api.render_backward_blend(scene, fr, dL)
    g_a = torch.empty((n, scene.stride), device="cuda")
    api.render_backward_project(scene, fr, g_a)
    loss_b = api.render_backward_blend_l1(scene, fr, target)
    g_b = torch.empty((n, scene.stride), device="cuda")
    api.render_backward_project(scene, fr, g_b)
    torch.cuda.synchronize()
    assert abs(loss_a.item() - loss_b.item()) <= 1e-5 * abs(loss_a.item())
    scale = g_a.abs().amax(dim=0) + 1e-30
    assert torch.all((g_a - g_b).abs() <= 1e-4 * scale)
    assert g_a.abs().max() > 0


def test_fused_l1_backward_with_an_8bit_target():
    """An 8-bit target (byte / 255 in the kernel) gives the loss and gradients
    of the float32 target holding the same quotients, up to the order of float
    atomic sums; wrong dtypes and shapes are refused before any launch."""
    from paper_2507_01110_b300 import api, build
    build.build()
    cfg = synth.config2_scene(n=200_000)
    scene = api.build_hierarchy(cfg["leaves"], 3, cfg["spt_volume"], cfg["kappa"])
    c = cfg["cameras"][9]
    cam = synth.camera_look(c.pos, c.R[2], c.R[0], 301, 177)
    gen = torch.Generator().manual_seed(21)
    t8 = torch.randint(0, 256, (cam.height, cam.width, 3), generator=gen, dtype=torch.uint8)
    t32 = t8.float() / 255.0                      # correctly rounded on the CPU
    fr = api.select_lod(scene, cam)
    api.render(scene, fr)
    n = fr.stats()["n_selected"]
    out = []
    for t in (t32.cuda(), t8.cuda()):
        loss = api.render_backward_blend_l1(scene, fr, t)
        g = torch.empty((n, scene.stride), device="cuda")
        api.render_backward_project(scene, fr, g)
        out.append((loss.item(), g))
    (la, ga), (lb, gb) = out
    assert la > 0 and abs(la - lb) <= 1e-5 * la
    scale = ga.abs().amax(dim=0) + 1e-30
    assert torch.all((ga - gb).abs() <= 1e-4 * scale) and ga.abs().max() > 0
    with pytest.raises(TypeError):
        api.render_backward_blend_l1(scene, fr, t8.cuda().to(torch.int32))
    with pytest.raises(ValueError):
        api.render_backward_blend_l1(scene, fr, t8.cuda()[:-1])


def test_work_counters_follow_profiling():
    """The work counters are tallied by profiling renders only: the backward
    visits exactly the forward's blended contributions; without profiling
    they read 0."""
    from paper_2507_01110_b300 import api, build
    build.build()
    cfg = synth.config2_scene(n=200_000)
    scene = api.build_hierarchy(cfg["leaves"], 3, cfg["spt_volume"], cfg["kappa"])
    c = cfg["cameras"][10]
    cam = synth.camera_look(c.pos, c.R[2], c.R[0], 320, 200)
    fr = api.Frame(scene)
    fr.set_profiling(True)
    api.select_lod(scene, cam, fr)
    img = api.render(scene, fr)
    w = fr.work()
    assert w["fwd_eval"] >= w["fwd_blend"] > 0 and w["bwd_eval"] == w["bwd_contrib"] == 0
    api.render_backward(scene, fr, torch.full_like(img, 1e-3))
    w = fr.work()
    assert w["bwd_contrib"] == w["fwd_blend"] and w["bwd_eval"] >= w["bwd_contrib"]
    fr.set_profiling(False)
    api.select_lod(scene, cam, fr)
    img = api.render(scene, fr)
    api.render_backward(scene, fr, torch.full_like(img, 1e-3))
    assert all(v == 0 for v in fr.work().values())
