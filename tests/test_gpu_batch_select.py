"""lodgs_select_lod_batch: the LoD cuts of up to eight views in one launch of
each selection pass give exactly what one lodgs_select_lod per view gives
(cut, counters and the image rendered from it, bit for bit), including views
whose SPT scans take the multi-block path; bad batches are refused with
nothing enqueued."""
import numpy as np
import pytest
import torch

from paper_2507_01110_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2507_01110_b300 import build
    build.build()
    from paper_2507_01110_b300 import api as a
    return a


def _cams_c1():
    c = synth.config1_scene()["cameras"][0]
    return [
        c,
        synth.camera_look([80.0, -60.0, 40.0], [-1.0, 0.7, -0.3], [0.0, 0.0, 1.0], 200, 120, tau=2.0),
        synth.camera_look([0.0, 0.0, 0.0], [0.3, 0.2, 1.0], [1.0, 0.0, 0.0], 161, 97, tau=0.5),
        synth.camera_look([0.0, 0.0, -300.0], [0.0, 0.0, -1.0], [1.0, 0.0, 0.0], 64, 64),   # looks away
        synth.camera_look([10.0, 5.0, -70.0], [0.0, 0.05, 1.0], [1.0, 0.0, 0.0], 333, 190, tau=1.0),
    ]


def _compare(api, scene, cams, stream=None):
    frames = [api.Frame(scene) for _ in cams]
    api.select_lod_batch(scene, cams, frames, stream=stream)
    for cam, fr in zip(cams, frames):
        ref = api.select_lod(scene, cam, api.Frame(scene))
        assert np.array_equal(fr.selection().cpu().numpy(), ref.selection().cpu().numpy())
        a, b = fr.stats(), ref.stats()
        for k in ("n_selected", "n_upper_selected", "n_spt_cut", "n_spt_scanned"):
            assert a[k] == b[k], k
        img = api.render(scene, fr, bg=(0.1, 0.2, 0.3))
        img_ref = api.render(scene, ref, bg=(0.1, 0.2, 0.3))
        assert torch.equal(img, img_ref)
    return frames


def test_batch_selection_equals_per_view_selection_config1(api):
    cfg = synth.config1_scene()
    scene = api.build_hierarchy(cfg["leaves"], 0, cfg["spt_volume"], cfg["kappa"])
    cams = _cams_c1()
    for k in (1, 2, 5):
        _compare(api, scene, cams[:k])
    _compare(api, scene, (cams + cams[::-1])[:8])                    # eight, the largest batch
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        _compare(api, scene, cams[:3], stream=side)                  # on another stream, rendered on the default


def test_batch_selection_equals_per_view_selection_on_1080p_views(api):
    """Four 1080p views of the 2M-leaf path in one batch."""
    cfg = synth.config2_scene()
    scene = api.build_hierarchy(cfg["leaves"], 3, cfg["spt_volume"], cfg["kappa"])
    _compare(api, scene, [cfg["cameras"][v] for v in (0, 9, 20, 31)])


def test_batch_selection_with_multi_block_spt_scans(api):
    """A scene of more than 16384 SPTs: each view's SPT prefix scan takes the
    multi-block path, with its own block sums, inside the batch."""
    leaves = synth.leaves_ground_and_boxes(60_000, seed=44, degree=0, extent=300.0, n_boxes=40)
    cams = [synth.camera_look([0.0, -80.0, 40.0], [0.0, 1.0, -0.5], [1.0, 0.0, 0.0], 320, 180, tau=1.0),
            synth.camera_look([30.0, -20.0, 10.0], [-0.2, 1.0, -0.3], [1.0, 0.2, 0.0], 256, 200, tau=0.5),
            synth.camera_look([-60.0, 40.0, 25.0], [0.5, -0.8, -0.4], [0.8, 0.5, 0.0], 300, 200, tau=2.0)]
    scene = api.build_hierarchy(leaves, 0, 0.05, float(cams[0].fx))
    assert scene.n_spt > 16384
    _compare(api, scene, cams)


def test_bad_batches_are_refused(api):
    import dataclasses
    from paper_2507_01110_b300 import _lib
    cfg = synth.config1_scene()
    scene = api.build_hierarchy(cfg["leaves"], 0, cfg["spt_volume"], cfg["kappa"])
    other = api.build_hierarchy(cfg["leaves"][:1000], 0, cfg["spt_volume"], cfg["kappa"])
    cams = _cams_c1()
    fr = [api.Frame(scene) for _ in range(9)]
    with pytest.raises(_lib.LodgsError):
        api.select_lod_batch(scene, (cams * 2)[:9], fr)                 # nine views: one too many
    with pytest.raises(_lib.LodgsError):
        api.select_lod_batch(scene, cams[:2], [fr[0], fr[0]])
    with pytest.raises(_lib.LodgsError):
        api.select_lod_batch(scene, cams[:2], [fr[0], api.Frame(other)])
    with pytest.raises(_lib.LodgsError):
        api.select_lod_batch(scene, [cams[0], dataclasses.replace(cams[1], spt_scale=-1.0)], fr[:2])
    with pytest.raises(_lib.LodgsError):
        api.select_lod_batch(scene, [], [])
