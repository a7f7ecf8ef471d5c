"""Batched, sync-free rendering (nvgs_render_batch) and its CUDA-graph replay: every view must equal
the synchronous nvgs_render of the same camera bit for bit (same pairs in the same order, same
compositing), whatever the batch, the view sizes or the replay; overflowing the pair capacity is
reported.  The synchronous path itself is checked against the FP64 oracle in test_gpu_render."""
import numpy as np
import pytest

import scenes
from gpu_common import renderer_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _cams(k0=0):
    eyes = [(0.0, 0.0, 3.0), (0.6, 0.9, 2.8), (-1.2, 0.4, 2.5), (2.0, -0.5, 2.2), (0.3, 2.1, 2.0)]
    sizes = [(256, 256), (97, 61), (128, 200), (256, 128), (160, 90)]
    return [scenes.look_at_camera(eyes[(k0 + k) % 5], (0, 0, 0), *sizes[k], 50.0) for k in range(5)]


def _sync_images(r, cams, fl):
    out = []
    for c in cams:
        img, st = r.render(c, fl)
        out.append((img.clone(), st))
    return out


@pytest.mark.parametrize("use_mlp", [0, 1])
def test_batch_equals_single_view_renders(use_mlp):
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.config1_scene(20000)
    w = scenes.mlp_weights(7)
    r = renderer_for(sc, w, precision=N.NVGS_PREC_BF16)
    try:
        cams = _cams()
        fl = r.flags(use_mlp=use_mlp, mlp_gate=0, bg=(0.1, 0.2, 0.3))
        ref = _sync_images(r, cams, fl)
        imgs, stats = r.render_batch(cams, r.flags(use_mlp=use_mlp, mlp_gate=0, bg=(0.1, 0.2, 0.3)))
        for (a, sa), b, sb in zip(ref, imgs, stats):
            assert torch.equal(a, b)
            assert sb["n_in_frustum"] == sa["n_in_frustum"] and sb["n_survivors"] == sa["n_survivors"]
            assert sb["n_pairs"] == sa["n_pairs"]
        if use_mlp:
            assert any(s["n_survivors"] < s["n_in_frustum"] for s in stats)
    finally:
        r.close()


def test_graph_replays_with_new_cameras():
    sc = scenes.tiny_scene(3000, 4, spread=0.6, log_scale_mean=-3.0, sh_degree=2, n_instances=3)
    r = renderer_for(sc)
    try:
        fl = r.flags(use_mlp=0)
        first, second = _cams(0), _cams(1)
        # same sizes in both sets (the graph is keyed by view sizes): reuse the first set's sizes
        second = [scenes.look_at_camera(-np.asarray(c.R).T @ np.asarray(c.t) * 1.1, (0, 0, 0), f.width, f.height, 50.0)
                  for c, f in zip(second, first)]
        out = [torch.zeros((c.height, c.width, 3), device="cuda") for c in first]
        for cams in (first, second, first, second):
            ref = _sync_images(r, cams, fl)
            _, st = r.render_batch(cams, r.flags(use_mlp=0), out=out, use_graph=True)
            for (a, sa), b, s in zip(ref, out, st):
                assert torch.equal(a, b)
                assert s["n_pairs"] == sa["n_pairs"]
        # without stats the call does not wait; the images are there after a synchronise
        N_ref = _sync_images(r, second, fl)
        r.render_batch(second, r.flags(use_mlp=0), out=out, use_graph=True, want_stats=False)
        torch.cuda.synchronize()
        for (a, _), b in zip(N_ref, out):
            assert torch.equal(a, b)
    finally:
        r.close()


def test_pair_capacity_overflow_is_reported():
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.config1_scene(20000)
    r = renderer_for(sc)
    try:
        cams = _cams()[:2]
        with pytest.raises(N.NvgsError) as e:
            r.render_batch(cams, r.flags(use_mlp=0), max_pairs=1000)
        assert e.value.status == N.NVGS_ERR_CAPACITY
        # and a sufficient capacity renders again
        imgs, st = r.render_batch(cams, r.flags(use_mlp=0), max_pairs=200000)
        assert all(s["n_pairs"] <= 200000 for s in st)
    finally:
        r.close()


def test_batch_rejects_unsupported_flags():
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.tiny_scene(100, 1)
    r = renderer_for(sc)
    try:
        with pytest.raises(N.NvgsError):
            r.render_batch(_cams()[:1], r.flags(use_mlp=0, keep_outputs=1))
        with pytest.raises(N.NvgsError):
            r.render_batch(_cams()[:1], r.flags(use_mlp=0, profile=1))
    finally:
        r.close()


def test_autotuner_times_every_candidate_and_images_do_not_depend_on_the_choice():
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.config1_scene(20000)
    r = renderer_for(sc, scenes.mlp_weights(3), precision=N.NVGS_PREC_BF16)
    try:
        cams = _cams()[:3]
        out = [torch.zeros((c.height, c.width, 3), device="cuda") for c in cams]
        base = r.flags(use_mlp=1, mlp_gate=0)
        best, table = N.nvgs_autotune(r.ctx, cams, base, out)
        print(table)
        assert len(table) == 3 * 4 * 2          # tiles x MLP CTAs per SM x split
        assert {t["tile_size"] for t in table} == {8, 16, 32}
        fastest = min(table, key=lambda t: t["ms_per_view"])
        assert best.tile_size == fastest["tile_size"] and best.mlp_ctas_per_sm == fastest["mlp_ctas_per_sm"]
        assert best.use_mlp == 1 and best.mlp_gate == 0
        imgs = {}
        for ts in (8, 16, 32):
            im, _ = r.render_batch(cams, r.flags(use_mlp=1, mlp_gate=0, tile_size=ts))
            imgs[ts] = im
        for k in range(len(cams)):
            assert torch.equal(imgs[8][k], imgs[16][k]) and torch.equal(imgs[16][k], imgs[32][k])
    finally:
        r.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_automatic_split_equals_the_synchronous_render(use_graph):
    """The automatic dense-tile split length depends on the frame's pair count.  The sync-free
    batch knows only its pair capacity (here 3x the count), so it resolves the length on the
    device from the count: it splits the same tiles as the synchronous render and the images are
    equal bit for bit."""
    sc = scenes.config1_scene(20000)
    # the torus covers a few of the 64 tiles of a 128 x 128 view: those tiles hold many times
    # the mean tile's pairs and more than the 4096-pair minimum
    cam = scenes.look_at_camera((0.0, 0.0, 12.0), (0, 0, 0), 128, 128, 50.0)
    r = renderer_for(sc)
    try:
        fl = lambda split: r.flags(use_mlp=0, blend_split_len=split)
        auto, st = r.render(cam, fl(0))
        auto = auto.clone()
        never, _ = r.render(cam, fl(-1))
        assert not torch.equal(auto, never), "no tile was split: the case does not exercise the path"
        out = [torch.empty_like(auto)]
        for _ in range(2):   # the second call replays the captured graph
            r.render_batch([cam], fl(0), out=out, max_pairs=3 * st["n_pairs"], use_graph=use_graph)
            torch.cuda.synchronize()
            assert torch.equal(out[0], auto)
    finally:
        r.close()
