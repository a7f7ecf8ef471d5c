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


def test_graph_is_recaptured_after_the_scene_or_a_buffer_changes():
    """A captured graph holds the scene's instance list and raw buffer addresses: after the
    instances change, or after another call grew (reallocated) a buffer, the next call with the
    same key must not replay the old graph -- its images equal the synchronous render of the
    scene as it is now."""
    sc = scenes.tiny_scene(3000, 4, spread=0.6, log_scale_mean=-3.0, sh_degree=2, n_instances=3)
    r = renderer_for(sc)
    try:
        fl = r.flags(use_mlp=0)
        cams = _cams(0)
        out = [torch.zeros((c.height, c.width, 3), device="cuda") for c in cams]

        def check():
            ref = _sync_images(r, cams, fl)
            r.render_batch(cams, r.flags(use_mlp=0), out=out, use_graph=True)   # replay or recapture
            torch.cuda.synchronize()
            for (a, _), b in zip(ref, out):
                assert torch.equal(a, b)

        r.render_batch(cams, r.flags(use_mlp=0), out=out, use_graph=True)   # render + capture
        check()
        r.set_instances(sc.instances[:2])                                    # fewer instances
        check()
        r.set_instances(sc.instances)
        check()
        big = scenes.look_at_camera((0.0, 0.0, 3.0), (0, 0, 0), 1600, 1200, 400.0)
        r.render(big, fl)                                                    # grows per-frame buffers
        check()
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
        assert len(table) == 3 * 4 * 2 * 3      # tiles x MLP CTAs per SM x split x radix digit width
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


# ----------------------------------------------------------------------------- views with own instance sets
def _pool_scene(n_instances=12, n=3000):
    """Three small assets (torus, sphere, box; SH degree 1) as n_instances rigid instances spread on a
    plane: the pool every view draws its own instance subset from."""
    assets = [scenes.torus_asset(n, seed=1, sh_degree=1), scenes.sphere_asset(n, 2, sh_degree=1),
              scenes.box_asset(n, 3, sh_degree=1)]
    rng = np.random.default_rng(31)
    insts = []
    for k in range(n_instances):
        q, rr = np.linalg.qr(rng.standard_normal((3, 3)))
        q = q * np.sign(np.diag(rr))
        if np.linalg.det(q) < 0:
            q[:, 0] *= -1
        t = np.array([rng.uniform(-3, 3), rng.uniform(-0.5, 0.5), rng.uniform(-3, 3)], np.float32)
        insts.append(scenes.Instance(k % 3, q.astype(np.float32), t, float(np.float32(rng.uniform(0.5, 1.2)))))
    return scenes.Scene(assets, insts)


def _view_sets(n_instances, n_views, seed=5):
    """Uneven instance subsets (2 .. all of the pool, shuffled order) and mixed camera sizes."""
    rng = np.random.default_rng(seed)
    sizes = [(256, 144), (320, 180), (97, 61), (200, 200), (128, 96), (61, 97)]
    sets, cams = [], []
    for v in range(n_views):
        k = int(rng.integers(2, n_instances + 1))
        sets.append(np.sort(rng.choice(n_instances, k, replace=False)).astype(np.int32))
        ang = rng.uniform(0, 2 * np.pi)
        eye = (8.0 * np.cos(ang), rng.uniform(1.0, 4.0), 8.0 * np.sin(ang))
        cams.append(scenes.look_at_camera(eye, (0, 0, 0), *sizes[v % len(sizes)], 55.0))
    return sets, cams


def _subset_render(r, sc, subset, cam, fl):
    r.set_instances([sc.instances[i] for i in subset])
    img, st = r.render(cam, fl)
    return img.clone(), st


@pytest.mark.parametrize("use_mlp", [0, 1])
def test_views_with_own_instance_sets_equal_their_single_view_renders(use_mlp):
    """nvgs_render_views: every view, with its own uneven instance subset and size, equals the
    synchronous render of that view over exactly those instances bit for bit (no dense-tile split),
    the batch's totals are the views' sums, and the BF16 MLP path culls in both."""
    from paper_2511_19202_b300 import nvgs as N
    sc = _pool_scene()
    ws = [scenes.mlp_weights(60 + k) for k in range(3)]
    r = renderer_for(sc, ws, precision=N.NVGS_PREC_BF16)
    try:
        sets, cams = _view_sets(len(sc.instances), 7)
        fl = dict(use_mlp=use_mlp, mlp_gate=0, bg=(0.05, 0.1, 0.2), blend_split_len=-1)
        imgs, tot = r.render_views(cams, [s.tolist() for s in sets], r.flags(**fl))
        imgs = [im.clone() for im in imgs]
        sums = dict(n_in_frustum=0, n_survivors=0, n_pairs=0)
        for v, (subset, cam) in enumerate(zip(sets, cams)):
            ref, st = _subset_render(r, sc, subset, cam, r.flags(**fl))
            assert torch.equal(imgs[v], ref), f"view {v}: max diff {float((imgs[v] - ref).abs().max()):.3e}"
            for k in sums:
                sums[k] += st[k]
        for k in sums:
            assert tot[k] == sums[k], (k, tot[k], sums[k])
        assert tot["n_pairs"] > 0
        if use_mlp:
            assert 0 < tot["n_survivors"] < tot["n_in_frustum"]
    finally:
        r.close()


def test_views_match_the_oracle():
    """Two views of one batch against the FP64 oracle over their own instance subsets: a small one
    and a ragged one (97 x 61, tiles cut at both edges), unculled, 1e-3 max-abs outside the band."""
    import oracle
    from gpu_common import compare_images, oracle_opts_for
    sc = _pool_scene()
    r = renderer_for(sc)
    try:
        sets, cams = _view_sets(len(sc.instances), 6, seed=9)
        fl = dict(use_mlp=0, bg=(0.05, 0.1, 0.2))
        imgs, tot = r.render_views(cams, [s.tolist() for s in sets], r.flags(**fl))
        for v in (2, 5):   # 97 x 61 and 61 x 97
            sub = scenes.Scene(sc.assets, [sc.instances[i] for i in sets[v]])
            ref = oracle.render(oracle.OracleScene(sub), cams[v], oracle_opts_for(fl))
            err, n_amb = compare_images(imgs[v].cpu().numpy().astype(np.float64), ref["image"], ref["ambiguous"])
            print(f"view {v} ({cams[v].width}x{cams[v].height}, {len(sets[v])} instances): max err {err:.2e}, "
                  f"{n_amb} ambiguous pixels")
    finally:
        r.close()


def test_views_graph_replay_with_new_cameras():
    """The batch captured into a CUDA graph replays with new cameras (same sizes, instance sets and
    images) and equals a plain call with those cameras; automatic dense-tile split on."""
    sc = _pool_scene()
    r = renderer_for(sc)
    try:
        sets, cams = _view_sets(len(sc.instances), 5, seed=3)
        sets2, cams2 = _view_sets(len(sc.instances), 5, seed=4)
        fl = r.flags(use_mlp=0)
        lists = [s.tolist() for s in sets]
        out = [torch.zeros((c.height, c.width, 3), device="cuda") for c in cams]
        r.render_views(cams, lists, fl, out=out, use_graph=True)          # render + capture
        cams_b = [scenes.look_at_camera(-np.asarray(c2.R).T @ np.asarray(c2.t), (0, 0, 0), c.width, c.height, 55.0)
                  for c, c2 in zip(cams, cams2)]
        r.render_views(cams_b, lists, fl, out=out, use_graph=True)        # replay
        torch.cuda.synchronize()
        replay = [o.clone() for o in out]
        plain, _ = r.render_views(cams_b, lists, fl)
        for a, b in zip(replay, plain):
            assert torch.equal(a, b)
    finally:
        r.close()


def test_views_reject_bad_sets():
    from paper_2511_19202_b300 import nvgs as N
    sc = _pool_scene(4)
    r = renderer_for(sc)
    try:
        cam = scenes.look_at_camera((0, 2, 8), (0, 0, 0), 64, 64, 55.0)
        with pytest.raises(N.NvgsError):
            r.render_views([cam], [[0, 7]], r.flags(use_mlp=0))            # instance out of range
        with pytest.raises(N.NvgsError):
            r.render_views([cam], [[0]], r.flags(use_mlp=0, keep_outputs=1))
        img, tot = r.render_views([cam, cam], [[], None], r.flags(use_mlp=0))   # an empty view is fine
        assert tot["n_instanced"] == 4 * 3000
    finally:
        r.close()
