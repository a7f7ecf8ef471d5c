"""GPU parity of the CUDA render pass (through the C ABI) against the FP64 oracle on the same seeded
inputs: images within 1e-3 max-abs outside the ambiguity band, culled sets / survivor order /
tile lists bit-exact from fixed logits, MLP logits and decisions, the radix sort, and edge cases.
"""
import math

import numpy as np
import pytest

import oracle
import scenes
from gpu_common import (check_exact_tile_lists, check_pruned_tile_lists, compare_images, gpu_image,
                        oracle_opts_for, renderer_for)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def cfg1_setup():
    sc, cam = scenes.config1_scene(), scenes.config1_camera()
    r = renderer_for(sc)
    yield sc, cam, r, oracle.OracleScene(sc)
    r.close()


def _random_weights(seed=42, bias_std=0.3):
    w = scenes.mlp_weights(seed)
    rng = np.random.default_rng(seed + 1)
    for k in range(1, 5):
        w[f"b{k}"] = rng.normal(0, bias_std, w[f"b{k}"].shape).astype(np.float32)
    return w


# ----------------------------------------------------------------------------- unculled path
@pytest.mark.parametrize("tile", [16])
def test_cfg1_unculled_image_matches_oracle(cfg1_setup, tile):
    sc, cam, r, osc = cfg1_setup
    img, st = gpu_image(r, cam, use_mlp=0, tile_size=tile)
    o = oracle_opts_for(dict(tile_size=tile))
    ref = oracle.render(osc, cam, o)
    err, n_amb = compare_images(img, ref["image"], ref["ambiguous"])
    assert st["n_survivors"] == st["n_in_frustum"] > 0
    print(f"max err {err:.2e}, ambiguous px {n_amb}")


def test_tile_size_does_not_change_the_image(cfg1_setup):
    sc, cam, r, osc = cfg1_setup
    imgs = [gpu_image(r, cam, use_mlp=0, tile_size=t)[0] for t in (8, 16, 32)]
    np.testing.assert_array_equal(imgs[0], imgs[1])
    np.testing.assert_array_equal(imgs[1], imgs[2])


def test_tile_id_width_does_not_change_the_image():
    """More than 65536 tiles (2080 x 2080 at 8 px: 67,600) sort 32-bit tile ids, fewer (16 px:
    16,900) 16-bit ones; the tile size never changes the image, so both must agree bit for bit, and
    the 8 px frame's tile lists must be sorted and cover every pair."""
    sc = scenes.config1_scene()
    cam = scenes.config1_camera(2080, 2080)
    r = renderer_for(sc)
    try:
        a, sa = gpu_image(r, cam, use_mlp=0, tile_size=8, keep_outputs=1)
        lf = r.last_frame()
        keys = lf["pair_keys"].cpu().numpy().astype(np.int64)
        ranges = lf["tile_ranges"].cpu().numpy().astype(np.int64)
        assert lf["tiles_x"] * lf["tiles_y"] == 260 * 260 > 65536
        assert keys.size == sa["n_pairs"] > 0 and np.all(np.diff(keys) >= 0) and keys[-1] < 260 * 260
        np.testing.assert_array_equal(np.diff(ranges, axis=1)[:, 0], np.bincount(keys, minlength=260 * 260))
        b, sb = gpu_image(r, cam, use_mlp=0, tile_size=16)
        np.testing.assert_array_equal(a, b)
        print(f"8 px: {sa['n_pairs']} pairs over {260 * 260} tiles; 16 px: {sb['n_pairs']} pairs")
    finally:
        r.close()


def test_background_and_host_output(cfg1_setup):
    sc, cam, r, osc = cfg1_setup
    bg = (0.2, 0.5, 0.9)
    dev, _ = gpu_image(r, cam, use_mlp=0, bg=bg)
    host = np.zeros((cam.height, cam.width, 3), np.float32)
    r.render_host(cam, r.flags(use_mlp=0, bg=bg), host)
    np.testing.assert_array_equal(dev, host.astype(np.float64))
    # a page-locked host image (what the end-to-end timing uses) gives the same image
    pinned = torch.full((cam.height, cam.width, 3), -1.0, dtype=torch.float32, pin_memory=True)
    r.render_host(cam, r.flags(use_mlp=0, bg=bg), pinned)
    np.testing.assert_array_equal(dev, pinned.numpy().astype(np.float64))
    ref = oracle.render(osc, cam, oracle_opts_for(dict(bg=bg)))
    compare_images(dev, ref["image"], ref["ambiguous"])


@pytest.mark.parametrize("size,tile,split", [((1000, 562), 16, 0), ((333, 301), 8, 0), ((640, 480), 16, 600),
                                             ((640, 480), 32, -1)])
def test_host_output_equals_device_output(cfg1_setup, size, tile, split):
    """A host image (page-locked or pageable) equals the device image bit for bit, over ragged
    image sizes, tile sizes and dense-tile splitting."""
    sc, _, r, _ = cfg1_setup
    cam = scenes.config1_camera(*size)
    flags = dict(use_mlp=0, tile_size=tile, blend_split_len=split, bg=(0.1, 0.2, 0.3))
    dev, st = gpu_image(r, cam, **flags)
    for pinned in (True, False):
        host = torch.full((cam.height, cam.width, 3), -1.0, dtype=torch.float32, pin_memory=pinned)
        r.render_host(cam, r.flags(**flags), host)
        np.testing.assert_array_equal(dev, host.numpy().astype(np.float64))


def test_profile_levels(cfg1_setup):
    """profile = 1 times stages without counting; profile = 2 also counts the compositing's
    (pixel, fragment) evaluations -- at least one per covered pixel -- and the image is the same."""
    sc, cam, r, osc = cfg1_setup
    a, s0 = r.render(cam, r.flags(use_mlp=0, profile=0))
    a = a.clone()
    b, s1 = r.render(cam, r.flags(use_mlp=0, profile=1))
    b = b.clone()
    c, s2 = r.render(cam, r.flags(use_mlp=0, profile=2))
    assert torch.equal(a, b) and torch.equal(a, c)
    assert s1["blend_evaluations"] == 0 and sum(s1["stage_ms"].values()) > 0
    covered = int((c.sum(-1) > 0).sum())
    assert s2["blend_evaluations"] >= covered > 0
    assert s2["blend_evaluations"] <= s2["n_pairs"] * r.flags().tile_size ** 2
    # at least one composited fragment per covered pixel, at most one per evaluation
    assert covered <= s2["blend_composited"] <= s2["blend_evaluations"]
    print(f"evaluations {s2['blend_evaluations']}, composited {s2['blend_composited']}")


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_isolated_needles_lose_no_fragment(tile):
    """Sparse splats of every orientation with axis ratios up to 1:80 and opacities from 0.005 to
    0.99, SH colour near 1: most pixels see a few splats at T near 1, so a fragment that the paired
    compositing dropped, doubled or took out of order (odd list lengths, the padding fragment, a
    pair's second fragment after the first one stopped) would move a pixel by at least alpha_min x
    colour (> 3e-3), three times the tolerance."""
    from helpers import axis_camera, one_asset
    rng = np.random.default_rng(11)
    n, W, H, fx = 1500, 256, 192, 200.0
    z = rng.uniform(2.0, 6.0, n)
    u, v = rng.uniform(-20, W + 20, n), rng.uniform(-20, H + 20, n)
    means = np.stack([(u - W / 2) * z / fx, (v - H / 2) * z / fx, z], 1)
    s_major = rng.uniform(-4.0, -1.5, n)
    ratio = np.exp(rng.uniform(0.0, math.log(80.0), n))
    log_scales = np.stack([s_major, s_major - np.log(ratio), s_major - np.log(ratio) - 0.5], 1)
    quats = rng.normal(size=(n, 4))
    op = rng.uniform(0.005, 0.99, n)
    a = one_asset(means, log_scales, quats / np.linalg.norm(quats, axis=1, keepdims=True),
                  np.log(op / (1 - op)), np.full((n, 1, 3), 1.75))
    sc = scenes.Scene([a], [scenes.Instance(0, np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 1.0)])
    cam = axis_camera(W, H, fx=fx)
    r = renderer_for(sc)
    try:
        img, st = gpu_image(r, cam, use_mlp=0, tile_size=tile, profile=2)
        ref = oracle.render(oracle.OracleScene(sc), cam, oracle_opts_for(dict(tile_size=tile)))
        err, n_amb = compare_images(img, ref["image"], ref["ambiguous"])
        covered = int((img.sum(-1) > 0).sum())
        assert covered > 0.3 * W * H
        print(f"needles tile {tile}: max err {err:.2e}, {n_amb} ambiguous px; evaluations "
              f"{st['blend_evaluations']}, composited {st['blend_composited']}")
    finally:
        r.close()


def test_radius_clipping_matches_the_oracle(cfg1_setup):
    """Sec. 4.4 radius clipping at the median 1-sigma area of the frame's splats: the image matches
    the oracle with the same clipping (splats whose FP64 det lies within 1e-3 of the threshold are
    ambiguous), about half the splats lose their tiles, and zero keeps the unclipped image."""
    sc, cam, r, osc = cfg1_setup
    sp = oracle.project(osc, cam)
    cov = sp["cov"][sp["valid"] == 1]
    thr = float(np.median(np.pi * np.sqrt(cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2)))
    fl = dict(bg=(0.05, 0.1, 0.2), radius_clip_area=thr)
    img, st = gpu_image(r, cam, use_mlp=0, **fl)
    base, st0 = gpu_image(r, cam, use_mlp=0, bg=(0.05, 0.1, 0.2))
    off, _ = gpu_image(r, cam, use_mlp=0, bg=(0.05, 0.1, 0.2), radius_clip_area=0.0)
    np.testing.assert_array_equal(off, base)
    assert 0.3 * st0["n_pairs"] < st["n_pairs"] < 0.8 * st0["n_pairs"]
    ref = oracle.render(osc, cam, oracle_opts_for(fl))
    compare_images(img, ref["image"], ref["ambiguous"])
    assert np.abs(img - base).max() > 1e-2                   # clipping changed the picture


def test_render_is_deterministic(cfg1_setup):
    sc, cam, r, osc = cfg1_setup
    a, _ = gpu_image(r, cam, use_mlp=0)
    b, _ = gpu_image(r, cam, use_mlp=0)
    np.testing.assert_array_equal(a, b)


# ----------------------------------------------------------------------------- S1-S3 bit-exact
def test_fixed_logits_culled_set_and_order_are_exact(cfg1_setup):
    sc, cam, r, osc = cfg1_setup
    rng = np.random.default_rng(123)
    logits = rng.normal(0, 1, sc.n_instanced).astype(np.float32)
    d_logits = torch.from_numpy(logits).cuda()
    flags = dict(use_mlp=1, mlp_gate=0, logits_override=d_logits)
    img, st = gpu_image(r, cam, **flags)
    lf = r.last_frame()
    surv = lf["survivors"].cpu().numpy()
    inside, f_amb = oracle.frustum(osc, cam)
    keep = inside & (logits > 0)
    ora = np.nonzero(keep)[0]                    # instance-major order, one instance here
    gpu = surv[:, 1].astype(np.int64)
    amb = set(np.nonzero(f_amb)[0].tolist())
    assert np.all(np.diff(gpu) > 0), "survivors must keep (instance, gaussian) order"
    sym = set(gpu.tolist()) ^ set(ora.tolist())
    assert sym <= amb, f"{len(sym - amb)} non-ambiguous differences"
    # the culled image equals the oracle render with the same decisions
    ref = oracle.render(osc, cam, oracle_opts_for({}), keep=keep.astype(np.uint8))
    compare_images(img, ref["image"], ref["ambiguous"])
    # nvgs_query_visibility reports the same decisions
    lg, kp, _ = r.query_visibility(cam, r.flags(**flags))
    kp = kp.cpu().numpy().astype(bool)
    assert set(np.nonzero(kp != keep)[0].tolist()) <= amb


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tile_lists_are_exact(cfg1_setup, tile):
    """S5 parity: every tile's list equals the oracle's FP64 list (the tiles of the splat's support
    rectangle whose pixel-centre box meets its support ellipse), element for element and in blend
    order (depth, instance, gaussian), outside the band of pairs a conservative FP32 binner may take
    either way; per-tile counts and ranges of every tile equal the oracle's outside that band."""
    sc, cam, r, osc = cfg1_setup
    o = oracle_opts_for(dict(tile_size=tile))
    _, st = gpu_image(r, cam, use_mlp=0, tile_size=tile)
    lf = r.last_frame()
    vals = lf["pair_values"].cpu().numpy().astype(np.int64)
    surv = lf["survivors"].cpu().numpy()
    rec = lf["records"].cpu().numpy().reshape(-1, 16)
    gpu_tiles = lf["pair_keys"].cpu().numpy().astype(np.int64)
    assert np.all(np.diff(gpu_tiles) >= 0)
    sp = oracle.project(osc, cam, o)
    ell = oracle.tile_lists_ellipse(sp, cam, tile)
    drop = set(zip(sp["instance"][sp["ambiguous"] != 0].tolist(), sp["gaussian"][sp["ambiguous"] != 0].tolist()))
    depth_of = dict(zip(zip(sp["instance"].tolist(), sp["gaussian"].tolist()), sp["depth"].tolist()))
    n, n_band, n_drop = check_exact_tile_lists(gpu_tiles, surv[vals, 0], surv[vals, 1], rec[vals, 11],
                                               ell, depth_of, drop)
    print(f"tile {tile}: {n} pairs equal, {n_band} in the band, {n_drop} of dropped splats "
          f"(gpu {len(gpu_tiles)} pairs)")
    assert n > 10000 and n_band <= 1e-3 * n
    # ranges of EVERY tile: [start, end) of its pairs in the sorted list; counts = oracle's counts
    # up to the tile's band and dropped pairs
    n_tiles = lf["tiles_x"] * lf["tiles_y"]
    rng_ = lf["tile_ranges"].cpu().numpy().reshape(-1, 2)[:n_tiles]
    cnt = np.bincount(gpu_tiles, minlength=n_tiles)
    starts = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    occupied = cnt > 0
    np.testing.assert_array_equal(rng_[occupied, 0], starts[occupied])
    np.testing.assert_array_equal(rng_[occupied, 1], starts[occupied] + cnt[occupied])
    assert np.all(rng_[~occupied, 0] == rng_[~occupied, 1])
    et, ei, eg, ea = ell
    band = set(zip(et[ea].tolist(), ei[ea].tolist(), eg[ea].tolist()))
    sure_o = ~ea & np.array([(b, c) not in drop for b, c in zip(ei.tolist(), eg.tolist())], bool)
    gi, gg = surv[vals, 0], surv[vals, 1]
    sure_g = np.array([(b, c) not in drop and (t, b, c) not in band
                       for t, b, c in zip(gpu_tiles.tolist(), gi.tolist(), gg.tolist())], bool)
    np.testing.assert_array_equal(np.bincount(gpu_tiles[sure_g], minlength=n_tiles),
                                  np.bincount(et[sure_o], minlength=n_tiles))


def test_tile_lists_lie_between_support_and_rect_lists(cfg1_setup):
    """Every tile holding a pixel a splat can blend at lists it (front to back); pruned tiles are
    only ever tiles of its rectangle."""
    sc, cam, r, osc = cfg1_setup
    o = oracle_opts_for(dict(tile_size=16))
    _, st = gpu_image(r, cam, use_mlp=0, tile_size=16)
    lf = r.last_frame()
    vals = lf["pair_values"].cpu().numpy().astype(np.int64)
    surv = lf["survivors"].cpu().numpy()
    gpu_tiles = lf["pair_keys"].cpu().numpy().astype(np.int64)
    sp = oracle.project(osc, cam, o)
    support = oracle.tile_lists(sp, cam, 16, mode="support")
    rect = oracle.tile_lists(sp, cam, 16, mode="rect")
    drop = set(zip(sp["instance"][sp["ambiguous"] != 0].tolist(), sp["gaussian"][sp["ambiguous"] != 0].tolist()))
    depth_of = dict(zip(zip(sp["instance"].tolist(), sp["gaussian"].tolist()), sp["depth"].tolist()))
    n_gpu, n_sup, n_rect = check_pruned_tile_lists(gpu_tiles, surv[vals, 0], surv[vals, 1], support, rect,
                                                   depth_of, drop)
    print(f"pairs: gpu {n_gpu}, support {n_sup}, rect {n_rect}")
    assert n_sup > 10000 and n_gpu < n_rect


# ----------------------------------------------------------------------------- S2 (FP32)
def test_fp32_mlp_logits_and_decisions_match_oracle():
    sc, cam = scenes.config1_scene(), scenes.config1_camera()
    w = _random_weights()
    r = renderer_for(sc, w, precision=0)
    try:
        lg, kp, st = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0))
        lg = lg.cpu().numpy().astype(np.float64)
        osc = oracle.OracleScene(sc)
        vis = oracle.visibility(osc, cam, w, gate=False)
        inside, _ = oracle.frustum(osc, cam)
        m = inside & np.isfinite(lg)
        assert m.sum() == inside.sum() > 0
        err = np.abs(lg[m] - vis["logits"][m])
        scale = np.abs(vis["logits"][inside]).max()
        assert err.max() <= 1e-4 * max(1.0, scale), err.max()
        big = np.abs(vis["logits"][m]) > 0.05
        agree = ((lg[m] > 0) == (vis["logits"][m] > 0))[big].mean()
        assert agree == 1.0
        # culled render with the MLP's own decisions, threshold at the median logit
        thr = float(np.float32(np.median(vis["logits"][inside])))
        img, st = gpu_image(r, cam, use_mlp=1, mlp_gate=0, logit_threshold=thr)
        # with |GPU - FP64 logit| <= tol (asserted above), only a decision within tol of the
        # threshold can differ: those are banded (15 Gaussians here, reaching ~3.4 % of pixels)
        tol = 1e-4 * max(1.0, scale)
        keep, kamb = oracle.cull_decision(vis, inside, thr, band=tol)
        ref = oracle.render(osc, cam, oracle_opts_for({}), keep=keep.astype(np.uint8),
                            keep_amb=kamb.astype(np.uint8))
        compare_images(img, ref["image"], ref["ambiguous"], max_amb_frac=0.05)
        assert st["n_survivors"] < st["n_in_frustum"]
    finally:
        r.close()


# ----------------------------------------------------------------------------- several instances, SH
@pytest.mark.parametrize("deg", [1, 2, 3])
def test_instances_and_sh_degrees_match_oracle(deg):
    sc = scenes.tiny_scene(300, 10 + deg, spread=0.6, log_scale_mean=-3.0, sh_degree=deg, n_instances=4)
    cam = scenes.look_at_camera((0.6, 0.9, 2.8), (0, 0, 0), 97, 61, 55.0)   # ragged tiles
    r = renderer_for(sc)
    try:
        img, st = gpu_image(r, cam, use_mlp=0)
        osc = oracle.OracleScene(sc)
        ref = oracle.render(osc, cam, oracle_opts_for({}))
        compare_images(img, ref["image"], ref["ambiguous"])
        assert st["n_instanced"] == 1200
    finally:
        r.close()


# ----------------------------------------------------------------------------- edge cases
def test_empty_frustum_gives_background():
    sc = scenes.config1_scene(2000)
    cam = scenes.look_at_camera((0, 0, 3), (0, 0, 10), 64, 48, 50.0)   # looking away
    r = renderer_for(sc)
    try:
        img, st = gpu_image(r, cam, use_mlp=0, bg=(0.1, 0.2, 0.3))
        assert st["n_in_frustum"] == 0 and st["n_pairs"] == 0
        np.testing.assert_array_equal(img, np.broadcast_to(np.float32([0.1, 0.2, 0.3]), img.shape))
    finally:
        r.close()


def test_everything_culled_gives_background(cfg1_setup):
    sc, cam, r, osc = cfg1_setup
    d_logits = torch.full((sc.n_instanced,), -1.0, device="cuda")
    img, st = gpu_image(r, cam, use_mlp=1, mlp_gate=0, logits_override=d_logits)
    assert st["n_survivors"] == 0
    assert np.all(img == 0.0)


def test_single_gaussian_peak_alpha():
    from helpers import axis_camera, identity_instance, logit, one_asset
    cam = axis_camera(32, 32, fx=32.0)
    a = one_asset([[(10.5 - 16) * 2 / 32, (13.5 - 16) * 2 / 32, 2.0]], [[-3.0] * 3], None,
                  [logit(0.7)], np.full((1, 1, 3), 1.0))
    r = renderer_for(scenes.Scene([a], [identity_instance()]))
    try:
        img, _ = gpu_image(r, cam, use_mlp=0)
        o = 1 / (1 + math.exp(-float(np.float32(logit(0.7)))))
        rgb = 0.5 + 0.28209479177387814 * 1.0
        np.testing.assert_allclose(img[13, 10], o * rgb, rtol=2e-6)
    finally:
        r.close()


def test_invalid_arguments_are_rejected(cfg1_setup):
    from paper_2511_19202_b300.nvgs import NvgsError
    sc, cam, r, osc = cfg1_setup
    with pytest.raises(NvgsError):
        r.render(cam, r.flags(tile_size=12))
    bad = scenes.Camera(cam.R, cam.t, -1.0, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    with pytest.raises(NvgsError):
        r.render(bad)


# ----------------------------------------------------------------------------- radix sort
# (20M elements: 4883 radix tiles, more than one step of the digit-row scan, with a ragged last step)
@pytest.mark.parametrize("n,bits,spread", [(0, 8, 0), (1, 8, 0), (2, 3, 2), (1000, 7, 100),
                                           (8191, 13, 1 << 13), (8192, 45, 1 << 45),
                                           (8193, 16, 5), (100_003, 40, 1 << 40),
                                           (1_000_003, 64, 0), (777_777, 20, 3),
                                           (20_000_003, 16, 1 << 16)])
def test_radix_sort_is_a_stable_sort(cfg1_setup, n, bits, spread):
    sc, cam, r, osc = cfg1_setup
    rng = np.random.default_rng(n + bits)
    if spread:
        keys = rng.integers(0, spread, n, dtype=np.uint64)
    else:
        keys = rng.integers(0, np.iinfo(np.uint64).max, n, dtype=np.uint64, endpoint=True)
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    keys = keys & mask
    vals = np.arange(n, dtype=np.uint32)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    r.sort_pairs(dk, dv, bits)
    torch.cuda.synchronize()
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(dk.cpu().numpy().view(np.uint64), keys[order])
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), vals[order])


@pytest.mark.parametrize("n,bits", [(65_537, 13), (8193, 4), (100_003, 20), (5000, 1)])
def test_radix_sort_ignores_key_bits_above_key_bits(cfg1_setup, n, bits):
    """Keys with random bits set above key_bits: the result is the stable sort on the low key_bits
    bits alone (the last digit pass is masked), the full keys carried along."""
    sc, cam, r, osc = cfg1_setup
    rng = np.random.default_rng(n + 7 * bits)
    low = rng.integers(0, 1 << bits, n, dtype=np.uint64)
    keys = low | (rng.integers(0, 1 << (63 - bits), n, dtype=np.uint64) << np.uint64(bits))
    vals = np.arange(n, dtype=np.uint32)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    r.sort_pairs(dk, dv, bits)
    torch.cuda.synchronize()
    order = np.argsort(low, kind="stable")
    np.testing.assert_array_equal(dv.cpu().numpy().view(np.uint32), vals[order])
    np.testing.assert_array_equal(dk.cpu().numpy().view(np.uint64), keys[order])


# ----------------------------------------------------------------------------- dense-tile split
@pytest.mark.parametrize("tile", [8, 16])
def test_split_compositing_matches_one_cta_per_tile(cfg1_setup, tile):
    """Cutting every tile into 256-pair chunks (separate CTAs) changes only the grouping of the
    transmittance products: the image equals the one-CTA-per-tile image to FP32 rounding and the
    oracle within the parity tolerance."""
    sc, cam, r, osc = cfg1_setup
    one, st = gpu_image(r, cam, use_mlp=0, tile_size=tile, blend_split_len=-1)
    split, st2 = gpu_image(r, cam, use_mlp=0, tile_size=tile, blend_split_len=256)
    assert st["n_pairs"] > 256 * 4
    np.testing.assert_allclose(split, one, atol=2e-6)
    ref = oracle.render(osc, cam, oracle_opts_for(dict(tile_size=tile)))
    compare_images(split, ref["image"], ref["ambiguous"])


def test_labeller_unchanged_by_split():
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.config1_scene(20000)
    cams = [scenes.look_at_camera(12.0 * d, (0, 0, 0), 128, 128, 50.0) for d in scenes.fibonacci_directions(3)]
    r = renderer_for(sc)
    try:
        n = sc.n_instanced
        out = []
        for split in (-1, 256):
            lab = torch.zeros(len(cams) * n, dtype=torch.uint8, device="cuda")
            N.nvgs_label_visibility(r.ctx, 0, cams, N.nvgs_default_flags(use_mlp=0, blend_split_len=split), lab)
            out.append(lab.cpu().numpy())
        assert (out[0] == out[1]).mean() >= 0.9999
        assert 0.02 < out[0].mean() < 0.98
    finally:
        r.close()
