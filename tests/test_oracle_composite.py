"""Pins of the oracle's compositing (Sec. 4.1 blending rules) and visibility labels (Sec. 3.1):
closed forms for one Gaussian, the telescoping identity of front-to-back compositing, brute
force on tiny scenes, invariance under removal of zero-contribution Gaussians, the opaque-slab
occlusion case, rigid-motion invariance and input-order invariance."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import scenes
from helpers import axis_camera, identity_instance, logit, one_asset


def _pixel_point(cam, px, py, z):
    """World point (camera = world frame) that projects onto the centre of pixel (px, py)."""
    return [((px + 0.5) - cam.cx) * z / cam.fx, ((py + 0.5) - cam.cy) * z / cam.fy, z]


C0 = 0.5 / math.sqrt(math.pi)


@pytest.mark.parametrize("opacity", [0.3, 0.7, 0.995])
def test_single_gaussian_peak_alpha_equals_opacity(opacity):
    cam = axis_camera(32, 32, fx=32.0)          # pixel centres map to binary-exact points
    sh0 = np.array([0.2, -0.4, 0.9]) / 1.0
    a = one_asset([_pixel_point(cam, 10, 13, 2.0)], [[-3.0, -3.0, -3.0]], None, [logit(opacity)],
                  sh0.reshape(1, 1, 3))
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]))
    r = oracle.render(osc, cam)
    rgb = np.maximum(0.0, 0.5 + C0 * sh0.astype(np.float32).astype(np.float64))
    al = min(0.99, float(1.0 / (1.0 + math.exp(-np.float32(logit(opacity))))))
    np.testing.assert_allclose(r["image"][13, 10], al * rgb, rtol=1e-12)
    assert r["T"][13, 10] == pytest.approx(1.0 - al, rel=1e-12)


def test_single_gaussian_off_centre_falloff():
    cam = axis_camera(32, 32, fx=32.0, cx=16.5, cy=16.5)   # pixel (16, 16) on the optical axis
    sigma, z = math.exp(-2.5), 2.0
    a = one_asset([_pixel_point(cam, 16, 16, z)], [[-2.5] * 3], None, [logit(0.8)],
                  np.full((1, 1, 3), 1.0))
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]))
    r = oracle.render(osc, cam)
    var = cam.fx ** 2 * sigma ** 2 / z ** 2 + 0.3          # isotropic closed form (on axis)
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit(0.8)))))
    rgb = 0.5 + C0 * float(np.float32(1.0))
    for dx, dy in [(1, 0), (0, 2), (2, 1), (-3, 1)]:
        al = o * math.exp(-0.5 * (dx * dx + dy * dy) / var)
        got = r["image"][16 + dy, 16 + dx, 0]
        if al >= 1 / 255:
            assert got == pytest.approx(al * rgb, rel=1e-10)
        else:
            assert got == 0.0


def test_telescoping_weights_sum_to_one(cfg1):
    scene, cam = cfg1
    osc = oracle.OracleScene(scene)
    o = oracle.opts()
    sp = oracle.project(osc, cam, o)
    rng = np.random.default_rng(0)
    for _ in range(25):
        x, y = int(rng.integers(40, 216)), int(rng.integers(40, 216))
        w, T = oracle.pixel_weights(sp, cam, o, x, y)
        assert w.sum() + T == pytest.approx(1.0, abs=1e-12)
        assert np.all(w >= 0) and T >= o.t_stop


def _python_brute_force(sp, cam, o):
    """Per pixel over ALL splats (no bounding box), explicit sort and loop."""
    H, W = cam.height, cam.width
    img = np.zeros((H, W, 3))
    v = sp[sp["valid"] != 0]
    for y in range(H):
        for x in range(W):
            frs = []
            for s in v:
                dx, dy = x + 0.5 - s["u"], y + 0.5 - s["v"]
                p = -0.5 * (s["conic"][0] * dx * dx + s["conic"][2] * dy * dy) - s["conic"][1] * dx * dy
                al = min(o.alpha_max, s["opacity"] * math.exp(p))
                if p > 0 or al < o.alpha_min:
                    continue
                frs.append((s["depth"], s["instance"], s["gaussian"], al, s["rgb"]))
            frs.sort(key=lambda f: (f[0], f[1], f[2]))
            T, C = 1.0, np.zeros(3)
            for f in frs:
                if T * (1 - f[3]) < o.t_stop:
                    break
                C += f[3] * T * f[4]
                T *= 1 - f[3]
            img[y, x] = C + T * np.array(o.bg[:])
    return img


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_support_restriction_equals_brute_force(seed):
    sc = scenes.tiny_scene(8, seed, spread=0.25, depth=3.0, log_scale_mean=-2.0, n_instances=2)
    cam = scenes.look_at_camera((0, 0, 3.0), (0, 0, 0), 12, 10, 30.0)
    o = oracle.opts(bg=(0.1, 0.2, 0.3))
    osc = oracle.OracleScene(sc)
    sp = oracle.project(osc, cam, o)
    fast = oracle.composite(sp, cam, o)["image"]
    brute_c = oracle.composite(sp, cam, o, brute_force=True)["image"]
    np.testing.assert_array_equal(fast, brute_c)
    np.testing.assert_allclose(fast, _python_brute_force(sp, cam, o), atol=1e-13)


def test_support_bbox_contains_every_pixel_above_alpha_min(cfg1):
    scene, cam = cfg1
    osc = oracle.OracleScene(scene)
    o = oracle.opts()
    sp = oracle.project(osc, cam, o)
    v = sp[sp["valid"] != 0][:400]
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    for s in v:
        dx, dy = xs + 0.5 - s["u"], ys + 0.5 - s["v"]
        p = -0.5 * (s["conic"][0] * dx * dx + s["conic"][2] * dy * dy) - s["conic"][1] * dx * dy
        hit = s["opacity"] * np.exp(p) >= o.alpha_min
        yy, xx = np.nonzero(hit)
        if yy.size:
            assert xx.min() >= s["px_min"][0] and xx.max() <= s["px_max"][0]
            assert yy.min() >= s["px_min"][1] and yy.max() <= s["px_max"][1]


def test_removing_zero_contribution_gaussians_is_exact(cfg1):
    scene, cam = cfg1
    osc = oracle.OracleScene(scene)
    o = oracle.opts()
    full = oracle.render(osc, cam, o, want_contrib=True)
    used = full["n_contrib"] > 0
    assert 0 < used.sum() < used.size
    keep = used.astype(np.uint8)
    culled = oracle.render(osc, cam, o, keep=keep)
    np.testing.assert_array_equal(full["image"], culled["image"])
    np.testing.assert_array_equal(full["T"], culled["T"])


def test_opaque_slab_occludes_what_lies_behind():
    """Two layers of near-opaque splats (alpha = 0.99) bring T to 1e-4 after the first layer
    pair; the stop rule (Sec. 4.1) then rejects every fragment behind them: those Gaussians are
    labelled invisible (Sec. 3.1), the ones in front stay visible."""
    cam = axis_camera(16, 16, fx=20.0)
    grid = [(((x + 0.5) - 8) * z / 20.0, ((y + 0.5) - 8) * z / 20.0, z)
            for z in (2.0, 2.1) for y in range(-2, 18, 2) for x in range(-2, 18, 2)]
    behind = [(0.0, 0.0, 3.0), (0.2, -0.1, 3.5)]
    front = [(0.1, 0.1, 1.5)]
    pts = grid + behind + front
    n = len(pts)
    a = one_asset(pts, np.full((n, 3), -1.2), None, np.full(n, 12.0), np.full((n, 1, 3), 0.5))
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]))
    r = oracle.render(osc, cam, want_contrib=True)
    c = r["n_contrib"]
    assert np.all(c[len(grid):len(grid) + len(behind)] == 0)
    assert c[-1] > 0
    assert np.all(r["T"] >= 1e-4)


def test_stop_rule_rejects_the_fragment_that_would_cross_t_stop():
    """Three fragments centred on one pixel, front to back with alpha 0.99 (clamped), 0.98 and
    0.6: T goes 1 -> 0.01 -> 2e-4; the third would leave T (1 - 0.6) = 8e-5 < 1e-4, so it is
    not blended and the pixel stops (Sec. 4.1; the test happens before blending)."""
    cam = axis_camera(8, 8, fx=10.0)
    pts = [_pixel_point(cam, 4, 4, z) for z in (1.0, 1.5, 2.0)]
    rgb = np.eye(3)
    a = one_asset(pts, np.full((3, 3), -3.0), None, [12.0, logit(0.98), logit(0.6)],
                  ((rgb - 0.5) / C0).reshape(3, 1, 3))
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]))
    r = oracle.render(osc, cam, oracle.opts(alpha_max=0.99))
    np.testing.assert_allclose(r["image"][4, 4], [0.99, 0.01 * 0.98, 0.0], rtol=1e-6, atol=1e-7)
    assert r["T"][4, 4] == pytest.approx(0.01 * 0.02, rel=1e-6)


def test_input_order_does_not_change_the_image(cfg1):
    scene, cam = cfg1
    a = scene.assets[0]
    perm = np.random.default_rng(9).permutation(a.n)
    sc2 = scenes.Scene([a.subset(perm)], scene.instances)
    i1 = oracle.render(oracle.OracleScene(scene), cam)["image"]
    i2 = oracle.render(oracle.OracleScene(sc2), cam)["image"]
    # equal up to the order of equal-depth ties, which the scene does not contain
    np.testing.assert_allclose(i1, i2, atol=1e-12)


def test_rigid_motion_of_the_world_leaves_the_image_unchanged():
    sc = scenes.tiny_scene(40, 3, spread=0.5, log_scale_mean=-2.5, sh_degree=2, n_instances=3)
    cam = scenes.look_at_camera((0.5, 0.8, 3.0), (0, 0, 0), 48, 40, 45.0)
    Q = Rotation.from_euler("xyz", [0.7, -0.2, 1.3]).as_matrix()
    d = np.array([1.0, -2.0, 0.5])
    insts = [scenes.Instance(i.asset_id, (Q @ i.R).astype(np.float64), Q @ i.t + d, i.s)
             for i in sc.instances]
    Rc = np.asarray(cam.R, np.float64) @ Q.T
    cam2 = scenes.Camera(Rc, np.asarray(cam.t, np.float64) - Rc @ d, cam.fx, cam.fy, cam.cx,
                         cam.cy, cam.width, cam.height)
    # keep FP64 transforms so that the motion is exact up to rounding
    sc1 = scenes.Scene(sc.assets, [scenes.Instance(i.asset_id, i.R.astype(np.float64), i.t.astype(np.float64), i.s)
                                   for i in sc.instances])
    i1 = oracle.render(oracle.OracleScene(sc1), cam)["image"]
    i2 = oracle.render(oracle.OracleScene(scenes.Scene(sc.assets, insts)), cam2)["image"]
    np.testing.assert_allclose(i1, i2, atol=1e-9)


def test_background_is_weighted_by_final_transmittance(cfg1):
    scene, cam = cfg1
    osc = oracle.OracleScene(scene)
    r0 = oracle.render(osc, cam, oracle.opts())
    r1 = oracle.render(osc, cam, oracle.opts(bg=(0.25, 0.5, 1.0)))
    np.testing.assert_allclose(r1["image"] - r0["image"], r0["T"][..., None] * [0.25, 0.5, 1.0],
                               atol=1e-13)


def test_row_subset_equals_full_frame(cfg1):
    scene, cam = cfg1
    osc = oracle.OracleScene(scene)
    full = oracle.render(osc, cam)["image"]
    rows = np.array([3, 100, 101, 200, 255], np.int32)
    sub = oracle.render(osc, cam, rows=rows)["image"]
    np.testing.assert_array_equal(sub, full[rows])


def test_memory_light_row_render_equals_full_frame():
    sc = scenes.tiny_scene(400, 21, spread=0.7, log_scale_mean=-3.0, sh_degree=1, n_instances=3)
    cam = scenes.look_at_camera((0.4, 0.7, 3.0), (0, 0, 0), 80, 60, 50.0)
    osc = oracle.OracleScene(sc)
    full = oracle.render(osc, cam)
    rows = np.array([0, 17, 30, 31, 59], np.int32)
    sub = oracle.render_rows(osc, cam, rows)
    np.testing.assert_array_equal(sub["image"], full["image"][rows])
    np.testing.assert_array_equal(sub["ambiguous"], full["ambiguous"][rows])
    assert 0 < sub["n_splats"] < sc.n_instanced


def test_tile_lists_cover_every_blended_pixel(cfg1):
    scene, cam = cfg1
    osc = oracle.OracleScene(scene)
    o = oracle.opts(tile_size=16)
    sp = oracle.project(osc, cam, o)
    tiles, inst, gs = oracle.tile_lists(sp, cam, 16)
    tw = cam.width // 16
    member = set(zip(tiles.tolist(), gs.tolist()))
    v = sp[sp["valid"] != 0][:300]
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    for s in v:
        dx, dy = xs + 0.5 - s["u"], ys + 0.5 - s["v"]
        p = -0.5 * (s["conic"][0] * dx * dx + s["conic"][2] * dy * dy) - s["conic"][1] * dx * dy
        yy, xx = np.nonzero(s["opacity"] * np.exp(p) >= o.alpha_min)
        for t in set(((yy // 16) * tw + xx // 16).tolist()):
            assert (t, s["gaussian"]) in member
    # blend order inside each tile: non-decreasing depth
    depth = dict(zip(sp["gaussian"].tolist(), sp["depth"].tolist()))
    d = np.array([depth[g] for g in gs.tolist()])
    same = tiles[1:] == tiles[:-1]
    assert np.all(d[1:][same] >= d[:-1][same])


def test_support_tile_lists_are_the_tiles_of_blendable_pixels(cfg1):
    """Support mode lists exactly the tiles holding a pixel with alpha >= 1/255 (brute force over
    the whole image, through the exponential rather than the quadratic form), inside the rect
    lists."""
    scene, cam = cfg1
    osc = oracle.OracleScene(scene)
    o = oracle.opts(tile_size=16)
    sp = oracle.project(osc, cam, o)
    v = sp[sp["valid"] != 0][:300]
    tiles, inst, gs = oracle.tile_lists(v, cam, 16, mode="support")
    rt, ri, rg = oracle.tile_lists(v, cam, 16, mode="rect")
    member = set(zip(tiles.tolist(), gs.tolist()))
    assert member <= set(zip(rt.tolist(), rg.tolist()))
    tw = cam.width // 16
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    brute = set()
    for s in v:
        dx, dy = xs + 0.5 - s["u"], ys + 0.5 - s["v"]
        p = -0.5 * (s["conic"][0] * dx * dx + s["conic"][2] * dy * dy) - s["conic"][1] * dx * dy
        yy, xx = np.nonzero(s["opacity"] * np.exp(p) >= o.alpha_min)
        brute |= {(t, int(s["gaussian"])) for t in set(((yy // 16) * tw + xx // 16).tolist())}
    assert member == brute


def test_support_tile_list_of_a_circle_off_a_tile_corner():
    """Closed form: a circular support of radius 5 px centred at (20, 20) has a 2 x 2 tile rectangle
    (pixels 15 ... 24) but misses tile (0, 0), whose nearest pixel centre (15.5, 15.5) lies 6.4 px
    away; tiles (1, 0) and (0, 1) are reached at (19.5, 15.5) and (15.5, 19.5), 4.5 px away."""
    cam = axis_camera(64, 64, fx=64.0)
    sp = np.zeros(1, oracle.SPLAT_DTYPE)
    op, am = 0.8, 1.0 / 255.0
    kk = 2.0 * math.log(op / am)
    sigma2 = 25.0 / kk                   # q = r^2 / sigma^2 = kk at r = 5
    sp["valid"], sp["u"], sp["v"], sp["opacity"] = 1, 20.0, 20.0, op
    sp["conic"] = [[1.0 / sigma2, 0.0, 1.0 / sigma2]]
    sp["px_min"], sp["px_max"] = [[15, 15]], [[24, 24]]
    sp["tile_min"], sp["tile_max"] = [[0, 0]], [[1, 1]]
    rect = oracle.tile_lists(sp, cam, 16, mode="rect")[0]
    supp = oracle.tile_lists(sp, cam, 16, mode="support")[0]
    assert rect.tolist() == [0, 1, 4, 5] and supp.tolist() == [1, 4, 5]
    sp["u"], sp["v"] = 16.0, 16.0        # on the corner: all four tiles are reached
    sp["px_min"], sp["px_max"] = [[11, 11]], [[20, 20]]
    assert oracle.tile_lists(sp, cam, 16, mode="support")[0].tolist() == [0, 1, 4, 5]


def test_box_min_quadratic_against_dense_sampling():
    """The minimum of a positive-definite quadratic over a box: never above any sampled value, and
    within the sampling's resolution of the densest sample (2001^2 points per box), for boxes that
    hold the origin, sit beside it and lie diagonally off it; the box on the origin gives 0."""
    rng = np.random.default_rng(3)
    for k in range(40):
        L = rng.normal(size=(2, 2)) + 0.3 * np.eye(2)
        a, b, c = (L @ L.T)[0, 0], (L @ L.T)[0, 1], (L @ L.T)[1, 1]
        x0, y0 = rng.uniform(-3, 3, 2)
        x1, y1 = x0 + rng.uniform(0.1, 2), y0 + rng.uniform(0.1, 2)
        m = float(oracle.box_min_quadratic(a, b, c, x0, x1, y0, y1))
        xs, ys = np.meshgrid(np.linspace(x0, x1, 2001), np.linspace(y0, y1, 2001))
        q = a * xs * xs + 2 * b * xs * ys + c * ys * ys
        assert m <= q.min() + 1e-12
        step = max(x1 - x0, y1 - y0) / 2000
        grad = 2 * math.sqrt(max(a, c) * max(q.min(), 1e-12)) * step + 2 * max(a, c) * step ** 2
        assert q.min() - m <= grad + 1e-12, (k, m, q.min())
    assert oracle.box_min_quadratic(1.0, 0.2, 2.0, -1, 1, -0.5, 0.5) == 0.0


def _circle_splat(u, v, radius, op=0.8, tile=((0, 0), (1, 1))):
    """One valid circular splat whose support (alpha >= 1/255) has the given radius in pixels."""
    sp = np.zeros(1, oracle.SPLAT_DTYPE)
    kk = 2.0 * math.log(op / (1.0 / 255.0))
    sigma2 = radius * radius / kk
    sp["valid"], sp["u"], sp["v"], sp["opacity"], sp["depth"] = 1, u, v, op, 1.0
    sp["conic"] = [[1.0 / sigma2, 0.0, 1.0 / sigma2]]
    sp["tile_min"], sp["tile_max"] = [tile[0]], [tile[1]]
    return sp


def test_ellipse_tile_list_of_a_circle_closed_form():
    """Closed form: a circle of radius 5 px at (20, 20) meets the pixel-centre boxes of tiles
    (1, 0), (0, 1) and (1, 1) (distances 4.5, 4.5 and 0) but not tile (0, 0)'s box [0.5, 15.5]^2,
    whose corner (15.5, 15.5) lies 6.364 px away; at radius 6.4, or 1e-7 px beyond the corner, it
    reaches that corner; 1e-7 px short of it the pair falls in the band a conservative binner may
    take either way, and 1 % short of it the pair is out.  A circle between the pixel centres of one tile row, x in [15.6, 15.9], never reaches
    tile (1, 0)'s box (x >= 16.5) although its rectangle holds it."""
    cam = axis_camera(64, 64, fx=64.0)
    t, i, g, amb = oracle.tile_lists_ellipse(_circle_splat(20.0, 20.0, 5.0), cam, 16)
    assert t.tolist() == [1, 4, 5] and not amb.any()
    t, i, g, amb = oracle.tile_lists_ellipse(_circle_splat(20.0, 20.0, 6.4), cam, 16)
    assert t.tolist() == [0, 1, 4, 5] and not amb.any()
    d = math.hypot(4.5, 4.5)
    t, i, g, amb = oracle.tile_lists_ellipse(_circle_splat(20.0, 20.0, d + 1e-7), cam, 16)
    assert t.tolist() == [0, 1, 4, 5] and not amb.any()
    t, i, g, amb = oracle.tile_lists_ellipse(_circle_splat(20.0, 20.0, d - 1e-7), cam, 16)
    assert t.tolist() == [0, 1, 4, 5] and amb.tolist() == [True, False, False, False]
    t, i, g, amb = oracle.tile_lists_ellipse(_circle_splat(20.0, 20.0, 0.99 * d), cam, 16)
    assert t.tolist() == [1, 4, 5] and not amb.any()
    t, i, g, amb = oracle.tile_lists_ellipse(_circle_splat(15.4, 8.0, 0.15, tile=((0, 0), (1, 0))), cam, 16)
    assert t.tolist() == [0] and not amb.any()
    # a one-tile rectangle is listed as it is
    t, i, g, amb = oracle.tile_lists_ellipse(_circle_splat(15.75, 8.0, 0.15, tile=((1, 0), (1, 0))), cam, 16)
    assert t.tolist() == [1]


def test_ellipse_tile_lists_between_support_and_rect_lists(cfg1):
    """On the workload-1 frame: support lists (tiles with a pixel centre the splat blends at)
    <= ellipse lists (tiles whose pixel-centre box the support ellipse meets) <= rect lists, in
    blend order; the band is a small fraction; each ellipse pair is confirmed by brute force (a
    point of the tile's pixel-centre box on a 65 x 65 grid inside the support, or the box's nearest
    grid point within the grid's resolution)."""
    scene, cam = cfg1
    osc = oracle.OracleScene(scene)
    sp = oracle.project(osc, cam, oracle.opts(tile_size=16))
    v = sp[sp["valid"] != 0][:400]
    et, ei, eg, ea = oracle.tile_lists_ellipse(v, cam, 16)
    st, si, sg = oracle.tile_lists(v, cam, 16, mode="support")
    rt, ri, rg = oracle.tile_lists(v, cam, 16, mode="rect")
    ell = set(zip(et[~ea].tolist(), eg[~ea].tolist()))
    assert set(zip(st.tolist(), sg.tolist())) <= ell
    assert set(zip(et.tolist(), eg.tolist())) <= set(zip(rt.tolist(), rg.tolist()))
    assert len(ell) < len(rt) and ea.mean() < 1e-2
    by_g = {int(s["gaussian"]): s for s in v}
    tw = cam.width // 16
    for t, gg, am in zip(et.tolist(), eg.tolist(), ea.tolist()):
        s = by_g[gg]
        if am or (s["tile_min"] == s["tile_max"]).all():
            continue
        tx, ty = t % tw, t // tw
        xs, ys = np.meshgrid(np.linspace(tx * 16 + 0.5, tx * 16 + 15.5, 65) - s["u"],
                             np.linspace(ty * 16 + 0.5, ty * 16 + 15.5, 65) - s["v"])
        a, b, c = s["conic"]
        q = a * xs * xs + 2 * b * xs * ys + c * ys * ys
        kk = 2.0 * math.log(s["opacity"] * 255.0)
        slack = 2 * math.sqrt(max(a, c) * kk) * (15.0 / 64) + 2 * max(a, c) * (15.0 / 64) ** 2
        assert q.min() <= kk + slack, (t, gg)
    # blend order inside each tile
    depth = dict(zip(v["gaussian"].tolist(), v["depth"].tolist()))
    d = np.array([depth[x] for x in eg.tolist()])
    same = et[1:] == et[:-1]
    assert np.all(d[1:][same] >= d[:-1][same])


@pytest.mark.parametrize("side", [-1, 1])
def test_radius_clipping_threshold_is_the_one_sigma_area(side):
    """Sec. 4.4 radius clipping, pinned on one isotropic Gaussian on the optical axis: there
    Sigma_2D = ((f sigma / z)^2 + 0.3) I, whose 1-sigma ellipse has area pi ((f sigma / z)^2 + 0.3).
    A threshold 1 % above it drops the splat (the image is the background); 1 % below keeps the
    unclipped image."""
    cam = axis_camera(32, 32, fx=32.0, cx=16.5, cy=16.5)
    sigma, z = math.exp(-2.5), 2.0
    a = one_asset([[0.0, 0.0, z]], [[math.log(sigma)] * 3], None, [logit(0.8)],
                  np.full((1, 1, 3), 0.6))
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]))
    s32 = math.exp(float(np.float32(math.log(sigma))))
    area = math.pi * ((32.0 * s32 / z) ** 2 + 0.3)
    bg = (0.1, 0.2, 0.3)
    ref = oracle.render(osc, cam, oracle.opts(bg=bg))["image"]
    got = oracle.render(osc, cam, oracle.opts(bg=bg, radius_clip_area=area * (1.0 + 0.01 * side)))["image"]
    assert np.abs(ref - np.asarray(bg)).max() > 0.1          # the splat is visible unclipped
    if side > 0:
        np.testing.assert_array_equal(got, np.broadcast_to(np.asarray(bg), got.shape))
    else:
        np.testing.assert_array_equal(got, ref)

