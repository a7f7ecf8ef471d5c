"""Pins of the FP64 oracle's geometry: Eq. 1, Eq. 2, MLP inputs and forward, frustum, quaternion,
3D covariance, EWA projection and SH basis.  Each expected value comes from a closed form, a
special value, an independent library routine (scipy / numpy) or a Monte Carlo estimate --
never from re-running the oracle's own formula."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle
import scenes
from helpers import axis_camera, identity_instance, one_asset


# ----------------------------------------------------------------------------- Eq. 1 (Sec. 3.1)
def test_eq1_distance_bound_closed_form():
    # r = sqrt(3), theta = 60 deg: tan(30 deg) = 1/sqrt(3), so d = 3 / p
    assert oracle.distance_bound(math.sqrt(3.0), math.pi / 3, 0.9) == pytest.approx(10.0 / 3.0, rel=1e-13)
    assert oracle.distance_bound(math.sqrt(3.0), math.pi / 3, 0.05) == pytest.approx(60.0, rel=1e-13)


def test_asset_prepare_bbox_and_eq1():
    corners = np.array([[x, y, z] for x in (-1, 1) for y in (-0.5, 0.5) for z in (-2, 2)], np.float32)
    a = one_asset(np.concatenate([corners, [[0.1, 0.2, 0.3]]]))
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]), theta_t=math.pi / 3)
    k = osc.asset_constants(0)
    np.testing.assert_array_equal(k["bbox_min"], [-1, -0.5, -2])
    np.testing.assert_array_equal(k["bbox_max"], [1, 0.5, 2])
    r = 0.5 * math.sqrt(4 + 1 + 16)              # half the box diagonal
    assert k["d_min"] == pytest.approx(r * math.sqrt(3) / 0.9, rel=1e-13)
    assert k["d_max"] == pytest.approx(r * math.sqrt(3) / 0.05, rel=1e-13)
    assert k["train_focal"] == pytest.approx(math.sqrt(3), rel=1e-13)


# ----------------------------------------------------------------------------- Eq. 2 (Sec. 3.3)
@pytest.mark.parametrize("d_local,expected", [(2.0, -1.0), (8.0, 0.0), (32.0, 1.0), (4.0, -0.5),
                                              (1.0, -1.0), (100.0, 1.0)])
def test_eq2_normalised_log_distance(d_local, expected):
    # f_t / f_r = 2, d_min = 4, d_max = 64: d_t = 2 d_local, log-min-max to [-1, 1], clamped
    assert oracle.normalised_distance(d_local, 2.0, 1.0, 4.0, 64.0) == pytest.approx(expected, abs=1e-14)


def test_eq2_instance_scale_and_fov_ratio_enter_distance():
    # one Gaussian at the local origin; instance scale s = 2 at world (0, 0, 10); camera at the
    # world origin looking down +z with f_r = 2 fx / W = 1 (90 deg); training fov 60 deg (f_t=sqrt 3)
    corners = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float32)
    a = one_asset(np.concatenate([[[0.0, 0.0, 0.0]], corners]))
    inst = scenes.Instance(0, np.eye(3, dtype=np.float32), np.array([0, 0, 10], np.float32), 2.0)
    osc = oracle.OracleScene(scenes.Scene([a], [inst]), theta_t=math.pi / 3, d_min=2.0, d_max=200.0)
    cam = axis_camera(64, 64, fx=32.0)
    f = oracle.visibility(osc, cam, return_features=True)["features"][0]
    d_t = (10.0 / 2.0) * math.sqrt(3.0) / 1.0                  # Eq. 2: d_r f_t / f_r / s
    expected = 2.0 * (math.log(d_t) - math.log(2.0)) / (math.log(200.0) - math.log(2.0)) - 1.0
    assert f[30] == pytest.approx(expected, abs=1e-13)
    np.testing.assert_allclose(f[27:30], [0, 0, 1], atol=1e-15)  # camera -> Gaussian, local frame


# ----------------------------------------------------------------------------- MLP inputs
def test_mlp_features_special_values():
    corners = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float32)
    a = one_asset(corners)
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]), d_min=1.0, d_max=100.0)
    mu = np.array([0.5, 1.0 / 6.0, 0.0])
    cl = np.array([0.5, 1.0 / 6.0, 10.0])
    f = oracle.features(osc, 0, mu, cl, f_r=osc.asset_constants(0)["train_focal"])
    s3 = math.sqrt(3) / 2
    np.testing.assert_allclose(f[0:3], mu, atol=1e-15)
    # sin(2^k pi p) for k = 0..3, axis-minor
    np.testing.assert_allclose(f[3:15], [1, 0.5, 0, 0, s3, 0, 0, s3, 0, 0, -s3, 0], atol=1e-14)
    # cos(2^k pi p)
    np.testing.assert_allclose(f[15:27], [0, s3, 1, -1, 0.5, 1, 1, -0.5, 1, 1, -0.5, 1], atol=1e-14)
    np.testing.assert_allclose(f[27:30], [0, 0, -1], atol=1e-15)
    # distance 10 with f_t = f_r: log-normalised between 1 and 100 -> exactly 0
    assert f[30] == pytest.approx(0.0, abs=1e-14)
    assert f[31] == 0.0


def test_mlp_features_bbox_normalisation():
    corners = np.array([[x, y, z] for x in (-3, 1) for y in (0, 2) for z in (5, 6)], np.float32)
    a = one_asset(corners)
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]), d_min=1.0, d_max=100.0)
    for mu, p in [((-3, 0, 5), (-1, -1, -1)), ((1, 2, 6), (1, 1, 1)), ((-1, 1, 5.5), (0, 0, 0))]:
        f = oracle.features(osc, 0, np.array(mu, float), np.array([0, 0, -20.0]), 1.0)
        np.testing.assert_allclose(f[0:3], p, atol=1e-15)


def test_mlp_forward_equals_numpy_matmul():
    rng = np.random.default_rng(3)
    w = scenes.mlp_weights(5)
    for k in range(1, 5):
        w[f"b{k}"] = rng.normal(0, 0.3, w[f"b{k}"].shape).astype(np.float32)
    x = rng.normal(0, 1, (257, 32))
    got = oracle.mlp_forward(w, x)
    h = x
    for k in range(1, 4):
        h = np.maximum(h @ w[f"W{k}"].astype(np.float64).T + w[f"b{k}"], 0.0)
    ref = (h @ w["W4"].astype(np.float64).T + w["b4"])[:, 0]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_visibility_gate_uses_corrected_centre_distance():
    corners = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float32)
    a = one_asset(corners)
    cam = axis_camera(64, 64, fx=32.0)                      # f_r = 1
    for z, s, bypass in [(3.0, 1.0, True), (6.0, 1.0, False), (6.0, 2.0, True)]:
        inst = scenes.Instance(0, np.eye(3, dtype=np.float32), np.array([0, 0, z], np.float32), s)
        osc = oracle.OracleScene(scenes.Scene([a], [inst]), theta_t=math.pi / 2, d_min=4.0, d_max=40.0)
        g = oracle.visibility(osc, cam, gate=True)["gated"]
        assert g.all() == bypass and g.any() == bypass      # d_t = z / s (f_t = f_r = 1)


def test_visibility_at_equals_the_full_evaluation():
    """The sampled entry point (used where a full FP64 evaluation of every Gaussian is too slow)
    returns exactly what the full evaluation returns at those Gaussians, gate flags included."""
    assets = [scenes.random_asset(k, 300 + 50 * k, sh_degree=0) for k in range(3)]
    rng = np.random.default_rng(3)
    insts = [scenes.Instance(k % 3, Rotation.random(random_state=k).as_matrix().astype(np.float32),
                             rng.uniform(-2, 2, 3).astype(np.float32), float(rng.uniform(0.5, 2)))
             for k in range(7)]
    sc = scenes.Scene(assets, insts)
    osc = oracle.OracleScene(sc, d_min=8.0, d_max=60.0)   # gates about half of the instances
    cam = scenes.look_at_camera((0, 1, 9), (0, 0, 0), 96, 64, 50.0)
    w = scenes.mlp_weights(5)
    full = oracle.visibility(osc, cam, w, gate=True, return_features=True)
    idx = np.concatenate([rng.integers(0, sc.n_instanced, 200), [0, sc.n_instanced - 1]])
    got = oracle.visibility_at(osc, cam, idx, w, gate=True, return_features=True)
    assert np.array_equal(got["logits"], full["logits"][idx])
    assert np.array_equal(got["gated"], full["gated"][idx])
    assert np.array_equal(got["features"], full["features"][idx])
    assert full["gated"].any() and not full["gated"].all()
    with pytest.raises(ValueError):
        oracle.visibility_at(osc, cam, [sc.n_instanced], w)


# ----------------------------------------------------------------------------- frustum (Sec. 3.3)
def test_frustum_guard_band_and_near_plane():
    cam = axis_camera(32, 32, fx=40.0)                     # tan(half fov) = 16/40 = 0.4
    lim = 1.3 * 0.4
    z = 2.0
    pts = [(0, 0, z, True), (lim * z * (1 - 1e-9), 0, z, True), (lim * z * (1 + 1e-9), 0, z, False),
           (0, -lim * z * (1 - 1e-9), z, True), (0, -lim * z * (1 + 1e-9), z, False),
           (0, 0, 0.2, False), (0, 0, 0.2 * (1 + 1e-9), True), (0, 0, -1.0, False)]
    a = one_asset([p[:3] for p in pts])
    a.means = np.array([p[:3] for p in pts], np.float64)     # keep the exact FP64 positions
    osc = oracle.OracleScene(scenes.Scene([a], [identity_instance()]))
    inside, amb = oracle.frustum(osc, cam)
    assert inside.tolist() == [p[3] for p in pts]
    assert amb[1] and amb[2] and not amb[0]


# ----------------------------------------------------------------------------- rotation / covariance
def test_quaternion_rotation_matches_scipy():
    rng = np.random.default_rng(0)
    for _ in range(50):
        q = rng.normal(0, 1, 4) * rng.uniform(0.2, 5.0)      # unnormalised on purpose
        R = oracle.quat_to_rot(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy is (x, y, z, w)
        np.testing.assert_allclose(R, ref, atol=1e-13)


def test_cov3d_eigendecomposition():
    rng = np.random.default_rng(1)
    for _ in range(20):
        ls = rng.normal(-1, 1, 3)
        q = rng.normal(0, 1, 4)
        S = oracle.cov3d(ls, q)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        for j in range(3):
            np.testing.assert_allclose(S @ R[:, j], math.exp(2 * ls[j]) * R[:, j], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(S)), np.sort(np.exp(2 * ls)), rtol=1e-12)


# ----------------------------------------------------------------------------- EWA projection
def _single_splat(mean_w, log_scale, quat=(1, 0, 0, 0), inst=None, cam=None, logit=2.0):
    a = one_asset([mean_w], [log_scale], [quat], [logit])
    inst = inst or identity_instance()
    cam = cam or axis_camera(64, 64, fx=50.0)
    osc = oracle.OracleScene(scenes.Scene([a], [inst]))
    return oracle.project(osc, cam)[0], cam


def test_projection_isotropic_on_axis_closed_form():
    sigma, z = math.exp(-3.0), 3.0
    sp, cam = _single_splat((0, 0, z), (-3, -3, -3))
    v = cam.fx ** 2 * sigma ** 2 / z ** 2 + 0.3
    np.testing.assert_allclose(sp["cov"], [v, 0, v], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(sp["conic"], [1 / v, 0, 1 / v], rtol=1e-12, atol=1e-15)
    assert sp["u"] == pytest.approx(cam.cx) and sp["v"] == pytest.approx(cam.cy)
    assert sp["depth"] == pytest.approx(z)


def test_projection_instance_scale_and_rotation_isotropic():
    sigma, z, s = math.exp(-3.0), 3.0, 2.0
    R = Rotation.from_euler("xyz", [0.3, -1.1, 2.0]).as_matrix().astype(np.float32)
    inst = scenes.Instance(0, R, np.array([0, 0, z], np.float32), s)
    sp, cam = _single_splat((0, 0, 0), (-3, -3, -3), inst=inst)
    v = cam.fx ** 2 * (s * sigma) ** 2 / z ** 2 + 0.3
    np.testing.assert_allclose(sp["cov"], [v, 0, v], rtol=1e-6, atol=1e-6)  # R is rounded to FP32


def test_projection_isotropic_off_axis_closed_form():
    sigma, z, x = math.exp(-3.0), 4.0, 1.0
    sp, cam = _single_splat((x, 0, z), (-3, -3, -3))
    exp_a = sigma ** 2 * cam.fx ** 2 / z ** 2 * (1 + x ** 2 / z ** 2) + 0.3
    exp_c = sigma ** 2 * cam.fy ** 2 / z ** 2 + 0.3
    np.testing.assert_allclose(sp["cov"], [exp_a, 0, exp_c], rtol=1e-12, atol=1e-15)
    assert sp["u"] == pytest.approx(cam.fx * x / z + cam.cx, rel=1e-14)


def test_projection_anisotropic_matches_monte_carlo():
    """Sample the 3D Gaussian, push every sample through the exact instance, camera and
    perspective maps, and compare the empirical 2D covariance with the oracle's EWA splat."""
    rng = np.random.default_rng(2)
    ls = np.array([-6.0, -7.0, -6.5])
    q = np.array([0.8, 0.3, -0.4, 0.2])
    mu = np.array([0.2, -0.1, 0.3])
    R_i = Rotation.from_euler("zyx", [0.7, 0.2, -0.4]).as_matrix()
    inst = scenes.Instance(0, R_i.astype(np.float32), np.array([0.4, 0.3, 3.0], np.float32), 1.7)
    Rc = Rotation.from_euler("xyz", [0.05, -0.1, 0.02]).as_matrix()
    cam = scenes.Camera(Rc.astype(np.float32), np.array([0.1, -0.2, 0.5], np.float32), 300.0, 280.0,
                        64.0, 48.0, 128, 96)
    sp, _ = _single_splat(mu, ls, q, inst=inst, cam=cam)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    L = R @ np.diag(np.exp(ls))
    n = 400_000
    x = mu[None, :] + rng.standard_normal((n, 3)) @ L.T
    xw = (np.asarray(inst.R, np.float64) @ (float(inst.s) * x).T).T + np.asarray(inst.t, np.float64)
    xc = (np.asarray(cam.R, np.float64) @ xw.T).T + np.asarray(cam.t, np.float64)
    u = cam.fx * xc[:, 0] / xc[:, 2] + cam.cx
    v = cam.fy * xc[:, 1] / xc[:, 2] + cam.cy
    emp = np.cov(np.stack([u, v]))
    got = np.array([[sp["cov"][0] - 0.3, sp["cov"][1]], [sp["cov"][1], sp["cov"][2] - 0.3]])
    scale = np.sqrt(np.outer(np.diag(emp), np.diag(emp)))
    np.testing.assert_allclose(got / scale, emp / scale, atol=1.5e-2)
    assert sp["u"] == pytest.approx(np.mean(u), abs=3e-3 * math.sqrt(emp[0, 0]) + 1e-2)


def test_projection_jacobian_matches_finite_differences():
    """J (with the guard-band clamp inactive) equals the numerical derivative of the pinhole map."""
    ls = np.array([-2.0, -2.5, -1.8])
    q = np.array([0.3, -0.6, 0.2, 0.7])
    mu = np.array([0.4, -0.3, 2.5])
    cam = axis_camera(128, 128, fx=90.0, fy=85.0)
    sp, _ = _single_splat(mu, ls, q, cam=cam)

    def proj(p):
        return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

    h = 1e-6
    J = np.stack([(proj(mu + h * e) - proj(mu - h * e)) / (2 * h) for e in np.eye(3)], 1)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    S = R @ np.diag(np.exp(2 * ls)) @ R.T
    ref = J @ S @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose([sp["cov"][0], sp["cov"][1], sp["cov"][2]],
                               [ref[0, 0], ref[0, 1], ref[1, 1]], rtol=1e-6)


# ----------------------------------------------------------------------------- SH (3DGS colour)
def _real_sh_scipy(l, m, d):
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    Y = sph_harm_y(l, abs(m), theta, phi)
    return math.sqrt(2) * (Y.real if m > 0 else Y.imag)


def test_sh_basis_matches_scipy_real_harmonics():
    rng = np.random.default_rng(4)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = oracle.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(got[:, l * l + l + m], _real_sh_scipy(l, m, d), atol=1e-12,
                                       err_msg=f"l={l} m={m}")


def test_sh_colour_uses_local_view_direction():
    """Rotating the instance together with its SH-coded colour field: the colour seen from a fixed
    camera depends only on the local direction, so rotating the instance by Q and the camera
    around it by Q gives the same colour."""
    rng = np.random.default_rng(5)
    sh = rng.normal(0, 0.4, (1, 16, 3))
    a = one_asset([[0, 0, 0]], [[-3, -3, -3]], None, [2.0], sh, sh_degree=3)
    cam0 = scenes.look_at_camera((0.3, 0.4, 3.0), (0, 0, 0), 64, 64, 50.0)
    Q = Rotation.from_euler("xyz", [0.4, 1.0, -0.3]).as_matrix()
    inst1 = scenes.Instance(0, Q.astype(np.float32), np.zeros(3, np.float32), 1.0)
    eye1 = Q @ cam0.center
    cam1 = scenes.Camera((np.asarray(cam0.R, np.float64) @ Q.T).astype(np.float32),
                         (-(np.asarray(cam0.R, np.float64) @ Q.T) @ eye1).astype(np.float32),
                         cam0.fx, cam0.fy, cam0.cx, cam0.cy, 64, 64)
    s0 = oracle.project(oracle.OracleScene(scenes.Scene([a], [identity_instance()])), cam0)[0]
    s1 = oracle.project(oracle.OracleScene(scenes.Scene([a], [inst1])), cam1)[0]
    np.testing.assert_allclose(s0["rgb"], s1["rgb"], atol=1e-6)
    d = -cam0.center / np.linalg.norm(cam0.center)
    Y = np.array([_real_sh_scipy(l, m, d[None])[0] for l in range(4) for m in range(-l, l + 1)])
    np.testing.assert_allclose(s0["rgb"], np.maximum(0.0, 0.5 + Y @ sh[0].astype(np.float32)), atol=1e-12)
