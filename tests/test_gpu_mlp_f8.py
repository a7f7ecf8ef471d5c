"""GPU parity of the FP8 (E4M3) tensor-core visibility MLP.

Two references: (1) a numpy restatement of the quantised pipeline the kernel documents (E4M3
round-to-nearest-even with saturation, per-tensor scales max|W|/448, inputs x 256, hidden bounds /
448, FP32 epilogue constants) on the oracle's FP64 inputs -- the kernel must match it up to
accumulation order and the rare quantisation decision that FP32 inputs take the other way; (2)
the FP64 oracle's unquantised logits -- FP8's error budget, and culling decisions that agree away
from the threshold."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_common import compare_images, gpu_image, layered_case, oracle_opts_for, renderer_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FP8 = 2


def e4m3(x):
    """Round to the nearest E4M3 value (ties to even), saturating at +-448; subnormals 2^-9 apart."""
    x = np.asarray(x, np.float64)
    a = np.minimum(np.abs(x), 448.0)
    out = np.zeros_like(a)
    sub = a < 2.0 ** -6
    out[sub] = np.rint(a[sub] / 2.0 ** -9) * 2.0 ** -9
    nrm = ~sub & (a > 0)
    e = np.floor(np.log2(a[nrm]))
    q = 2.0 ** (e - 3)
    out[nrm] = np.minimum(np.rint(a[nrm] / q) * q, 448.0)
    return np.sign(x) * out


def f8_reference(w, feats):
    W1, b1 = w["W1"].astype(np.float64), w["b1"].astype(np.float64)
    W2, b2 = w["W2"].astype(np.float64), w["b2"].astype(np.float64)
    W3, b3 = w["W3"].astype(np.float64), w["b3"].astype(np.float64)
    W4, b4 = w["W4"].astype(np.float64).ravel(), float(np.ravel(w["b4"])[0])
    f32 = np.float32
    sW = [np.abs(W).max() / 448.0 for W in (W1, W2, W3)]
    B1 = (np.abs(W1).sum(1) + np.abs(b1)).max()
    B2 = (np.abs(W2).sum(1) * B1 + np.abs(b2)).max()
    sh1, sh2 = B1 / 448.0, B2 / 448.0
    a1, a2, a3 = f32(sW[0] / 256.0 / sh1), f32(sh1 * sW[1] / sh2), f32(sh2 * sW[2])
    be1, be2 = (b1 / sh1).astype(f32), (b2 / sh2).astype(f32)
    qx = e4m3(256.0 * feats)
    acc1 = (qx @ e4m3(W1 / sW[0]).T).astype(f32)
    q1 = e4m3(np.maximum(acc1 * a1 + be1, 0).astype(f32))
    acc2 = (q1 @ e4m3(W2 / sW[1]).T).astype(f32)
    q2 = e4m3(np.maximum(acc2 * a2 + be2, 0).astype(f32))
    acc3 = (q2 @ e4m3(W3 / sW[2]).T).astype(f32)
    h3 = np.maximum(acc3 * a3 + b3.astype(f32), 0).astype(np.float64)
    return h3 @ W4.astype(f32).astype(np.float64) + b4


def test_e4m3_rounding_reference():
    # exact values, ties to even, saturation, subnormals
    assert e4m3([1.0, 1.0625, 1.1875, 448.0, 500.0, -3.3, 2.0 ** -9, 3 * 2.0 ** -10]).tolist() == \
        [1.0, 1.0, 1.25, 448.0, 448.0, -3.25, 2.0 ** -9, 2 * 2.0 ** -9]


def _weights(seed, bias_std=0.3):
    w = scenes.mlp_weights(seed)
    rng = np.random.default_rng(seed + 7)
    for k in range(1, 5):
        w[f"b{k}"] = rng.normal(0, bias_std, w[f"b{k}"].shape).astype(np.float32)
    return w


def test_fp8_logits_match_the_quantised_reference_and_the_oracle():
    sc, cam = scenes.config1_scene(), scenes.config1_camera()
    w = _weights(42)
    r = renderer_for(sc, w, precision=FP8)
    try:
        lg, kp, st = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0))
        lg = lg.cpu().numpy().astype(np.float64)
        kp = kp.cpu().numpy().astype(bool)
    finally:
        r.close()
    osc = oracle.OracleScene(sc)
    vis = oracle.visibility(osc, cam, w, gate=False, return_features=True)
    inside, _ = oracle.frustum(osc, cam)
    assert np.isfinite(lg[inside]).all()
    ref = f8_reference(w, vis["features"][inside])
    scale = float(np.percentile(np.abs(vis["logits"][inside]), 99))
    e_q = np.abs(lg[inside] - ref)
    e_o = np.abs(lg[inside] - vis["logits"][inside])
    big = np.abs(vis["logits"][inside]) > 0.1 * scale
    agree = float(((lg[inside] > 0) == (vis["logits"][inside] > 0))[big].mean())
    big05 = np.abs(vis["logits"][inside]) > 0.05
    agree05 = float(((lg[inside] > 0) == (vis["logits"][inside] > 0))[big05].mean())
    print(f"fp8: vs quantised reference p99 {np.percentile(e_q, 99):.3e} max {e_q.max():.3e}; "
          f"vs FP64 p99 {np.percentile(e_o, 99):.3e} (scale {scale:.3f}); agree {agree:.4f} "
          f"beyond 10 % of the scale, {agree05:.4f} beyond |logit| 0.05 (random weights)")
    # (1) the documented quantised arithmetic, up to accumulation order and rare boundary flips
    assert np.percentile(e_q, 99) <= 2e-3 * scale
    assert (e_q > 2e-2 * scale).mean() <= 0.01
    # (2) E4M3 keeps 3 mantissa bits: a few percent of the logit scale; decisions hold away from 0
    assert np.percentile(e_o, 99) <= 0.15 * scale
    assert agree >= 0.98
    np.testing.assert_array_equal(kp, inside & (lg > 0))


def test_fp8_culling_in_a_multi_asset_render():
    """Three assets with FP8 MLPs render end to end; the culled set is the logits' decision and the
    image equals the render with those decisions injected (FP32 path)."""
    assets = [scenes.random_asset(k, 4000, sh_degree=1) for k in range(3)]
    rng = np.random.default_rng(5)
    insts = [scenes.Instance(k % 3, np.eye(3, dtype=np.float32),
                             rng.uniform(-2, 2, 3).astype(np.float32) * np.float32([1, 0.3, 1]), 1.0)
             for k in range(9)]
    sc = scenes.Scene(assets, insts)
    cam = scenes.look_at_camera((0.5, 2.0, 7.0), (0, 0, 0), 160, 120, 55.0)
    ws = [_weights(10 + k) for k in range(3)]
    r = renderer_for(sc, ws, precision=FP8)
    try:
        lg, kp, _ = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0))
        img, st = r.render(cam, r.flags(use_mlp=1, mlp_gate=0))
        assert 0 < st["n_survivors"] < st["n_in_frustum"]
        inj = torch.where(kp.bool(), torch.ones_like(lg), -torch.ones_like(lg)).float()
        inj = torch.nan_to_num(inj, nan=-1.0)
        img2, st2 = r.render(cam, r.flags(use_mlp=1, mlp_gate=0, logits_override=inj))
        assert st2["n_survivors"] == st["n_survivors"]
        assert torch.equal(img, img2)
    finally:
        r.close()


def test_fp8_culled_render_matches_oracle_on_bimodal_logits():
    """Trained-like, bimodal logits (the layered torus case, a distance cut): FP8 decisions agree
    with the FP64 oracle on every Gaussian with |logit| > 0.05, and the FP8-culled image matches
    the oracle render with the oracle's decisions (the quantised reference's decisions agree)."""
    sc, cam, dist, osc, inside, w = layered_case()
    r = renderer_for(sc, w, precision=FP8, **dist)
    try:
        lg, kp, _ = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0))
        lg = lg.cpu().numpy().astype(np.float64)
        kp = kp.cpu().numpy().astype(bool)
        img, st = gpu_image(r, cam, use_mlp=1, mlp_gate=0)
    finally:
        r.close()
    vis = oracle.visibility(osc, cam, w, gate=False, return_features=True)
    ora = vis["logits"]
    big = inside & (np.abs(ora) > 0.05)
    agree = float(((lg > 0) == (ora > 0))[big].mean())
    q = f8_reference(w, vis["features"][inside])
    print(f"fp8 bimodal: agreement {agree:.5f} on {big.sum()} Gaussians with |logit| > 0.05; "
          f"quantised-reference decisions equal: {((q > 0) == (ora[inside] > 0)).mean():.5f}")
    assert agree >= 0.999
    keep = inside & (ora > 0)
    np.testing.assert_array_equal(kp, inside & (lg > 0))
    np.testing.assert_array_equal(kp[big], keep[big])
    amb = inside & ~big
    ref = oracle.render(osc, cam, oracle_opts_for({}), keep=keep.astype(np.uint8), keep_amb=amb.astype(np.uint8))
    compare_images(img, ref["image"], ref["ambiguous"], max_amb_frac=0.02)
    assert 0 < st["n_survivors"] < st["n_in_frustum"]
