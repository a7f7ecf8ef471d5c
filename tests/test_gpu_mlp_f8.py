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
from gpu_common import compare_images, e4m3, f8_reference, gpu_image, layered_case, oracle_opts_for, renderer_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FP8 = 2


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
