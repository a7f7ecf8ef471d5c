"""GPU parity of the BF16 tensor-core visibility MLP (tcgen05) against the FP64 oracle: logits
within the BF16 error budget, decisions agreeing on >= 99.9% of Gaussians with |logit| > 0.05;
against the kernel's own quantised arithmetic on the oracle's inputs, logits within 1e-3 of the
scale and decisions equal outside a 1% band; multi-asset tiles; and the culled image against the
oracle render with the decisions taken in BF16 on the oracle's side."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_common import (BF16_DECISION_BAND, bf16_reference, bf16_round, compare_images, gpu_image,
                        layered_case, oracle_opts_for, renderer_for)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

BF16 = 1


def _weights(seed, bias_std=0.3):
    w = scenes.mlp_weights(seed)
    rng = np.random.default_rng(seed + 7)
    for k in range(1, 5):
        w[f"b{k}"] = rng.normal(0, bias_std, w[f"b{k}"].shape).astype(np.float32)
    return w


def _check_logits(lg_gpu, lg_ora, mask):
    lg_gpu = lg_gpu[mask].astype(np.float64)
    lg_ora = lg_ora[mask]
    err = np.abs(lg_gpu - lg_ora)
    big = np.abs(lg_ora) > 0.05
    agree = float(((lg_gpu > 0) == (lg_ora > 0))[big].mean())
    # BF16 operands (8-bit mantissa) through three 64-wide layers: a few 1e-2 of the logit scale
    scale = float(np.percentile(np.abs(lg_ora), 99))
    assert np.percentile(err, 99) <= 0.02 * max(1.0, scale), (np.percentile(err, 99), scale)
    assert agree >= 0.999, agree
    return err, agree


def test_bf16_logits_match_oracle_cfg1():
    sc, cam = scenes.config1_scene(), scenes.config1_camera()
    w = _weights(42)
    r = renderer_for(sc, w, precision=BF16)
    try:
        lg, kp, st = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0))
        lg = lg.cpu().numpy()
        osc = oracle.OracleScene(sc)
        vis = oracle.visibility(osc, cam, w, gate=False)
        inside, _ = oracle.frustum(osc, cam)
        assert np.isfinite(lg[inside]).all()
        err, agree = _check_logits(lg, vis["logits"], inside)
        print(f"bf16 logits: max err {err.max():.3e}, p99 {np.percentile(err, 99):.3e}, agree {agree:.5f}")
        kp = kp.cpu().numpy().astype(bool)
        np.testing.assert_array_equal(kp, inside & (lg > 0))
    finally:
        r.close()


def test_bf16_rounding_reference():
    # exact values, ties to even (1 + 2^-8 down, 1 + 3 * 2^-8 up), a carry into the exponent
    assert bf16_round([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7 + 2.0 ** -9, -3.3,
                       255.9]).tolist() == [1.0, 1.0, 1.015625, 1.0078125, -3.296875, 256.0]


def test_bf16_logits_match_the_quantised_reference():
    """The kernel's logits against its own quantised arithmetic (BF16 operands, exact sums) on
    the oracle's FP64 inputs: the decision is taken in the kernel's precision on both sides."""
    sc, cam = scenes.config1_scene(), scenes.config1_camera()
    w = _weights(42)
    r = renderer_for(sc, w, precision=BF16)
    try:
        lg, kp, _ = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0))
        lg = lg.cpu().numpy().astype(np.float64)
    finally:
        r.close()
    osc = oracle.OracleScene(sc)
    inside, _ = oracle.frustum(osc, cam)
    ref = bf16_reference(w, oracle.visibility(osc, cam, w, gate=False, return_features=True)["features"][inside])
    scale = float(np.percentile(np.abs(ref), 99))
    e = np.abs(lg[inside] - ref)
    amb = np.abs(ref) <= BF16_DECISION_BAND * scale
    print(f"bf16 vs quantised reference: p99 {np.percentile(e, 99):.3e} max {e.max():.3e} "
          f"(scale {scale:.3f}), banded {amb.mean():.4f}")
    assert np.percentile(e, 99) <= 1e-3 * scale
    assert e.max() <= BF16_DECISION_BAND * scale
    assert amb.mean() <= 0.05
    np.testing.assert_array_equal((lg[inside] > 0)[~amb], (ref > 0)[~amb])


@pytest.mark.parametrize("side,ctas_per_sm", [(3, 0), (6, 1)])
def test_bf16_multi_asset_tiles(side, ctas_per_sm):
    """Three assets, side^2 instances: tiles straddle instance and asset boundaries.  With 36
    instances (~90k rows) and one CTA per SM every CTA walks several steps, so the inputs built
    ahead for a CTA's next step meet asset changes too."""
    assets = [scenes.torus_asset(3001, seed=1, sh_degree=0), scenes.sphere_asset(2500, 2, sh_degree=0),
              scenes.box_asset(1999, 3, sh_degree=0)]
    rng = np.random.default_rng(5)
    insts = []
    for k in range(side * side):
        q, rr = np.linalg.qr(rng.standard_normal((3, 3)))
        q = q * np.sign(np.diag(rr))
        if np.linalg.det(q) < 0:
            q[:, 0] *= -1
        insts.append(scenes.Instance(k % 3, q.astype(np.float32),
                                     np.array([(k % side - (side - 1) / 2) * 2.5,
                                               (k // side - (side - 1) / 2) * 2.5, 0], np.float32),
                                     float(np.float32(rng.uniform(0.6, 1.2)))))
    sc = scenes.Scene(assets, insts)
    cam = scenes.look_at_camera((0.5, 1.0, 3.0 * side), (0, 0, 0), 320, 240, 60.0)
    ws = [_weights(100 + k) for k in range(3)]
    r = renderer_for(sc, ws, precision=BF16)
    try:
        lg, kp, st = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0, mlp_ctas_per_sm=ctas_per_sm))
        if side == 6:
            assert st["n_in_frustum"] > 148 * 256 * 2   # several 256-row steps per CTA
        osc = oracle.OracleScene(sc)
        inside, _ = oracle.frustum(osc, cam)
        # oracle logits per asset's own weights (one instance at a time)
        ora = np.zeros(sc.n_instanced)
        off = 0
        for k, inst in enumerate(insts):
            n = assets[inst.asset_id].n
            sub = oracle.OracleScene(scenes.Scene(assets, [inst]))
            ora[off:off + n] = oracle.visibility(sub, cam, ws[inst.asset_id], gate=False)["logits"]
            off += n
        _check_logits(lg.cpu().numpy(), ora, inside)
    finally:
        r.close()


def test_bf16_culled_render_matches_oracle_with_same_decisions():
    """The BF16-culled image against the oracle render with the decisions taken in the kernel's
    precision on the oracle's side (the quantised reference on FP64 features), on trained-like
    bimodal logits: no decision inside the band, at most 2 % of the pixels ambiguous."""
    sc, cam, dist, osc, inside, w = layered_case()
    r = renderer_for(sc, w, precision=BF16, **dist)
    try:
        lg, kp, _ = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0))
        kp = kp.cpu().numpy().astype(bool)
        img, st = gpu_image(r, cam, use_mlp=1, mlp_gate=0)
    finally:
        r.close()
    vis = oracle.visibility(osc, cam, w, gate=False, return_features=True)
    q = np.zeros(sc.n_instanced)
    q[inside] = bf16_reference(w, vis["features"][inside])
    band = BF16_DECISION_BAND * float(np.percentile(np.abs(q[inside]), 99))
    keep = inside & (q > 0)
    amb = inside & (np.abs(q) <= band)
    assert amb.sum() <= 0.001 * inside.sum()
    assert 0.2 * inside.sum() < keep.sum() < 0.5 * inside.sum()
    np.testing.assert_array_equal(kp[inside & ~amb], keep[inside & ~amb])
    ref = oracle.render(osc, cam, oracle_opts_for({}), keep=keep.astype(np.uint8),
                        keep_amb=amb.astype(np.uint8))
    err, n_amb = compare_images(img, ref["image"], ref["ambiguous"], max_amb_frac=0.02)
    print(f"bf16 culled render: kept {keep.sum()}/{inside.sum()}, max err {err:.2e}, "
          f"ambiguous pixels {n_amb}")
    assert st["n_mlp_queries"] == st["n_in_frustum"]
