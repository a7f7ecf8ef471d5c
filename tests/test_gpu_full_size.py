"""GPU parity at the full size of the timed workload: the composed scene (16 assets x 500k
Gaussians, 64 instances = 32M instanced Gaussians, SH degree 3) at 1920 x 1080 with 16 x 16 tiles
and BF16 visibility MLPs, through the same C-ABI calls and launch configuration the bench times.
Where the FP64 oracle cannot evaluate the whole frame in seconds, the test compares outputs it can
compute one by one: MLP logits and decisions at sampled Gaussians, the in-frustum and survivor
sets, and sampled image rows (unculled, and culled with injected logits that both sides use)."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_common import (BF16_DECISION_BAND, bf16_reference, compare_images, oracle_opts_for,
                        renderer_for)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

BF16 = 1
# first and last rows, a tile boundary (15 | 16), the middle, and a ragged last tile row (1072+)
ROWS = np.array([0, 15, 16, 540, 1075, 1079], np.int32)


@pytest.fixture(scope="module")
def full():
    sc = scenes.config2_scene()
    cam = scenes.config2_camera(0)
    weights = [scenes.mlp_weights(42 + k) for k in range(len(sc.assets))]
    r = renderer_for(sc, weights, precision=BF16)
    osc = oracle.OracleScene(sc)
    inside, f_amb = oracle.frustum(osc, cam)
    try:
        yield sc, cam, weights, r, osc, inside, f_amb
    finally:
        r.close()


def _instanced_index(sc, surv):
    offs = np.cumsum([0] + [sc.assets[i.asset_id].n for i in sc.instances])
    return offs[surv[:, 0].astype(np.int64)] + surv[:, 1].astype(np.int64)


def test_full_size_sampled_logits_and_decisions(full):
    sc, cam, weights, r, osc, inside, f_amb = full
    assert sc.n_instanced == 32_000_000 and (cam.width, cam.height) == (1920, 1080)
    flags = r.flags(use_mlp=1, mlp_gate=1, tile_size=16, logit_threshold=0.0)
    lg, kp, st = r.query_visibility(cam, flags)
    lg = lg.cpu().numpy().astype(np.float64)
    kp = kp.cpu().numpy().astype(bool)
    # every decision is the kernel's own logit against the threshold, at all 32M Gaussians
    assert st["n_in_frustum"] > 10_000_000
    assert abs(st["n_in_frustum"] - int(inside.sum())) <= int(f_amb.sum())
    sure_in = inside & ~f_amb
    assert not np.isnan(lg[sure_in]).any()          # bypassed instances report +inf
    np.testing.assert_array_equal(kp[sure_in], lg[sure_in] > 0)
    assert not kp[~inside & ~f_amb].any()
    # 20k sampled in-frustum Gaussians through the oracle
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(np.nonzero(sure_in)[0], 20000, replace=False))
    vis = oracle.visibility_at(osc, cam, idx, None, gate=True, return_features=True)
    gated = vis["gated"]
    assert gated.any() and not gated.all()          # both paths occur in this frame
    assert np.isinf(lg[idx[gated]]).all() and kp[idx[gated]].all()   # bypassed: kept
    q = np.empty(idx.size)
    for k in range(len(sc.assets)):   # each sample through its own asset's weights
        m = np.array([sc.instances[i].asset_id == k for i in _instance_of(sc, idx)]) & ~gated
        if m.any():
            q[m] = bf16_reference(weights[k], vis["features"][m])
    ng = ~gated
    scale = float(np.percentile(np.abs(q[ng]), 99))
    e = np.abs(lg[idx[ng]] - q[ng])
    amb = np.abs(q[ng]) <= BF16_DECISION_BAND * scale
    print(f"full size: {ng.sum()} sampled MLP queries, vs quantised reference p99 "
          f"{np.percentile(e, 99):.3e} max {e.max():.3e} (scale {scale:.3f}), banded {amb.mean():.4f}")
    assert np.percentile(e, 99) <= 1e-3 * scale
    assert e.max() <= BF16_DECISION_BAND * scale
    assert amb.mean() <= 0.05
    np.testing.assert_array_equal((lg[idx[ng]] > 0)[~amb], (q[ng] > 0)[~amb])


def _instance_of(sc, idx):
    offs = np.cumsum([0] + [sc.assets[i.asset_id].n for i in sc.instances])
    return np.searchsorted(offs, idx, side="right") - 1


def test_full_size_unculled_rows_match_oracle(full):
    sc, cam, weights, r, osc, inside, f_amb = full
    img, st = r.render(cam, r.flags(use_mlp=0, tile_size=16))
    img = img.cpu().numpy().astype(np.float64)
    ref = oracle.render_rows(osc, cam, ROWS, oracle_opts_for(dict(tile_size=16)))
    err, n_amb = compare_images(img[ROWS], ref["image"], ref["ambiguous"], max_amb_frac=0.12)
    print(f"full size unculled: {st['n_pairs']} pairs, rows {ROWS.tolist()}: max err {err:.2e}, "
          f"{n_amb} ambiguous pixels of {ROWS.size * cam.width}")
    assert st["n_pairs"] > 50_000_000


def test_full_size_culled_survivors_and_rows_match_oracle(full):
    """Culling with injected logits (the same seeded values on both sides): the survivor set is
    exact outside the frustum band and the sampled rows equal the oracle's culled render."""
    sc, cam, weights, r, osc, inside, f_amb = full
    logits = np.random.default_rng(77).normal(0.0, 1.0, sc.n_instanced).astype(np.float32)
    d_logits = torch.from_numpy(logits).cuda()
    img, st = r.render(cam, r.flags(use_mlp=1, mlp_gate=0, tile_size=16, logits_override=d_logits))
    img = img.cpu().numpy().astype(np.float64)
    lf = r.last_frame()
    keep = inside & (logits > 0)
    gpu = np.sort(_instanced_index(sc, lf["survivors"].cpu().numpy()))
    ora = np.nonzero(keep)[0]
    sym = np.setxor1d(gpu, ora)
    assert f_amb[sym].all(), f"{int((~f_amb[sym]).sum())} survivors differ outside the frustum band"
    assert abs(gpu.size - ora.size) <= int(f_amb.sum())
    ref = oracle.render_rows(osc, cam, ROWS, oracle_opts_for(dict(tile_size=16)), keep=keep.astype(np.uint8))
    err, n_amb = compare_images(img[ROWS], ref["image"], ref["ambiguous"], max_amb_frac=0.12)
    print(f"full size culled (injected logits): {gpu.size} survivors, {st['n_pairs']} pairs; rows: "
          f"max err {err:.2e}, {n_amb} ambiguous pixels")
