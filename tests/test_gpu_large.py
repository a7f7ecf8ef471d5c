"""GPU parity on the large instanced scene with FP8 MLPs (8 assets x 1M Gaussians, SH degree 3, at
3840 x 2160): the scene's first 50 of its 200 instances (the instances are drawn one after another
from one seeded stream, so these are exactly the full scene's first 50: 50M instanced Gaussians),
through the same C-ABI calls the bench times.  The FP64 oracle checks what it can compute one by
one: FP8 logits and decisions at sampled Gaussians (against the kernel's documented quantised
arithmetic and against the unquantised FP64 MLP), the survivor set of a culled frame, and sampled
4K image rows of that frame (injected logits that both sides use), unculled and culled."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_common import compare_images, f8_reference, oracle_opts_for, renderer_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

FP8 = 2
N_INSTANCES = 50
# first and last rows, a tile boundary (15 | 16), the middle, a ragged last tile row (2160 = 135 x 16)
ROWS = np.array([0, 15, 16, 1080, 2150, 2159], np.int32)


def _weights(k):
    w = scenes.mlp_weights(300 + k)
    rng = np.random.default_rng(900 + k)
    for j in range(1, 5):
        w[f"b{j}"] = rng.normal(0, 0.3, w[f"b{j}"].shape).astype(np.float32)
    return w


@pytest.fixture(scope="module")
def large():
    sc = scenes.config5_scene(n_instances=N_INSTANCES)
    cam = scenes.config5_camera(0)
    weights = [_weights(k) for k in range(len(sc.assets))]
    r = renderer_for(sc, weights, precision=FP8)
    osc = oracle.OracleScene(sc)
    inside, f_amb = oracle.frustum(osc, cam)
    try:
        yield sc, cam, weights, r, osc, inside, f_amb
    finally:
        r.close()


def _instance_of(sc, idx):
    offs = np.cumsum([0] + [sc.assets[i.asset_id].n for i in sc.instances])
    return np.searchsorted(offs, idx, side="right") - 1


def _instanced_index(sc, surv):
    offs = np.cumsum([0] + [sc.assets[i.asset_id].n for i in sc.instances])
    return offs[surv[:, 0].astype(np.int64)] + surv[:, 1].astype(np.int64)


def test_large_fp8_sampled_logits_and_decisions(large):
    sc, cam, weights, r, osc, inside, f_amb = large
    assert sc.n_instanced == N_INSTANCES * 1_000_000 and (cam.width, cam.height) == (3840, 2160)
    lg, kp, st = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0, tile_size=16))
    lg = lg.cpu().numpy().astype(np.float64)
    kp = kp.cpu().numpy().astype(bool)
    assert st["n_in_frustum"] > 5_000_000
    assert abs(st["n_in_frustum"] - int(inside.sum())) <= int(f_amb.sum())
    sure_in = inside & ~f_amb
    np.testing.assert_array_equal(kp[sure_in], lg[sure_in] > 0)
    assert not kp[~inside & ~f_amb].any()
    rng = np.random.default_rng(2025)
    idx = np.sort(rng.choice(np.nonzero(sure_in)[0], 20000, replace=False))
    vis = oracle.visibility_at(osc, cam, idx, None, gate=False, return_features=True)
    inst = _instance_of(sc, idx)
    q = np.empty(idx.size)
    ora = np.empty(idx.size)
    for k in range(len(sc.assets)):
        m = np.array([sc.instances[i].asset_id == k for i in inst])
        if m.any():
            q[m] = f8_reference(weights[k], vis["features"][m])
            ora[m] = oracle.mlp_forward(weights[k], vis["features"][m])
    scale = float(np.percentile(np.abs(ora), 99))
    e_q = np.abs(lg[idx] - q)
    e_o = np.abs(lg[idx] - ora)
    big = np.abs(ora) > 0.1 * scale
    agree = float(((lg[idx] > 0) == (ora > 0))[big].mean())
    print(f"large FP8: {idx.size} sampled queries; vs quantised reference p99 {np.percentile(e_q, 99):.3e} "
          f"max {e_q.max():.3e}; vs FP64 p99 {np.percentile(e_o, 99):.3e} (scale {scale:.3f}); "
          f"agree {agree:.4f} beyond 10 % of the scale")
    # the documented quantised arithmetic, up to accumulation order and rare boundary flips
    assert np.percentile(e_q, 99) <= 2e-3 * scale
    assert (e_q > 2e-2 * scale).mean() <= 0.01
    # E4M3's 3 mantissa bits: a few percent of the logit scale; decisions hold away from 0
    assert np.percentile(e_o, 99) <= 0.15 * scale
    assert agree >= 0.98


def test_large_unculled_rows_match_oracle(large):
    sc, cam, weights, r, osc, inside, f_amb = large
    img, st = r.render(cam, r.flags(use_mlp=0, tile_size=16))
    img = img.cpu().numpy().astype(np.float64)
    ref = oracle.render_rows(osc, cam, ROWS, oracle_opts_for(dict(tile_size=16)))
    err, n_amb = compare_images(img[ROWS], ref["image"], ref["ambiguous"], max_amb_frac=0.12)
    print(f"large unculled: {st['n_pairs']} pairs, rows {ROWS.tolist()}: max err {err:.2e}, "
          f"{n_amb} ambiguous pixels of {ROWS.size * cam.width}")


def test_large_culled_survivors_and_rows_match_oracle(large):
    """Culling with injected logits (the same seeded values on both sides) at 4K: the survivor set is
    exact outside the frustum band and the sampled rows equal the oracle's culled render."""
    sc, cam, weights, r, osc, inside, f_amb = large
    logits = np.random.default_rng(78).normal(0.0, 1.0, sc.n_instanced).astype(np.float32)
    d_logits = torch.from_numpy(logits).cuda()
    img, st = r.render(cam, r.flags(use_mlp=1, mlp_gate=0, tile_size=16, logits_override=d_logits))
    img = img.cpu().numpy().astype(np.float64)
    lf = r.last_frame()
    keep = inside & (logits > 0)
    gpu = np.sort(_instanced_index(sc, lf["survivors"].cpu().numpy()))
    ora = np.nonzero(keep)[0]
    sym = np.setxor1d(gpu, ora)
    assert f_amb[sym].all(), f"{int((~f_amb[sym]).sum())} survivors differ outside the frustum band"
    ref = oracle.render_rows(osc, cam, ROWS, oracle_opts_for(dict(tile_size=16)), keep=keep.astype(np.uint8))
    err, n_amb = compare_images(img[ROWS], ref["image"], ref["ambiguous"], max_amb_frac=0.12)
    print(f"large culled (injected logits): {gpu.size} survivors, {st['n_pairs']} pairs; rows: "
          f"max err {err:.2e}, {n_amb} ambiguous pixels")
