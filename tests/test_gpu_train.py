"""GPU parity of the visibility labeller and the MLP training step (N1) against the FP64 oracle,
and an end-to-end check that training on GPU labels learns the occlusion it is shown."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_common import renderer_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_labeller_matches_oracle_contributions():
    sc = scenes.config1_scene(6000)
    cams = [scenes.look_at_camera(3.0 * d, (0, 0, 0), 160, 120, 50.0) for d in scenes.fibonacci_directions(5)]
    r = renderer_for(sc)
    try:
        from paper_2511_19202_b300 import nvgs as N
        n = sc.n_instanced
        labels = torch.zeros(len(cams) * n, dtype=torch.uint8, device="cuda")
        N.nvgs_label_visibility(r.ctx, 0, cams, N.nvgs_default_flags(use_mlp=0), labels)
        gpu = labels.cpu().numpy().reshape(len(cams), n).astype(bool)
        osc = oracle.OracleScene(sc)
        ora = oracle.labels(osc, cams)
        agree = (gpu == ora).mean()
        print(f"labels: agree {agree:.5f}, visible {ora.mean():.3f}, differ {(gpu != ora).sum()}")
        assert agree >= 0.999
        assert 0.05 < ora.mean() < 0.95
        # the user's scene is back in place after labelling
        img, st = r.render(scenes.config1_camera(), r.flags(use_mlp=0))
        assert st["n_instanced"] == n
    finally:
        r.close()


def test_train_step_matches_oracle_gradient():
    """With beta1 = beta2 = 0 and lr = eps = 1e6 one Adam step moves each weight by
    g / (1 + |g| / 1e6) ~ g, so the updated weights expose the batch gradient."""
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.config1_scene(3000)
    cams = [scenes.look_at_camera(3.0 * d, (0, 0, 0), 128, 128, 50.0) for d in scenes.fibonacci_directions(6)]
    rng = np.random.default_rng(0)
    labels = (rng.random((6, 3000)) < 0.4).astype(np.uint8)
    B = 1000
    sv = rng.integers(0, 6, B).astype(np.int32)
    sg = rng.integers(0, 3000, B).astype(np.int32)
    w = scenes.mlp_weights(3)
    for k in range(1, 5):
        w[f"b{k}"] = rng.normal(0, 0.2, w[f"b{k}"].shape).astype(np.float32)
    w0 = N.flat_weights(w)
    r = renderer_for(sc)
    try:
        N.nvgs_train_init(r.ctx, 0, w0, cams)
        d_lab = torch.from_numpy(labels.ravel()).cuda()
        loss = N.nvgs_train_visibility_step(r.ctx, 0, d_lab, B, 0, 1e6, sample_view=torch.from_numpy(sv).cuda(),
                                            sample_gauss=torch.from_numpy(sg).cuda(), beta1=0.0, beta2=0.0,
                                            eps=1e6, want_loss=True)
        w1 = N.nvgs_train_get_weights(r.ctx, 0).astype(np.float64)
    finally:
        r.close()
    osc = oracle.OracleScene(sc)
    views = oracle.training_views_table(cams)
    w_or = oracle.flat_weights(w)                 # the oracle packs its own copy of the weights
    np.testing.assert_array_equal(np.asarray(w0, np.float64), w_or)   # same layout on both sides
    ref_loss, g = oracle.train_loss_grad(osc, 0, views, labels, sv, sg, w_or)
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    step_gpu = w0.astype(np.float64) - w1
    step_ref = g / (1.0 + np.abs(g) / 1e6)
    scale = np.abs(step_ref).max()
    err = np.abs(step_gpu - step_ref).max()
    print(f"train step: loss {loss:.6f} vs {ref_loss:.6f}, max grad err {err:.2e} (scale {scale:.2e})")
    assert err <= 1e-4 * scale + 2e-7


@pytest.mark.parametrize("B", [1000, 4096])
def test_bf16_train_step_matches_oracle_gradient(B):
    """The BF16 tensor-core step (tcgen05 forward and backward, FP32 master weights): its gradient
    against the FP64 oracle's.  BF16 keeps 8 significant bits (unit roundoff u = 2^-9 ~ 2e-3); each
    GEMM rounds its operands once and accumulates in FP32, and the error compounds over the three
    forward and three backward GEMMs, so each layer's gradient is held to a relative L2 error of
    3e-2 and the loss to 1e-2.  The labels are structured (visible iff the mean's x > 0, like the
    spatially coherent labels of an occluder): with random labels the class-balanced gradient is a
    near-cancelling sum of +- terms and BF16 rounding of the terms dominates it, whatever the
    kernel.  B = 1000 leaves a ragged last block of 104 samples."""
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.config1_scene(3000)
    cams = [scenes.look_at_camera(3.0 * d, (0, 0, 0), 128, 128, 50.0) for d in scenes.fibonacci_directions(6)]
    rng = np.random.default_rng(1 + B)
    labels = np.tile((sc.assets[0].means[:, 0] > 0).astype(np.uint8), (6, 1))
    sv = rng.integers(0, 6, B).astype(np.int32)
    sg = rng.integers(0, 3000, B).astype(np.int32)
    w = scenes.mlp_weights(3)
    for k in range(1, 5):
        w[f"b{k}"] = rng.normal(0, 0.2, w[f"b{k}"].shape).astype(np.float32)
    w0 = N.flat_weights(w)
    r = renderer_for(sc)
    try:
        N.nvgs_train_init(r.ctx, 0, w0, cams)
        d_lab = torch.from_numpy(labels.ravel()).cuda()
        loss = N.nvgs_train_visibility_step(r.ctx, 0, d_lab, B, 0, 1e6, sample_view=torch.from_numpy(sv).cuda(),
                                            sample_gauss=torch.from_numpy(sg).cuda(), beta1=0.0, beta2=0.0,
                                            eps=1e6, want_loss=True, precision=N.NVGS_PREC_BF16)
        w1 = N.nvgs_train_get_weights(r.ctx, 0).astype(np.float64)
    finally:
        r.close()
    osc = oracle.OracleScene(sc)
    views = oracle.training_views_table(cams)
    ref_loss, g = oracle.train_loss_grad(osc, 0, views, labels, sv, sg, oracle.flat_weights(w))
    step_gpu = w0.astype(np.float64) - w1
    step_ref = g / (1.0 + np.abs(g) / 1e6)
    layers = {"W1": (0, 2048), "b1": (2048, 2112), "W2": (2112, 6208), "b2": (6208, 6272),
              "W3": (6272, 10368), "b3": (10368, 10432), "W4": (10432, 10496), "b4": (10496, 10497)}
    errs = {}
    for name, (a, b) in layers.items():
        ref = step_ref[a:b]
        errs[name] = float(np.linalg.norm(step_gpu[a:b] - ref) / max(np.linalg.norm(ref), 1e-30))
    print(f"bf16 train step B={B}: loss {loss:.6f} vs {ref_loss:.6f}; relative L2 error per layer "
          + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert loss == pytest.approx(ref_loss, rel=1e-2)
    for name, e in errs.items():
        if name != "b4":
            assert e <= 3e-2, (name, e)
    # gb4 = sum of dL/dz: under class balancing the two classes' sums nearly cancel, so its error is
    # bounded against the RMS entry of gW4 (the output layer's gradient scale) instead
    a4, b4_ = layers["W4"]
    rms_w4 = float(np.sqrt(np.mean(step_ref[a4:b4_] ** 2)))
    assert abs(step_gpu[10496] - step_ref[10496]) <= 3e-2 * rms_w4


def test_training_learns_back_face_occlusion():
    """A dense sphere hides its far side: after training on GPU labels, the MLP predicts fresh
    labels of held-out views clearly better than the majority class, and a conservative threshold
    keeps nearly every visible Gaussian while still culling."""
    from paper_2511_19202_b300 import nvgs as N
    from paper_2511_19202_b300.train import train_visibility
    a = scenes.sphere_asset(40000, seed=5, sh_degree=0)
    sc = scenes.Scene([a], [scenes.Instance(0, np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 1.0)])
    r = renderer_for(sc)
    try:
        w, info = train_visibility(r.ctx, 0, n_dirs=96, n_dist=3, res=256, steps=500, batch=32768,
                                   precision=N.NVGS_PREC_BF16, log_every=100)
        print({k: info[k] for k in ("label_s", "total_s", "visible_fraction", "losses")})
        assert info["losses"][-1][1] < 0.7 * info["losses"][0][1]
        dirs = scenes.fibonacci_directions(9)[1::2]
        held = [scenes.look_at_camera(d * dirv, (0, 0, 0), 256, 256, 50.0) for dirv in dirs for d in (8.0, 20.0)]
        n = a.n
        labels = torch.zeros(len(held) * n, dtype=torch.uint8, device="cuda")
        N.nvgs_label_visibility(r.ctx, 0, held, N.nvgs_default_flags(use_mlp=0, tile_size=16), labels)
        lab = labels.cpu().numpy().reshape(len(held), n).astype(bool)
        gain, recall, culled = [], [], []
        for k, cam in enumerate(held):
            lg, kp, _ = r.query_visibility(cam, r.flags(use_mlp=1, mlp_gate=0))
            kp = kp.cpu().numpy().astype(bool)
            lg = lg.cpu().numpy()
            majority = max(lab[k].mean(), 1.0 - lab[k].mean())
            gain.append((kp == lab[k]).mean() - majority)
            keep = lg > -2.0
            recall.append((keep & lab[k]).sum() / max(1, lab[k].sum()))
            culled.append(1.0 - keep.mean())
        print("accuracy over majority", np.round(gain, 3), "recall at -2", np.round(recall, 4),
              "culled at -2", np.round(culled, 3))
        assert np.mean(gain) > 0.05
        assert np.mean(recall) > 0.97 and np.mean(culled) > 0.05
    finally:
        r.close()


def _centre(c):
    R = np.asarray(c.R, np.float64).reshape(3, 3)
    return -R.T @ np.asarray(c.t, np.float64), R


def test_training_views_with_auxiliary_cones_and_offsets():
    """Sec. 3.1 / 4.1 view variants: each main view is followed by n_aux cameras at the same
    distance on the cone of the given half-angle around its direction, looking at the box centre;
    the random offset moves a main camera only in its image plane, not at d_min, and by at most
    sqrt(2) s(d) d with s growing linearly to d_min / d_max at d_max; without variants the main
    views are those of nvgs_training_views."""
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.config1_scene(3000)
    r = renderer_for(sc)
    try:
        info = N.nvgs_get_asset_info(r.ctx, 0)
        bc = np.asarray(info.bbox_center, np.float64)
        dmin, dmax = float(info.d_min), float(info.d_max)
        plain = N.nvgs_training_views(r.ctx, 0, 8, 3, 64, 64)
        same = N.nvgs_training_views_ex(r.ctx, 0, 8, 3, 64, 64)
        for a, b in zip(plain, same):
            assert list(a.R) == list(b.R) and list(a.t) == list(b.t)
        ang = np.radians(2.5)
        ex = N.nvgs_training_views_ex(r.ctx, 0, 8, 3, 64, 64, n_aux=6, aux_angle=ang, random_offset=True, seed=3)
        assert len(ex) == 8 * 3 * 7
        shifted = 0
        for v in range(24):
            main, base = ex[7 * v], plain[v]
            cm, Rm = _centre(main)
            cb, Rb = _centre(base)
            np.testing.assert_allclose(Rm, Rb, atol=1e-6)          # same orientation
            f = Rb[2]
            d = float(np.linalg.norm(cb - bc))
            off = cm - cb
            assert abs(off @ f) < 1e-4 * d                          # in the image plane
            s = (d - dmin) / (dmax - dmin) * dmin / dmax
            assert np.linalg.norm(off) <= np.sqrt(2) * s * d * (1 + 1e-4) + 1e-5
            if v % 3 == 0:
                assert np.linalg.norm(off) < 1e-5 * d               # none at d_min
            else:
                shifted += np.linalg.norm(off) > 1e-3 * s * d
            main_dir = (cb - bc) / d
            for m in range(1, 7):
                ca, Ra = _centre(ex[7 * v + m])
                da = float(np.linalg.norm(ca - bc))
                assert abs(da - d) < 1e-4 * d
                cosang = float(((ca - bc) / da) @ main_dir)
                assert abs(np.arccos(min(1.0, cosang)) - ang) < 1e-4
                np.testing.assert_allclose(Ra[2], -(ca - bc) / da, atol=1e-5)   # looks at the centre
        assert shifted >= 8
    finally:
        r.close()


def test_auxiliary_views_only_add_visible_labels():
    """A Gaussian is visible for a main view if the main view or any of its auxiliary views blends
    it (Sec. 3.1): labels with the cones contain those of the main views alone, and add some."""
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.config1_scene(6000)
    r = renderer_for(sc)
    try:
        n = sc.n_instanced
        allv = N.nvgs_training_views_ex(r.ctx, 0, 6, 2, 128, 128, n_aux=6, aux_angle=np.radians(2.5))
        mains = (N.Camera * 12)(*[allv[k] for k in range(0, len(allv), 7)])
        fl = N.nvgs_default_flags(use_mlp=0)
        lab_main = torch.zeros(12 * n, dtype=torch.uint8, device="cuda")
        N.nvgs_label_visibility(r.ctx, 0, mains, fl, lab_main)
        lab_aux = torch.zeros(12 * n, dtype=torch.uint8, device="cuda")
        N.nvgs_label_visibility(r.ctx, 0, allv, fl, lab_aux, group=7)
        a = lab_main.cpu().numpy().astype(bool)
        b = lab_aux.cpu().numpy().astype(bool)
        assert not (a & ~b).any()
        assert b.sum() > a.sum()
    finally:
        r.close()


def test_training_resumes_bit_for_bit_from_a_checkpoint():
    """Checkpoint / resume: save the training state (master weights, Adam moments) after 20 steps,
    run 20 more; a fresh state loaded from the checkpoint and run over the same 20 steps ends with
    the same weights, bit for bit."""
    from paper_2511_19202_b300 import nvgs as N
    from paper_2511_19202_b300.train import init_weights
    sc = scenes.config1_scene(6000)
    r = renderer_for(sc)
    try:
        views = N.nvgs_training_views(r.ctx, 0, 12, 2, 96, 96)
        n = sc.n_instanced
        labels = torch.zeros(len(views) * n, dtype=torch.uint8, device="cuda")
        N.nvgs_label_visibility(r.ctx, 0, views, N.nvgs_default_flags(use_mlp=0), labels)
        w0 = init_weights(5)

        def run(first, last):
            for step in range(first, last):
                N.nvgs_train_visibility_step(r.ctx, 0, labels, 4096, step, 1e-3, seed=9)

        N.nvgs_train_init(r.ctx, 0, w0, views)
        run(0, 20)
        ckpt = N.nvgs_train_save_state(r.ctx, 0)
        run(20, 40)
        straight = N.nvgs_train_get_weights(r.ctx, 0)
        N.nvgs_train_init(r.ctx, 0, w0, views)          # a fresh state ...
        N.nvgs_train_load_state(r.ctx, 0, ckpt)           # ... resumed from the checkpoint
        run(20, 40)
        resumed = N.nvgs_train_get_weights(r.ctx, 0)
        np.testing.assert_array_equal(N.flat_weights(straight), N.flat_weights(resumed))
        assert not np.array_equal(N.flat_weights(straight), ckpt[:10497])   # it did train
    finally:
        r.close()
