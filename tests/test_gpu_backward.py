"""Gradients of the render (nvgs_render_backward) against FP64 central differences of the oracle
render, for a linear loss L = sum(G * image) with a seeded random cotangent G.

The derivative is piecewise smooth: a parameter whose perturbation moves a fragment across the
1/255 skip, the 0.99 clamp, the stop rule, the support cut-off or a depth swap has no derivative
there.  Such parameters are found on the oracle side alone (the difference quotients at h and 2h
disagree) and left out; all others must match."""
import numpy as np
import pytest

import oracle
import scenes
from gpu_common import renderer_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")
BG = (0.2, 0.1, 0.3)


def fd_grads(sc, cam, G, o, keep=None, h=1e-5, only=None):
    """Central differences of sum(G * oracle image) over every parameter of asset 0 (or the
    Gaussians listed in ``only``); returns (grads, discontinuous)."""
    osc = oracle.OracleScene(sc)
    arrs = osc._keep[0]          # the FP64 arrays the oracle reads, perturbed in place

    def loss():
        return float(np.sum(oracle.render(osc, cam, o, keep=keep)["image"] * G))

    grads, bad = {}, {}
    for name, a in zip(NAMES, arrs):
        g = np.zeros(a.shape)
        b = np.zeros(a.shape, bool)
        rows = range(a.shape[0]) if only is None else only
        for gi in rows:
            for j in np.ndindex(a.shape[1:]):
                idx = (gi,) + j
                x = a[idx]
                d = []
                for hh in (h, 2 * h):
                    a[idx] = x + hh
                    lp = loss()
                    a[idx] = x - hh
                    lm = loss()
                    d.append((lp - lm) / (2 * hh))
                a[idx] = x
                g[idx] = d[0]
                b[idx] = abs(d[0] - d[1]) > 1e-4 * max(1.0, abs(d[0]))
        grads[name], bad[name] = g, b
    return grads, bad


def gpu_grads(r, cam, G, **flags):
    from paper_2511_19202_b300 import nvgs as N
    img, st = r.render(cam, r.flags(keep_outputs=1, **flags))
    a = r._scene.assets[0]
    gr = {n: torch.zeros(np.shape(getattr(a, n)), dtype=torch.float32, device="cuda") for n in NAMES}
    dG = torch.from_numpy(np.ascontiguousarray(G, np.float32)).cuda()
    N.nvgs_render_backward(r.ctx, dG, 0, *(gr[n] for n in NAMES))
    torch.cuda.synchronize()
    return img.cpu().numpy(), st, {n: gr[n].cpu().numpy().astype(np.float64) for n in NAMES}


def compare(gpu, fd, bad, rows=None, rtol=2e-3, max_outliers=0.003, max_bad=0.05):
    report = {}
    for n in NAMES:
        sel = np.zeros(fd[n].shape, bool)
        if rows is None:
            sel[:] = True
        else:
            sel[list(rows)] = True
        ok = sel & ~bad[n]
        assert bad[n][sel].mean() <= max_bad, f"{n}: too many discontinuous parameters"
        g, f = gpu[n][ok], fd[n][ok]
        scale = np.abs(f).max()
        assert scale > 0, f"{n}: no gradient at all"
        err = np.abs(g - f)
        out = (err > rtol * (scale + np.abs(f))).mean()
        rel = np.linalg.norm(g - f) / np.linalg.norm(f)
        report[n] = (round(float(rel), 7), round(float(out), 5), int(bad[n][sel].sum()))
        assert out <= max_outliers and rel <= rtol, (n, rel, out)
    print("relative L2 error, outlier fraction, discontinuous:", report)
    return report


def _renderer(sc, **kw):
    r = renderer_for(sc, **kw)
    r._scene = sc
    return r


def test_backward_matches_oracle_finite_differences():
    from paper_2511_19202_b300 import nvgs as N
    sc = scenes.tiny_scene(64, 7, spread=0.5, log_scale_mean=-2.3, sh_degree=3)
    cam = scenes.look_at_camera((0.4, 0.5, 2.6), (0, 0, 0), 40, 36, 50.0)   # ragged 16-px tiles
    G = np.random.default_rng(1).normal(0, 1, (36, 40, 3))
    r = _renderer(sc)
    try:
        # without kept outputs there is nothing to differentiate
        r.render(cam, r.flags(use_mlp=0))
        with pytest.raises(N.NvgsError):
            N.nvgs_render_backward(r.ctx, torch.zeros(36 * 40 * 3, device="cuda"), 0,
                                   *(torch.zeros(1, device="cuda") for _ in NAMES))
        img, st, gpu = gpu_grads(r, cam, G, use_mlp=0, bg=BG)
    finally:
        r.close()
    o = oracle.opts(bg=BG)
    ref = oracle.render(oracle.OracleScene(sc), cam, o)
    assert np.abs(img - ref["image"])[~ref["ambiguous"]].max() < 1e-4
    fd, bad = fd_grads(sc, cam, G, o)
    compare(gpu, fd, bad)


def test_backward_accumulates_instances_and_skips_culled():
    """Two instances (rotated, scaled) of one asset add their gradients; Gaussians culled by the
    visibility decision receive none (the oracle renders with the same keep mask)."""
    sc = scenes.tiny_scene(40, 11, spread=0.45, log_scale_mean=-2.2, sh_degree=1, n_instances=2)
    cam = scenes.look_at_camera((-0.3, 0.6, 2.4), (0, 0, 0), 33, 31, 55.0)
    G = np.random.default_rng(2).normal(0, 1, (31, 33, 3))
    n = sc.n_instanced
    logits = np.random.default_rng(3).normal(0.5, 1.0, n).astype(np.float32)
    keep = (logits > 0).astype(np.uint8)
    r = _renderer(sc, weights=scenes.mlp_weights(3))
    try:
        d_log = torch.from_numpy(logits).cuda()
        img, st, gpu = gpu_grads(r, cam, G, use_mlp=1, mlp_gate=0, logits_override=d_log, bg=BG)
        assert st["n_survivors"] < st["n_in_frustum"]
    finally:
        r.close()
    o = oracle.opts(bg=BG)
    fd, bad = fd_grads(sc, cam, G, o, keep=keep)
    compare(gpu, fd, bad)
    both_culled = (keep[:40] == 0) & (keep[40:] == 0)
    for nme in NAMES:
        assert np.all(gpu[nme][both_culled] == 0.0)


def test_split_compositing_backward_matches_one_pass():
    """A dense frame whose tiles are long enough for the chunked compositing: the kept last-fragment
    indices and transmittances it leaves give the same gradients as the one-CTA-per-tile pass."""
    sc = scenes.tiny_scene(3000, 5, spread=0.4, log_scale_mean=-2.8, sh_degree=2)
    a = sc.assets[0]
    a.opacity_logits = (a.opacity_logits - 3.5).astype(np.float32)   # faint: pixels stay unsaturated
    cam = scenes.look_at_camera((0.2, 0.3, 2.2), (0, 0, 0), 48, 40, 50.0)
    G = np.random.default_rng(4).normal(0, 1, (40, 48, 3))
    r = _renderer(sc)
    try:
        _, st1, g1 = gpu_grads(r, cam, G, use_mlp=0, blend_split_len=-1)
        _, st2, g2 = gpu_grads(r, cam, G, use_mlp=0, blend_split_len=256)
    finally:
        r.close()
    assert st1["n_pairs"] > 2 * 9 * 256   # 3 x 3 tiles, over twice the chunk length on average
    for nme in NAMES:
        scale = np.abs(g1[nme]).max()
        assert np.abs(g1[nme] - g2[nme]).max() <= 1e-3 * scale, nme


def test_autograd_fits_a_target_image():
    """torch.autograd through the library: Adam on the asset's parameters brings a perturbed asset
    closer to the image of the original; uploading the original parameters back reproduces the
    original render bit for bit."""
    from paper_2511_19202_b300.autograd import PARAM_NAMES, render_asset
    sc = scenes.tiny_scene(200, 9, spread=0.5, log_scale_mean=-2.6, sh_degree=1)
    cam = scenes.look_at_camera((0.0, 0.4, 2.5), (0, 0, 0), 64, 64, 50.0)
    a = sc.assets[0]
    r = _renderer(sc)
    try:
        fl = r.flags(use_mlp=0)
        target, _ = r.render(cam, fl)
        target = target.clone()
        orig = {k: torch.from_numpy(np.ascontiguousarray(getattr(a, k), np.float32)).cuda() for k in PARAM_NAMES}
        g = torch.Generator(device="cuda").manual_seed(0)
        params = {k: (v + 0.05 * torch.randn(v.shape, device="cuda", generator=g)).requires_grad_(True)
                  for k, v in orig.items()}
        opt = torch.optim.Adam(params.values(), lr=2e-3)
        losses = []
        for _ in range(120):
            opt.zero_grad()
            img = render_asset(r, 0, params, cam, r.flags(use_mlp=0))
            loss = ((img - target) ** 2).mean()
            loss.backward()
            opt.step()
            losses.append(float(loss.detach()))
        print("losses", [round(x, 6) for x in losses[::20]], losses[-1])
        assert losses[-1] < 0.5 * losses[0]
        with torch.no_grad():
            back = render_asset(r, 0, orig, cam, r.flags(use_mlp=0))
        assert torch.equal(back, target)
    finally:
        r.close()
