"""Shared helpers of the GPU parity tests: build the library, run the CUDA path through the
C ABI, and compare with the FP64 oracle on the same seeded inputs."""
import numpy as np

import oracle
import scenes


def renderer_for(scene, weights=None, precision=0, **kw):
    from paper_2511_19202_b300 import build
    build.build()
    from paper_2511_19202_b300.render import Renderer
    r = Renderer(0)
    r.load_scene(scene, weights, precision, **kw)
    return r


def gpu_image(r, cam, **flags):
    img, st = r.render(cam, r.flags(**flags))
    return img.cpu().numpy().astype(np.float64), st


def oracle_opts_for(flags: dict, **eps):
    return oracle.opts(alpha_min=flags.get("alpha_min", 1 / 255), alpha_max=flags.get("alpha_max", 0.99),
                       t_stop=flags.get("t_stop", 1e-4), bg=flags.get("bg", (0, 0, 0)),
                       tile_size=flags.get("tile_size", 16),
                       radius_clip_area=flags.get("radius_clip_area", 0.0), **eps)


def compare_images(gpu, ora, amb, tol=1e-3, max_amb_frac=0.02):
    """Max-abs error over pixels outside the ambiguity band; returns (err, n_ambiguous)."""
    ok = ~amb
    err = float(np.max(np.abs(gpu[ok] - ora[ok]))) if ok.any() else 0.0
    frac = float(amb.mean())
    assert frac <= max_amb_frac, f"ambiguous fraction {frac:.4f} too large"
    assert err <= tol, f"max abs error {err:.3e} > {tol}"
    return err, int(amb.sum())


def survivors_set(lf):
    s = lf["survivors"].cpu().numpy()
    return s


def check_pruned_tile_lists(gpu_tiles, gpu_inst, gpu_g, support, rect, depth_of, drop, eps=1e-6):
    """Per tile, with the ambiguous splats in ``drop`` removed: the oracle's support list (tiles
    holding a pixel the splat reaches at alpha >= 1/255) is contained in the GPU list, which is
    contained in the rect list, and the GPU order is non-decreasing in the oracle's FP64 depth
    except within ``eps`` (relative).  Returns (GPU pairs, support pairs, rect pairs)."""
    def split(t, i, g):
        d = {}
        for a, b, c in zip(t.tolist(), i.tolist(), g.tolist()):
            if (b, c) in drop:
                continue
            d.setdefault(a, []).append((b, c))
        return d
    G, S, R = split(gpu_tiles, gpu_inst, gpu_g), split(*support), split(*rect)
    for t, lst in S.items():
        assert set(lst) <= set(G.get(t, [])), f"tile {t}: a reachable Gaussian is missing"
    for t, lst in G.items():
        assert len(set(lst)) == len(lst), f"tile {t}: duplicate pair"
        assert set(lst) <= set(R.get(t, [])), f"tile {t}: a Gaussian outside its rectangle"
        ds = [depth_of[e] for e in lst]
        for k in range(len(ds) - 1):
            assert ds[k + 1] >= ds[k] - eps * abs(ds[k]), f"tile {t}: order broken at {k}"
    count = lambda d: sum(len(v) for v in d.values())
    return count(G), count(S), count(R)


def check_exact_tile_lists(gpu_tiles, gpu_inst, gpu_g, gpu_depth, ell, depth_of, drop, eps=4e-7):
    """Exact tile-list parity against the oracle's FP64 ellipse lists ``ell`` = (tiles, instances,
    gaussians, ambiguous).  Splats in ``drop`` (ambiguous for another reason: frustum plane,
    support-box edge, ...) and the oracle's band pairs are left out of both sides; the rest must
    be equal per tile, element for element and in order, where two neighbours may only trade places
    if their FP64 depths lie within ``eps`` (relative) of each other.  Among equal FP32 depths
    (``gpu_depth``, the GPU's sort key) the GPU order must be (instance, gaussian) ascending.
    Returns (compared pairs, band pairs, dropped pairs)."""
    et, ei, eg, ea = ell
    band = set(zip(et[ea].tolist(), ei[ea].tolist(), eg[ea].tolist()))

    def lists(t, i, g, extra=None):
        d = {}
        for k, (a, b, c) in enumerate(zip(t.tolist(), i.tolist(), g.tolist())):
            if (b, c) in drop or (a, b, c) in band:
                continue
            d.setdefault(a, []).append((b, c) if extra is None else (b, c, extra[k]))
        return d
    G = lists(gpu_tiles, gpu_inst, gpu_g, gpu_depth.tolist())
    O = lists(et, ei, eg)
    assert set(G) == set(O), f"tiles differ: {sorted(set(G) ^ set(O))[:10]}"
    n = 0
    for t in O:
        g_seq = [(b, c) for b, c, _ in G[t]]
        o_seq = O[t]
        assert len(set(g_seq)) == len(g_seq), f"tile {t}: duplicate pair"
        assert sorted(g_seq) == sorted(o_seq), (f"tile {t}: {len(set(g_seq) - set(o_seq))} extra, "
                                               f"{len(set(o_seq) - set(g_seq))} missing")
        for k, (x, y) in enumerate(zip(g_seq, o_seq)):
            if x != y:
                dx, dy = depth_of[x], depth_of[y]
                assert abs(dx - dy) <= eps * max(abs(dx), abs(dy)), f"tile {t}: order differs at {k}"
        for (b0, c0, z0), (b1, c1, z1) in zip(G[t][:-1], G[t][1:]):
            if z0 == z1:
                assert (b0, c0) < (b1, c1), f"tile {t}: equal depths out of (instance, gaussian) order"
        n += len(o_seq)
    n_drop = sum(1 for b, c in zip(ei.tolist(), eg.tolist()) if (b, c) in drop)
    return n, len(band), n_drop


def bf16_round(x):
    """Round to nearest even to BF16 (as the kernel's cvt.rn and its weight packing do), as FP64."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def bf16_reference(w, feats):
    """The BF16 tensor-core MLP's quantised arithmetic with exact accumulation: FP32 inputs,
    weights and the ReLU'd activations that feed a tensor-core layer rounded to BF16; the hidden
    biases as BF16 high + low pairs; the output layer in FP32 (w4, b4) on the third layer's FP32
    ReLU activations.  Only the accumulation order and precision differ from the kernel."""
    def pair(v):
        v = np.ascontiguousarray(v, np.float32)
        hi = bf16_round(v)
        return hi + bf16_round(v - hi.astype(np.float32))
    h = bf16_round(np.asarray(feats, np.float64).astype(np.float32))
    for k in (1, 2, 3):
        a = h @ bf16_round(w[f"W{k}"]).T + pair(w[f"b{k}"])
        h = np.maximum(a, 0.0)
        if k < 3:
            h = bf16_round(h.astype(np.float32))
    return h @ np.ravel(w["W4"]).astype(np.float32).astype(np.float64) + float(np.float32(np.ravel(w["b4"])[0]))


# BF16 decisions are compared outside a band of 1 % of the logit scale (p99 |logit|): inside it,
# one BF16 rounding of an input or activation that falls the other way (FP32 features and FP32
# accumulation on the GPU) can move the logit by a few 1e-3 of the scale.
BF16_DECISION_BAND = 1e-2


def layered_case(width=320, height=240, n=20000):
    """Three instances of the workload-1 torus in separate distance ranges, with weights whose
    logit is 10 x (cut - normalised log distance) plus small random terms through every layer:
    trained-like, bimodal decisions (the nearest instance kept, the others culled) with the cut
    placed by the oracle's FP64 features in the middle of the gap between the first two ranges."""
    sc, cam = scenes.layered_scene(n), scenes.layered_camera(width, height)
    dist = dict(d_min=1.0, d_max=20.0)
    osc = oracle.OracleScene(sc, **dist)
    inside, _ = oracle.frustum(osc, cam)
    u = np.zeros(32)
    u[30] = -1.0
    f = oracle.visibility(osc, cam, scenes.planar_mlp_weights(3, direction=u), gate=False,
                          return_features=True)["features"][:, 30]
    m = sc.assets[0].n
    near, mid = f[:m][inside[:m]], f[m:2 * m][inside[m:2 * m]]
    cut = 0.5 * (near.max() + mid.min())
    w = scenes.planar_mlp_weights(3, direction=u, offset=10.0 * cut)
    return sc, cam, dist, osc, inside, w


# ----------------------------------------------------------------------------- FP8 (E4M3) MLP
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
