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
    weights and the ReLU'd hidden activations rounded to BF16; the hidden biases as BF16 high +
    low pairs; the output layer in FP32 (w4, b4) on the BF16-rounded third-layer activations.
    Only the accumulation order and precision differ from the kernel."""
    def pair(v):
        v = np.ascontiguousarray(v, np.float32)
        hi = bf16_round(v)
        return hi + bf16_round(v - hi.astype(np.float32))
    h = bf16_round(np.asarray(feats, np.float64).astype(np.float32))
    for k in (1, 2, 3):
        a = h @ bf16_round(w[f"W{k}"]).T + pair(w[f"b{k}"])
        h = bf16_round(np.maximum(a, 0.0).astype(np.float32))
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
