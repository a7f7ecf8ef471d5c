"""Pins of the oracle's MLP training step (Sec. 3.2, 4.1): the analytic gradient against central
finite differences of the loss, the class balancing of the loss, and the closed form of the first
Adam step."""
import math

import numpy as np
import pytest

import oracle
import scenes


@pytest.fixture(scope="module")
def setup():
    sc = scenes.config1_scene(3000)
    osc = oracle.OracleScene(sc)
    cams = [scenes.look_at_camera(3.0 * d, (0, 0, 0), 128, 128, 50.0)
            for d in scenes.fibonacci_directions(6)]
    views = oracle.training_views_table(cams)
    rng = np.random.default_rng(0)
    labels = (rng.random((6, 3000)) < 0.4).astype(np.uint8)
    B = 96
    sv = rng.integers(0, 6, B).astype(np.int32)
    sg = rng.integers(0, 3000, B).astype(np.int32)
    w = scenes.mlp_weights(3)
    for k in range(1, 5):
        w[f"b{k}"] = rng.normal(0, 0.2, w[f"b{k}"].shape).astype(np.float32)
    return osc, views, labels, sv, sg, oracle.flat_weights(w)


def test_gradient_matches_finite_differences(setup):
    osc, views, labels, sv, sg, w = setup
    loss, g = oracle.train_loss_grad(osc, 0, views, labels, sv, sg, w)
    rng = np.random.default_rng(1)
    # a sample of weights from every layer, biases included
    idx = np.concatenate([rng.integers(0, 2048, 12), rng.integers(2048, 2112, 4),
                          rng.integers(2112, 6208, 12), rng.integers(6272, 10368, 12),
                          rng.integers(10432, 10496, 6), [10496]])
    for i in idx:
        h = 1e-6 * max(1.0, abs(w[i]))
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (oracle.train_loss_grad(osc, 0, views, labels, sv, sg, wp)[0] -
              oracle.train_loss_grad(osc, 0, views, labels, sv, sg, wm)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i


def test_class_balanced_loss(setup):
    """With all logits at 0 (zero output layer), every sample's BCE is ln 2 and the class weights
    B/(2 N_c) sum to B, so the balanced mean loss is exactly ln 2."""
    osc, views, labels, sv, sg, w = setup
    w0 = w.copy()
    w0[10432:] = 0.0            # W4 and b4
    loss, g = oracle.train_loss_grad(osc, 0, views, labels, sv, sg, w0)
    assert loss == pytest.approx(math.log(2.0), rel=1e-14)
    # dL/db4 = sum_k w_k (1/2 - y_k) / B = (N_neg w_neg - N_pos w_pos) / (2B) = 0
    assert g[10496] == pytest.approx(0.0, abs=1e-15)


def test_first_adam_step_closed_form(setup):
    osc, views, labels, sv, sg, w = setup
    _, g = oracle.train_loss_grad(osc, 0, views, labels, sv, sg, w)
    w1, m, v = w.copy(), np.zeros(10497), np.zeros(10497)
    lr, eps = 1e-3, 1e-8
    oracle.train_step(osc, 0, views, labels, sv, sg, w1, m, v, lr, 0.9, 0.999, eps, 0)
    # bias-corrected first moments are g and g^2: the step is lr g / (|g| + eps)
    np.testing.assert_allclose(w1 - w, -lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)
