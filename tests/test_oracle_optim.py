"""Pins of the oracle's training pieces (oracle/optim.py): Adam under a constant gradient has
the closed form raw_T = raw_0 - T lr g / (|g| + eps) (the bias-corrected moments are g and g^2
exactly); the activations' chain rule against finite differences; the L1 loss on a hand-made
example and its gradient against finite differences."""
import numpy as np

from oracle import optim


def test_adam_constant_gradient_closed_form():
    rng = np.random.default_rng(0)
    raw0 = rng.normal(size=50)
    g = rng.normal(size=50)
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    raw, m, v = raw0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 41):
        raw, act, m, v = optim.adam_step(raw, g, m, v, optim.ACT_NONE, lr, b1, b2, eps, t)
        want = raw0 - t * lr * g / (np.abs(g) + eps)
        assert np.allclose(raw, want, rtol=0, atol=1e-12)


def test_activation_chain_matches_finite_differences():
    rng = np.random.default_rng(1)
    raw = rng.normal(size=20)
    ga = rng.normal(size=20)
    for act in (optim.ACT_EXP, optim.ACT_SIGMOID):
        # the first step's raw gradient, read back from m = (1 - beta1) g
        _, _, m, _ = optim.adam_step(raw, ga, np.zeros(20), np.zeros(20), act, 0.0, 0.5, 0.5, 1.0, 1)
        g_raw = m / 0.5
        h = 1e-6
        fd = ga * (optim.activate(raw + h, act) - optim.activate(raw - h, act)) / (2 * h)
        assert np.allclose(g_raw, fd, rtol=1e-7, atol=1e-10)


def test_l1_loss_example_and_gradient():
    img = np.array([0.2, 0.5, 0.9, 0.3])
    tgt = np.array([0.1, 0.5, 1.0, 0.0])
    L, g = optim.loss_l1(img, tgt, 0.5)
    assert abs(L - 0.5 * (0.1 + 0.0 + 0.1 + 0.3)) < 1e-15
    h = 1e-7
    for i in (0, 2, 3):
        e = np.zeros(4)
        e[i] = h
        fd = (optim.loss_l1(img + e, tgt, 0.5)[0] - optim.loss_l1(img - e, tgt, 0.5)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6
    assert g[1] == 0.0
