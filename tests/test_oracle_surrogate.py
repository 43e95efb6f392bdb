"""Pins of the FP64 surrogate-network oracle: the convolution against
scipy's independent correlation routine, pooling/upsampling adjoints, and the
analytic gradient of the whole network against central finite differences."""
import numpy as np
import pytest

from oracle import surrogate as S

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 9, 3))
    W = rng.normal(size=(3, 3, 3, 4))
    b = rng.normal(size=4)
    y = S.conv3x3(x, W, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy_signal.correlate2d(x[n, :, :, i], W[:, :, i, o], mode="same",
                                                      boundary="fill") for i in range(3))
            assert np.abs(y[n, :, :, o] - ref).max() < 1e-12


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 6, 5, 3))
    W = rng.normal(size=(3, 3, 3, 2))
    g = rng.normal(size=(2, 6, 5, 2))
    gx, gW, gb = S.conv3x3_backward(x, W, g)
    # <conv(x), g> is linear in x and in W: its derivatives are gx and gW
    f = lambda xx, WW: np.sum(S.conv3x3(xx, WW, np.zeros(2)) * g)
    dx = rng.normal(size=x.shape)
    dW = rng.normal(size=W.shape)
    assert abs(f(dx, W) - np.sum(gx * dx)) < 1e-10
    assert abs(f(x, dW) - np.sum(gW * dW)) < 1e-10
    assert np.allclose(gb, g.sum(axis=(0, 1, 2)))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 8, 6, 3))
    g = rng.normal(size=(2, 4, 3, 3))
    assert abs(np.sum(S.avgpool2(x) * g) - np.sum(x * S.avgpool2_backward(g))) < 1e-12
    u = rng.normal(size=(2, 4, 3, 3))
    gu = rng.normal(size=(2, 8, 6, 3))
    assert abs(np.sum(S.upsample2(u) * gu) - np.sum(u * S.upsample2_backward(gu))) < 1e-12


def test_network_gradient_matches_central_differences():
    widths = (4, 6, 8)
    rng = np.random.default_rng(3)
    P = S.init_params(widths, 2, 3, seed=5)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.normal(0, 0.1, P[k].shape)
    x = rng.normal(size=(2, 8, 8, 2))
    t = rng.normal(size=(2, 8, 8, 3))
    loss, G = S.loss_and_grad(P, x, t, widths)
    eps = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = S.forward(P, x, widths)
            flat[idx] = old - eps
            lm, _ = S.forward(P, x, widths)
            flat[idx] = old
            fd = (np.mean((lp - t) ** 2) - np.mean((lm - t) ** 2)) / (2 * eps)
            an = G[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, idx, fd, an)


def test_adam_first_step_moves_each_parameter_by_lr():
    P = {"a": np.array([1.0, -2.0, 3.0])}
    G = {"a": np.array([0.5, -1e-3, 0.0])}
    M = {"a": np.zeros(3)}
    V = {"a": np.zeros(3)}
    S.adam(P, G, M, V, 1, lr=0.01)
    # bias-corrected first step is lr * sign(g) (to within eps)
    assert np.allclose(P["a"], [0.99, -1.99, 3.0], atol=1e-7)
