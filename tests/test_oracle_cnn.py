"""Pins of the CNN oracle: the convolution against scipy's 2D
cross-correlation, the analytic gradients against central finite
differences, the residual structure (a zero last layer is the identity)."""
import numpy as np
import pytest

from oracle import cnn

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv_equals_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 9, 11))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    out = cnn.conv3x3(x, w, b)
    for n in range(2):
        for co in range(4):
            ref = sum(scipy_signal.correlate2d(x[n, ci], w[co, ci], mode="same", boundary="fill")
                      for ci in range(3)) + b[co]
            np.testing.assert_allclose(out[n, co], ref, rtol=0, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    # the same five-layer structure, 4 channels wide (the brute force stays small)
    shapes = [(4, 1), (4, 4), (4, 4), (4, 4), (1, 4)]
    params = [(rng.standard_normal((co, ci, 3, 3)) * 0.7, rng.standard_normal(co) * 0.1) for co, ci in shapes]
    x = rng.uniform(0, 1, (2, 6, 7))
    t = x + 0.05 * rng.standard_normal(x.shape)
    _, grads = cnn.backward(params, x, t)
    eps = 1e-6
    for k, (w, b) in enumerate(params):
        for idx in [(0, 0, 1, 1), tuple(s - 1 for s in w.shape), (w.shape[0] // 2, 0, 2, 0)]:
            wp = [(ww.copy(), bb.copy()) for ww, bb in params]
            wm = [(ww.copy(), bb.copy()) for ww, bb in params]
            wp[k][0][idx] += eps
            wm[k][0][idx] -= eps
            fd = (cnn.loss(wp, x, t) - cnn.loss(wm, x, t)) / (2 * eps)
            assert grads[k][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-10), (k, idx)
        bp = [(ww.copy(), bb.copy()) for ww, bb in params]
        bm = [(ww.copy(), bb.copy()) for ww, bb in params]
        bp[k][1][0] += eps
        bm[k][1][0] -= eps
        fd = (cnn.loss(bp, x, t) - cnn.loss(bm, x, t)) / (2 * eps)
        assert grads[k][1][0] == pytest.approx(fd, rel=1e-5, abs=1e-10), k


def test_zero_last_layer_is_identity():
    rng = np.random.default_rng(2)
    params = cnn.init_params(4)
    params[-1] = (np.zeros_like(params[-1][0]), np.zeros(1))
    x = rng.uniform(0, 1, (1, 8, 8))
    y, _ = cnn.forward(params, x)
    np.testing.assert_array_equal(y, x)


def test_psnr_closed_form():
    a = np.zeros((4, 4))
    assert cnn.psnr(a, a + 1.0) == pytest.approx(10 * np.log10(255.0 ** 2))
