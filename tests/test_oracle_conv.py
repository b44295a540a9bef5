"""Pins of the learned-stage oracle (oracle/conv.py): the convolution against
scipy.signal.correlate2d, the hand-written gradients against central finite
differences, and the loss gradient against its definition."""
import numpy as np
import pytest
import scipy.signal

from oracle import conv as C


def rand_params(rng, chans):
    return [(rng.standard_normal((co, 3, 3, ci)) / np.sqrt(9 * ci), rng.standard_normal(co) * 0.1)
            for ci, co in zip(chans[:-1], chans[1:])]


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = C.conv3x3(x, W, b)
    for bi in range(2):
        for co in range(4):
            ref = b[co] + sum(scipy.signal.correlate2d(x[bi, :, :, ci], W[co, :, :, ci], mode="same")
                              for ci in range(3))
            np.testing.assert_allclose(y[bi, :, :, co], ref, rtol=1e-12, atol=1e-12)


def test_input_and_weight_grads_finite_differences():
    rng = np.random.default_rng(1)
    chans = [3, 5, 4, 2]
    params = rand_params(rng, chans)
    x = rng.standard_normal((2, 6, 5, 3))
    gout = rng.standard_normal((2, 6, 5, 2))
    ys = C.forward(x, params)
    grads, gx = C.backward(ys, params, gout)

    def f(xx, pp):
        return float(np.sum(C.forward(xx, pp)[-1] * gout))

    eps = 1e-6
    for _ in range(6):     # random entries of every tensor
        idx = tuple(rng.integers(0, n) for n in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        assert abs((f(xp, params) - f(xm, params)) / (2 * eps) - gx[idx]) < 1e-6 * max(1, abs(gx[idx]))
    for l in range(len(params)):
        W, b = params[l]
        for _ in range(4):
            idx = tuple(rng.integers(0, n) for n in W.shape)
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += eps
            Wm[idx] -= eps
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            num = (f(x, pp) - f(x, pm)) / (2 * eps)
            assert abs(num - grads[l][0][idx]) < 1e-6 * max(1, abs(num))
        k = rng.integers(0, b.shape[0])
        bp, bm = b.copy(), b.copy()
        bp[k] += eps
        bm[k] -= eps
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        num = (f(x, pp) - f(x, pm)) / (2 * eps)
        assert abs(num - grads[l][1][k]) < 1e-6 * max(1, abs(num))


def test_loss_grad():
    rng = np.random.default_rng(2)
    p, t = rng.standard_normal((3, 4, 4, 2)), rng.standard_normal((3, 4, 4, 2))
    g = C.loss_grad(p, t)
    eps = 1e-7
    idx = (1, 2, 3, 0)
    pp, pm = p.copy(), p.copy()
    pp[idx] += eps
    pm[idx] -= eps
    assert abs((C.loss(pp, t) - C.loss(pm, t)) / (2 * eps) - g[idx]) < 1e-6
    assert C.loss(t, t) == 0.0
