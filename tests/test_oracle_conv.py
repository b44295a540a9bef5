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


# --------------------------------------------------------------------------
# residual loss of the corrected iterate
# --------------------------------------------------------------------------

def _resid_case(seed=5, B=2, H=7, W=9):
    rng = np.random.default_rng(seed)
    pred = rng.standard_normal((B, H, W, 4))
    r = rng.standard_normal((B, H, W)) + 1j * rng.standard_normal((B, H, W))
    kappa = rng.uniform(0.1, 0.6, (B, H, W))
    gam = rng.uniform(0.0, 0.8, (B, H, W))
    return pred, r, kappa * (1 - 1j * gam), kappa, gam


def test_image_operator_is_h2_times_helmholtz_matrix():
    """K e on the image equals h^2 A e with A the operator oracle's sparse
    Helmholtz matrix (node i W + j = pixel (i, j)), for m and gamma chosen so
    that coef = h^2 omega^2 m (1 - i gamma)."""
    from oracle import helmholtz as HO
    _, r, coef, kappa, gam = _resid_case(B=1)
    h, omega = 12.5, 2.0
    m = kappa[0] / (h * h * omega * omega)
    A = HO.helmholtz_matrix(m, gam[0], omega, h)
    got = C.h2A_image(r, coef)[0].ravel()
    np.testing.assert_allclose(got, h * h * (A @ r[0].ravel()), rtol=1e-12, atol=1e-12)
    AH = A.conj().T
    np.testing.assert_allclose(C.h2A_image(r, coef, adjoint=True)[0].ravel(),
                               h * h * (AH @ r[0].ravel()), rtol=1e-12, atol=1e-12)


def test_residual_loss_zero_at_exact_inverse_and_one_at_zero():
    """pred = K^{-1} r (dense solve) leaves no residual; pred = 0 leaves all."""
    _, r, coef, _, _ = _resid_case(B=1, H=5, W=6)
    n = 30
    K = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        K[:, k] = C.h2A_image(e.reshape(1, 5, 6), coef).ravel()
    e = np.linalg.solve(K, r.ravel()).reshape(1, 5, 6)
    pred = np.stack([e.real, e.imag], axis=-1)
    assert C.residual_loss(pred, r, coef) < 1e-24
    assert abs(C.residual_loss(np.zeros_like(pred), r, coef) - 1.0) < 1e-14


def test_residual_loss_gradient_finite_differences():
    pred, r, coef, _, _ = _resid_case()
    g = C.residual_loss_grad(pred, r, coef)
    rng = np.random.default_rng(6)
    for _ in range(12):
        b, i, j, c = rng.integers(0, 2), rng.integers(0, 7), rng.integers(0, 9), rng.integers(0, 4)
        eps = 1e-6
        pp, pm = pred.copy(), pred.copy()
        pp[b, i, j, c] += eps
        pm[b, i, j, c] -= eps
        fd = (C.residual_loss(pp, r, coef) - C.residual_loss(pm, r, coef)) / (2 * eps)
        assert abs(fd - g[b, i, j, c]) <= 1e-6 * max(1.0, abs(fd)), (b, i, j, c, fd, g[b, i, j, c])
