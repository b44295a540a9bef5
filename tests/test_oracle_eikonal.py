"""Pins of the factored-eikonal oracle (oracle/eikonal.py) to facts the
paper and the mathematics fix (Sec. 2.5):

* constant slowness: the factored equation is solved exactly by
  tau1 = sqrt(m) (|p0| = 1), so fast marching must return it to rounding;
* constant velocity gradient v = v0 + g z: the analytic first-arrival time
  (1/g) arccosh(1 + g^2 r^2 / (2 v(z_s) v(z))) is approached at first order
  as h halves;
* every node's final value satisfies its Godunov equation with the
  derivatives fast marching chose, and those neighbours were accepted before
  it (the triangular structure the sensitivity relies on);
* J v matches central finite differences of fast marching, agrees with a
  dense solve of Eq. Sensitivity2, and <J v, w> = <v, J^T w>.
"""
import math

import numpy as np
import pytest

from oracle import eikonal as E


def smooth_velocity(shape, seed):
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.linspace(0, 1, n) for n in shape], indexing="ij")
    v = 2000.0 + 1500.0 * grids[0]
    for _ in range(3):
        c = rng.uniform(0, 1, len(shape))
        r2 = sum((grids[a] - c[a]) ** 2 for a in range(len(shape)))
        v = v + rng.uniform(-400, 400) * np.exp(-r2 / 0.05)
    return v


@pytest.mark.parametrize("shape,src", [((17, 25), (0, 12)), ((9, 11, 13), (4, 0, 6)), ((12, 12), (11, 11))])
def test_constant_slowness_is_exact(shape, src):
    m = np.full(shape, 1.0 / 2500.0 ** 2)
    fm = E.fast_marching(m, 12.5, src)
    np.testing.assert_allclose(fm["tau1"], math.sqrt(m.flat[0]), rtol=1e-13)
    t0, _ = E.tau0_p0(shape, 12.5, src)
    np.testing.assert_allclose(fm["tau"], t0.reshape(-1) / 2500.0, rtol=1e-13, atol=1e-18)
    assert len(fm["order"]) == m.size


def test_constant_gradient_converges_first_order():
    L, v0, g = 1600.0, 1500.0, 0.8            # 1.6 km square, v = 1500 + 0.8 z m/s
    errs = []
    for n in (32, 64):
        h = L / n
        z = np.arange(n + 1) * h
        v = np.repeat((v0 + g * z)[:, None], n + 1, axis=1)
        src = (n // 4, n // 2)
        fm = E.fast_marching(1.0 / v ** 2, h, src)
        zz, xx = np.meshgrid(z, np.arange(n + 1) * h, indexing="ij")
        r2 = (zz - z[src[0]]) ** 2 + (xx - xx[0, src[1]]) ** 2
        exact = np.arccosh(1.0 + g * g * r2 / (2.0 * (v0 + g * z[src[0]]) * (v0 + g * zz))) / g
        errs.append(np.max(np.abs(fm["tau"].reshape(n + 1, n + 1) - exact)))
    assert errs[1] < 0.62 * errs[0], errs
    assert errs[1] < 2e-3                    # seconds, over ~1 s travel times


@pytest.mark.parametrize("shape,src", [((17, 25), (3, 7)), ((7, 9, 8), (0, 4, 3))])
def test_godunov_equation_and_causality(shape, src):
    v = smooth_velocity(shape, 1)
    m = 1.0 / v ** 2
    h = 10.0
    fm = E.fast_marching(m, h, src)
    d = len(shape)
    strides = [int(np.prod(shape[a + 1:])) for a in range(d)]
    pos = np.empty(m.size, dtype=np.int64)
    pos[fm["order"]] = np.arange(m.size)
    t0, p0, t1 = fm["t0"], fm["p0"], fm["tau1"]
    for i in range(m.size):
        dv = int(fm["dir"][i])
        if dv == 0xFF:
            assert math.isclose(t1[i] ** 2, m.flat[i], rel_tol=1e-14)
            continue
        lhs = 0.0
        for a in range(d):
            c = (dv >> (2 * a)) & 3
            if c == 0:
                continue
            nb = i + (-1 if c == 1 else 1) * strides[a]
            assert pos[nb] < pos[i]                           # chosen neighbour known first
            if c == 1:
                f = t0[i] * (t1[i] - t1[nb]) / h + p0[a][i] * t1[i]
            else:
                f = -(t0[i] * (t1[nb] - t1[i]) / h + p0[a][i] * t1[i])
            assert f >= -1e-12 * abs(t1[i])
            lhs += f * f
        assert lhs > 0.0
        assert math.isclose(lhs, m.flat[i], rel_tol=1e-10), (i, lhs, m.flat[i])
    # levels: one more than the deepest chosen neighbour
    assert fm["level"][fm["src"]] == 0 and fm["level"].max() > 0


@pytest.mark.parametrize("shape,src", [((17, 25), (3, 7)), ((6, 7, 9), (2, 0, 4))])
def test_sensitivity_matches_finite_differences_and_adjoint(shape, src):
    v = smooth_velocity(shape, 2)
    m = 1.0 / v ** 2
    h = 10.0
    fm = E.fast_marching(m, h, src)
    rng = np.random.default_rng(5)
    vv = rng.standard_normal(m.size)
    z = E.sens_jv(fm, vv)
    eps = 1e-12                                           # relative perturbation ~1e-5
    fp = E.fast_marching(m + eps * vv.reshape(shape), h, src)["tau1"]
    fmn = E.fast_marching(m - eps * vv.reshape(shape), h, src)["tau1"]
    fd = (fp - fmn) / (2 * eps)
    assert np.linalg.norm(fd - z) <= 1e-6 * np.linalg.norm(z)
    M = E.sens_matrix(fm)
    assert np.linalg.norm(np.linalg.solve(M, vv) - z) <= 1e-12 * np.linalg.norm(z)
    P = fm["order"]
    assert np.all(np.triu(M[np.ix_(P, P)], 1) == 0.0)     # lower triangular in FM order
    w = rng.standard_normal(m.size)
    y = E.sens_jtw(fm, w)
    assert math.isclose(np.dot(z, w), np.dot(vv, y), rel_tol=1e-12)
    assert np.linalg.norm(np.linalg.solve(M.T, w) - y) <= 1e-12 * np.linalg.norm(y)
