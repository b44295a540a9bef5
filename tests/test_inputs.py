"""The seeded input recipe (paper_1607_00968_gb300/inputs.py) has the
properties the workloads are defined by: node shapes, seeded determinism,
the 1.5-4.5 km/s velocity range with a 4.5 km/s salt body, the quadratic
absorbing-layer ramp that is 1 at the outermost node and absent at the free
surface, unit point sources as finite-volume deltas, and the frequency rule of
ten points per wavelength at the lowest velocity.
"""
import math

import numpy as np
import pytest

from paper_1607_00968_gb300 import inputs as I


def test_node_shape_and_frequency_rule():
    assert I.node_shape((128, 64)) == (65, 129)
    assert I.node_shape((128, 128, 64)) == (65, 129, 129)
    w = I.omega_for_ppw(25.0)
    # wavelength 2 pi v / w at v_min spans 10 cells
    assert math.isclose(2 * math.pi * I.V_MIN / w / 25.0, 10.0, rel_tol=1e-14)


@pytest.mark.parametrize("make", [lambda: I.salt2d_problem(seed=3, freq_hz=5.0),
                                  lambda: I.layered2d_problem(seed=3)])
def test_seeded_models_are_deterministic_and_in_range(make):
    a, b = make(), make()
    np.testing.assert_array_equal(a.m, b.m)
    np.testing.assert_array_equal(a.gamma, b.gamma)
    v = 1.0 / np.sqrt(a.m)
    assert v.min() >= I.V_MIN * (1 - 1e-12) and v.max() <= I.V_MAX * (1 + 1e-12)
    assert a.m.shape == I.node_shape(a.cells)


def test_salt_model_has_the_salt_body_and_differs_by_seed():
    P = I.salt2d_problem(seed=0)
    v = 1.0 / np.sqrt(P.m)
    assert np.mean(np.isclose(v, I.V_MAX)) > 0.005          # a 4.5 km/s body of some extent
    Q = I.salt2d_problem(seed=1)
    assert not np.array_equal(P.m, Q.m)


@pytest.mark.parametrize("shape,width", [((65, 129), 10), ((33, 41, 57), 6)])
def test_absorbing_layer_profile(shape, width):
    g = I.absorbing_gamma(shape, width)
    assert g.shape == shape
    # interior (away from every side but the top) is unattenuated
    inner = tuple(slice(0 if ax == 0 else width, n - width) for ax, n in enumerate(shape))
    assert np.all(g[inner] == 0.0)
    # the outermost node of every side but the top has gamma 1; the top row none from the depth axis
    assert np.all(g[-1] == 1.0)
    for ax in range(1, len(shape)):
        assert np.all(np.take(g, 0, axis=ax) == 1.0)
        assert np.all(np.take(g, shape[ax] - 1, axis=ax) == 1.0)
    # quadratic ramp along the bottom edge of the depth axis, mid-domain laterally
    mid = tuple(n // 2 for n in shape[1:])
    col = g[(slice(None),) + mid]
    for d in range(width):
        assert math.isclose(col[shape[0] - 1 - d], ((width - d) / width) ** 2, rel_tol=1e-15)
    assert 0.0 <= g.min() and g.max() == 1.0


def test_point_sources_are_finite_volume_deltas():
    shape, h = (17, 33), 12.5
    pos = I.line_positions(shape, 5, 0, 4)
    Q = I.point_sources(shape, pos, h)
    assert Q.shape == (5, shape[0] * shape[1])
    for k, p in enumerate(pos):
        col = Q[k].reshape(shape)
        assert np.count_nonzero(col) == 1
        assert col[tuple(p)] == pytest.approx(1.0 / h ** 2)
        assert p[0] == 0 and 4 <= p[1] <= shape[1] - 1 - 4       # on the row, outside the layer
    P = I.layered3d_problem(seed=0)
    assert len(P.sources) == 256 and len(set(map(tuple, P.sources))) == 256
    assert all(p[0] == 0 for p in P.sources)                  # on the surface row
