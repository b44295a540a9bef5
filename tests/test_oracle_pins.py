"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself:
the Fourier symbol printed in Sec. 3 (high-order regularisation paragraph),
closed forms derived by hand, library routines, invariants and brute force on
tiny inputs.  No GPU is used.
"""
import math

import numpy as np
import pytest
import scipy.fft
import scipy.sparse as sp

from oracle import helmholtz as O
from paper_1607_00968_gb300 import inputs as I


def crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# --------------------------------------------------------------------------
# operator
# --------------------------------------------------------------------------

@pytest.mark.parametrize("theta", [0.3, 1.1, 2.0, math.pi * 0.9])
def test_fourier_symbol_1d_paper(theta):
    """Sec. 3: for m = 1, h = 1 the 1D operator Lap + omega^2 m has the
    eigenvalue 2cos(theta) - 2 + omega^2 on exp(i theta x); ours is its
    negative (A = -A_paper)."""
    n, omega = 41, 0.7
    A = O.helmholtz_matrix(np.ones(n), np.zeros(n), omega, 1.0)
    u = np.exp(1j * theta * np.arange(n))
    Au = A @ u
    sym = -(2 * math.cos(theta) - 2 + omega ** 2)
    np.testing.assert_allclose(Au[1:-1], sym * u[1:-1], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_fourier_symbol_nd_with_attenuation(dim):
    """Interior nodes: A exp(i theta.x/h) = [sum_k (2-2cos th_k)/h^2
    - omega^2 m (1 - i(gamma+beta))] exp(...)."""
    rng = np.random.default_rng(1)
    shape = (9, 11, 13)[:dim]
    h, omega, m0, g0, beta = 12.5, 31.0, 2.5e-7, 0.3, 0.5
    M = O.helmholtz_matrix(np.full(shape, m0), np.full(shape, g0), omega, h, beta)
    th = rng.uniform(-3, 3, dim)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    phase = sum(t * g for t, g in zip(th, grids))
    u = np.exp(1j * phase)
    y = (M @ u.ravel()).reshape(shape)
    sym = sum((2 - 2 * math.cos(t)) / h ** 2 for t in th) \
        - omega ** 2 * m0 * (1 - 1j * (g0 + beta))
    inner = tuple(slice(1, -1) for _ in shape)
    np.testing.assert_allclose(y[inner], sym * u[inner], rtol=1e-12)


def test_operator_complex_symmetric():
    """A = A^T (symmetric stencil, diagonal mass): x^T A y = y^T A x."""
    rng = np.random.default_rng(2)
    shape = (7, 9)
    A = O.helmholtz_matrix(rng.uniform(1, 2, shape), rng.uniform(0, 1, shape),
                           3.0, 0.5, 0.5)
    x, y = crand(rng, A.shape[0]), crand(rng, A.shape[0])
    assert abs(x @ (A @ y) - y @ (A @ x)) < 1e-12 * abs(x @ (A @ y))
    assert abs(A - A.T).max() == 0


def test_dirichlet_boundary_row():
    """A corner node sees only its in-grid neighbours (zero beyond the node
    grid): row = (2d/h^2 - c) on the diagonal and -1/h^2 per neighbour."""
    shape, h, omega = (5, 6), 2.0, 1.5
    m, g = np.full(shape, 0.7), np.full(shape, 0.2)
    A = O.helmholtz_matrix(m, g, omega, h).toarray()
    c = omega ** 2 * 0.7 * (1 - 0.2j)
    assert A[0, 0] == pytest.approx(4 / h ** 2 - c)
    assert A[0, 1] == pytest.approx(-1 / h ** 2)
    assert A[0, 6] == pytest.approx(-1 / h ** 2)
    assert np.count_nonzero(A[0]) == 3


# --------------------------------------------------------------------------
# discrete-sine closed form (constant medium, gamma = 0, no layer)
# --------------------------------------------------------------------------

def dst_solve(shape, h, omega, m0, q):
    """u = S diag(1/lambda) S q with S the orthonormal DST-I per axis and
    lambda = sum_k (4/h^2) sin^2(pi kappa_k / (2(N_k+1))) - omega^2 m0."""
    lam = -omega ** 2 * m0 * np.ones(shape)
    for ax, n in enumerate(shape):
        k = np.arange(1, n + 1)
        view = [1] * len(shape)
        view[ax] = n
        lam = lam + (4 / h ** 2 * np.sin(np.pi * k / (2 * (n + 1))) ** 2).reshape(view)
    qq = q.reshape(shape)
    qh = scipy.fft.dstn(qq.real, type=1, norm="ortho") + \
        1j * scipy.fft.dstn(qq.imag, type=1, norm="ortho")
    uh = qh / lam
    u = scipy.fft.idstn(uh.real, type=1, norm="ortho") + \
        1j * scipy.fft.idstn(uh.imag, type=1, norm="ortho")
    return u.ravel(), lam


def well_separated_omega(shape, h, m0, lo, hi):
    """An omega in [lo, hi] making A indefinite with min|lambda| >= 1e-2
    max|lambda| (scan of the closed-form spectrum)."""
    best, arg = -1.0, None
    for omega in np.linspace(lo, hi, 401):
        _, lam = dst_solve(shape, h, omega, m0, np.zeros(int(np.prod(shape))))
        sep = np.min(np.abs(lam)) / np.max(np.abs(lam))
        if np.min(lam) < 0 < np.max(lam) and sep > best:
            best, arg = sep, omega
    return arg


@pytest.mark.parametrize("cells", [(16, 8), (8, 8, 4)])
def test_dense_lu_matches_dst_closed_form(cells):
    shape = I.node_shape(cells)
    h, m0 = 1.0, 1.0
    omega = well_separated_omega(shape, h, m0, 0.5, 1.5)
    rng = np.random.default_rng(3)
    q = crand(rng, int(np.prod(shape)))
    u_ref, lam = dst_solve(shape, h, omega, m0, q)
    assert np.min(np.abs(lam)) >= 1e-2 * np.max(np.abs(lam))
    assert np.min(lam) < 0 < np.max(lam)   # indefinite, as in the paper
    A = O.helmholtz_matrix(np.full(shape, m0), np.zeros(shape), omega, h)
    u = O.dense_solve(A, q)
    np.testing.assert_allclose(u, u_ref, rtol=1e-10, atol=1e-12 * np.abs(u_ref).max())


def test_fgmres_matches_dst_closed_form():
    cells = (32, 16)
    shape = I.node_shape(cells)
    h, m0 = 1.0, 1.0
    omega = well_separated_omega(shape, h, m0, 0.3, 0.8)
    rng = np.random.default_rng(4)
    Q = crand(rng, int(np.prod(shape)), 3)
    S = O.Solver(np.full(shape, m0), np.zeros(shape), omega, h, levels=3)
    U, infos = S.solve(Q, tol=1e-11, restart=10, block=3)
    assert infos[0].converged
    for k in range(3):
        u_ref, _ = dst_solve(shape, h, omega, m0, Q[:, k])
        assert np.linalg.norm(U[:, k] - u_ref) <= 1e-8 * np.linalg.norm(u_ref)


# --------------------------------------------------------------------------
# dense LU against numpy
# --------------------------------------------------------------------------

def test_lu_against_numpy_with_pivoting():
    rng = np.random.default_rng(5)
    n = 40
    A = crand(rng, n, n)
    A[0, 0] = 0.0           # forces a row exchange at the first step
    B = crand(rng, n, 3)
    np.testing.assert_allclose(O.lu_solve(O.lu_factor(A), B),
                               np.linalg.solve(A, B), rtol=1e-10, atol=1e-11)


def test_hierarchy_coarse_solve_matches_own_lu():
    rng = np.random.default_rng(19)
    shape = I.node_shape((8, 4))
    M = O.helmholtz_matrix(rng.uniform(1, 2, shape), rng.uniform(0, 1, shape), 2.0, 1.0, 0.5)
    H = O.Hierarchy(M, shape, 2)
    f = crand(rng, H.M[1].shape[0], 3)
    np.testing.assert_allclose(H.coarse_solve(f), O.dense_solve(H.M[1], f), rtol=1e-11)


def test_lu_singular_raises():
    with pytest.raises(np.linalg.LinAlgError):
        O.lu_factor(np.zeros((3, 3)))


# --------------------------------------------------------------------------
# grid transfers and Galerkin coarse operators
# --------------------------------------------------------------------------

def test_prolongation_1d_explicit():
    P = O.prolongation_1d(3).toarray()
    ref = np.array([[1, 0, 0], [.5, .5, 0], [0, 1, 0], [0, .5, .5], [0, 0, 1]])
    np.testing.assert_array_equal(P, ref)


@pytest.mark.parametrize("cells", [(8, 4), (4, 6, 2)])
def test_prolongation_reproduces_multilinear(cells):
    """Bi/trilinear interpolation reproduces multilinear functions exactly."""
    shape = I.node_shape(cells)
    cs = O.coarse_shape(shape)
    P = O.prolongation(shape)
    rng = np.random.default_rng(6)
    a = rng.standard_normal(2 ** len(shape))

    def f(grid_shape, scale):
        g = np.meshgrid(*[np.arange(n) * scale for n in grid_shape], indexing="ij")
        val = np.zeros(grid_shape)
        for bits in range(2 ** len(shape)):
            term = np.full(grid_shape, a[bits])
            for ax in range(len(shape)):
                if bits >> ax & 1:
                    term = term * g[ax]
            val += term
        return val.ravel()

    np.testing.assert_allclose(P @ f(cs, 2.0), f(shape, 1.0), rtol=1e-12, atol=1e-12)


def test_galerkin_2d_closed_form():
    """Constant coefficients, interior coarse node:  P^T (-Lap - c) P =
    (1/h^2)[-1/2, 1, -1/2] (x) [1/4, 3/2, 1/4] + [1/4,3/2,1/4] (x)
    (1/h^2)[-1/2, 1, -1/2] - c [1/4,3/2,1/4] (x) [1/4,3/2,1/4]
    (derived by hand from the 1D products P^T L P and P^T P)."""
    cells, h, omega, m0, g0 = (16, 16), 0.5, 2.0, 1.3, 0.4
    shape = I.node_shape(cells)
    M = O.helmholtz_matrix(np.full(shape, m0), np.full(shape, g0), omega, h)
    H = O.Hierarchy(M, shape, 2)
    Mc = H.M[1].toarray()
    cs = H.shapes[1]
    lap = np.array([-0.5, 1.0, -0.5]) / h ** 2
    mass = np.array([0.25, 1.5, 0.25])
    c = omega ** 2 * m0 * (1 - 1j * g0)
    ref = np.outer(lap, mass) + np.outer(mass, lap) - c * np.outer(mass, mass)
    J = (4, 5)
    row = Mc[np.ravel_multi_index(J, cs)].reshape(cs)
    np.testing.assert_allclose(row[J[0] - 1:J[0] + 2, J[1] - 1:J[1] + 2], ref, rtol=1e-13)
    assert np.count_nonzero(row) == 9


def test_galerkin_symmetric_and_triple_product():
    rng = np.random.default_rng(7)
    shape = I.node_shape((8, 8, 4))
    M = O.helmholtz_matrix(rng.uniform(1, 2, shape), rng.uniform(0, 1, shape), 2.0, 1.0, 0.5)
    H = O.Hierarchy(M, shape, 3)
    for l in range(1, 3):
        assert abs(H.M[l] - H.M[l].T).max() < 1e-12 * abs(H.M[l]).max()
    x = crand(rng, H.M[1].shape[0])
    np.testing.assert_allclose(H.M[1] @ x, H.P[0].T @ (M @ (H.P[0] @ x)), rtol=1e-12)
    # 27-point stencil on the first coarse level of a 3D grid
    assert max(np.diff(H.M[1].indptr)) == 27


# --------------------------------------------------------------------------
# relaxation and cycle
# --------------------------------------------------------------------------

def small_problem(cells=(16, 8), seed=0, omega_scale=1.0):
    v = I.layered_velocity_2d(seed, cells)
    shape = I.node_shape(cells)
    return dict(m=1.0 / v ** 2, gamma=I.absorbing_gamma(shape, 3),
                omega=I.omega_for_ppw(25.0) * omega_scale, h=25.0)


def test_jacobi_fixed_point():
    p = small_problem()
    M = O.helmholtz_matrix(p["m"], p["gamma"], p["omega"], p["h"], 0.5)
    rng = np.random.default_rng(8)
    f = crand(rng, M.shape[0], 2)
    u = O.dense_solve(M, f)
    np.testing.assert_allclose(O.jacobi(M, M.diagonal(), u, f, 0.8, 3), u, rtol=1e-10)


def test_two_grid_without_smoothing_is_coarse_projection():
    """With no relaxation the two-grid cycle is B = P Mc^{-1} P^T, and for a
    Galerkin Mc = P^T M P it satisfies B M P = P exactly."""
    p = small_problem()
    shape = p["m"].shape
    M = O.helmholtz_matrix(p["m"], p["gamma"], p["omega"], p["h"], 0.5)
    H = O.Hierarchy(M, shape, 2)
    rng = np.random.default_rng(9)
    ec = crand(rng, H.M[1].shape[0], 2)
    Pe = H.P[0] @ ec
    out = O.vcycle(H, M @ Pe, 0, pre=0, post=0)
    np.testing.assert_allclose(out, Pe, rtol=1e-9, atol=1e-12 * np.abs(Pe).max())


def test_jacobi_sweeps_hand_computed():
    """Damped Jacobi with weight 0.8 on a 3-node 1D operator, worked by hand.
    h = 1, omega = 1, m = (1, 2, 1), gamma = 0, shift 0.5, so c = m (1 - 0.5i)
    and M = tridiag(-1, 2, -1) - diag(c) has diagonal (1 + 0.5i, 1i, 1 + 0.5i).
    From u = (1, 0, 0) with f = (0, 1, 0): r = (-1 - 0.5i, 2, 0), D^-1 r =
    (-1, -2i, 0), so one sweep gives (0.2, -1.6i, 0); a second sweep gives
    (-0.472 - 1.024i, -1.28i, -0.512 - 1.024i).  A wrong weight, a wrong sign
    or a diagonal without the shift (diag(A)) changes these numbers."""
    M = O.helmholtz_matrix(np.array([1.0, 2.0, 1.0]), np.zeros(3), 1.0, 1.0, 0.5)
    np.testing.assert_allclose(M.diagonal(), [1 + 0.5j, 1j, 1 + 0.5j], rtol=0, atol=1e-15)
    u0 = np.array([[1.0], [0.0], [0.0]], dtype=complex)
    f = np.array([[0.0], [1.0], [0.0]], dtype=complex)
    one = O.jacobi(M, M.diagonal(), u0, f, 0.8, 1).ravel()
    two = O.jacobi(M, M.diagonal(), u0, f, 0.8, 2).ravel()
    np.testing.assert_allclose(one, [0.2, -1.6j, 0.0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(two, [-0.472 - 1.024j, -1.28j, -0.512 - 1.024j], rtol=0, atol=1e-14)


def test_jacobi_zero_guess_sweep_is_scaled_diagonal_solve():
    """One sweep from u = 0 is 0.8 f / diag(M), elementwise."""
    p = small_problem()
    M = O.helmholtz_matrix(p["m"], p["gamma"], p["omega"], p["h"], 0.5)
    rng = np.random.default_rng(21)
    f = crand(rng, M.shape[0], 3)
    u = O.jacobi(M, M.diagonal(), np.zeros_like(f), f, 0.8, 1)
    np.testing.assert_allclose(u, 0.8 * f / M.diagonal()[:, None], rtol=1e-15)


def _interp_1d(nc):
    """Linear interpolation written out from its definition: coarse node J
    sits on fine node 2J (weight 1) and feeds its two fine neighbours 2J - 1,
    2J + 1 with weight 1/2."""
    nf = 2 * nc - 1
    P = np.zeros((nf, nc))
    for J in range(nc):
        P[2 * J, J] = 1.0
        if 2 * J - 1 >= 0:
            P[2 * J - 1, J] = 0.5
        if 2 * J + 1 < nf:
            P[2 * J + 1, J] = 0.5
    return P


def _dense_cycle_operator(Md, shape, levels, pre, post, w, gamma):
    """B with z = B f for the cycle of Alg. "Two-grid cycle" applied
    recursively, from dense matrices only.  Its error propagation is
        I - B M = S^post (I - P B_c^(gamma) P^T M) S^pre,
    S = I - w D^-1 M with D = diag(M) of the shifted operator, M_c = P^T M P,
    B_c^(gamma) = (I - (I - B_c M_c)^gamma) M_c^-1 (gamma cycles on the
    coarse level, each on the residual of the last; the coarsest level is
    solved exactly)."""
    n = Md.shape[0]
    if levels == 1:
        return np.linalg.inv(Md)
    P = _interp_1d((shape[0] - 1) // 2 + 1)
    for ax in range(1, len(shape)):
        P = np.kron(P, _interp_1d((shape[ax] - 1) // 2 + 1))
    cshape = tuple((k - 1) // 2 + 1 for k in shape)
    Mc = P.T @ Md @ P
    Bc = _dense_cycle_operator(Mc, cshape, levels - 1, pre, post, w, gamma)
    if levels - 1 > 1 and gamma == 2:
        Ec = np.eye(Mc.shape[0]) - Bc @ Mc
        Bc = (np.eye(Mc.shape[0]) - Ec @ Ec) @ np.linalg.inv(Mc)
    I_ = np.eye(n)
    S = I_ - w * np.diag(1.0 / np.diag(Md)) @ Md
    E = np.linalg.matrix_power(S, post) @ (I_ - P @ Bc @ P.T @ Md) @ np.linalg.matrix_power(S, pre)
    return (I_ - E) @ np.linalg.inv(Md)


@pytest.mark.parametrize("levels,pre,post,gamma", [(2, 2, 2, 1), (2, 1, 0, 1), (2, 0, 1, 1),
                                                   (2, 2, 1, 1), (3, 2, 2, 1), (3, 1, 2, 1),
                                                   (3, 2, 2, 2)])
def test_cycle_error_propagation_matches_dense_restatement(levels, pre, post, gamma):
    """The oracle's cycle, applied to the columns of M (so that its output is
    B M), against the dense error-propagation product of Alg. "Two-grid
    cycle" on 9 x 5 nodes (weight 0.8 and D = diag(M) of the shifted operator,
    written in the restatement).  Swapped pre/post counts, a missing sweep, a
    sweep on the wrong level, another weight or diag(A) for diag(M) each
    change B M."""
    cells = (8, 4)
    shape = I.node_shape(cells)
    rng = np.random.default_rng(22)
    m = rng.uniform(0.5, 1.5, shape)
    gam = np.zeros(shape)
    gam[:, :2] = 0.6
    omega, h = 1.1, 1.0
    M = O.helmholtz_matrix(m, gam, omega, h, 0.5)
    Md = M.toarray()
    H = O.Hierarchy(M, shape, levels)
    if (pre, post, gamma) == (2, 2, 1):
        got = O.vcycle(H, Md.astype(complex))           # defaults: V(2,2), weight 0.8
    else:
        got = O.vcycle(H, Md.astype(complex), 0, pre, post, 0.8, gamma)
    want = _dense_cycle_operator(Md, shape, levels, pre, post, 0.8, gamma) @ Md
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_cycle_restatement_detects_planted_mistakes():
    """The dense restatement separates the readings a mistake would give:
    swapped pre/post counts, weight 1.0 for 0.8 and diag(A) for diag(M) all
    move B M by far more than the tolerance of the test above."""
    cells = (8, 4)
    shape = I.node_shape(cells)
    rng = np.random.default_rng(22)
    m = rng.uniform(0.5, 1.5, shape)
    gam = np.zeros(shape)
    gam[:, :2] = 0.6
    M = O.helmholtz_matrix(m, gam, 1.1, 1.0, 0.5).toarray()
    A = O.helmholtz_matrix(m, gam, 1.1, 1.0, 0.0).toarray()
    ref = _dense_cycle_operator(M, shape, 2, 2, 1, 0.8, 1) @ M
    tol = 1e-11 * np.abs(ref).max()
    assert np.abs(_dense_cycle_operator(M, shape, 2, 1, 2, 0.8, 1) @ M - ref).max() > 1e3 * tol
    assert np.abs(_dense_cycle_operator(M, shape, 2, 2, 1, 1.0, 1) @ M - ref).max() > 1e3 * tol
    # diag(A) in the smoother: restate S with the unshifted diagonal
    n = M.shape[0]
    P = np.kron(_interp_1d(3), _interp_1d(5))
    Bc = np.linalg.inv(P.T @ M @ P)
    S = np.eye(n) - 0.8 * np.diag(1.0 / np.diag(A)) @ M
    E = S @ (np.eye(n) - P @ Bc @ P.T @ M) @ S @ S
    assert np.abs((np.eye(n) - E) - ref).max() > 1e3 * tol


def test_vcycle_is_linear():
    p = small_problem((16, 16))
    shape = p["m"].shape
    M = O.helmholtz_matrix(p["m"], p["gamma"], p["omega"], p["h"], 0.5)
    H = O.Hierarchy(M, shape, 3)
    rng = np.random.default_rng(10)
    f1, f2 = crand(rng, M.shape[0], 1), crand(rng, M.shape[0], 1)
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    np.testing.assert_allclose(O.vcycle(H, a * f1 + b * f2),
                               a * O.vcycle(H, f1) + b * O.vcycle(H, f2), rtol=1e-11)


def test_vcycle_poisson_convergence_factor():
    """omega = 0 (Poisson): the V(2,2) iteration with weighted Jacobi
    converges at the textbook rate (factor well below 0.5)."""
    shape = I.node_shape((32, 32))
    M = O.helmholtz_matrix(np.ones(shape), np.zeros(shape), 0.0, 1.0)
    H = O.Hierarchy(M, shape, 4)
    rng = np.random.default_rng(11)
    f = crand(rng, M.shape[0], 1)
    u = np.zeros_like(f)
    r0 = np.linalg.norm(f)
    for _ in range(6):
        u = u + O.vcycle(H, f - M @ u)
    rate = (np.linalg.norm(f - M @ u) / r0) ** (1 / 6)
    assert rate < 0.3


# --------------------------------------------------------------------------
# block FGMRES
# --------------------------------------------------------------------------

def test_fgmres_residual_estimates_match_brute_force():
    """With a fixed linear preconditioner B, block FGMRES after j steps
    minimises each column's residual over A B K_j, K_j the block Krylov space
    of A B started at R_0 = Q.  Brute force: build the space explicitly and
    solve the least-squares problems with numpy."""
    p = small_problem((8, 8), seed=3)
    shape = p["m"].shape
    S = O.Solver(p["m"], p["gamma"], p["omega"], p["h"], levels=2)
    rng = np.random.default_rng(12)
    Q = crand(rng, S.A.shape[0], 2)
    _, info = O.block_fgmres(S.A, S.precond, Q, tol=1e-14, restart=4, max_restarts=1)
    K = [Q]
    for _ in range(3):
        K.append(S.A @ S.precond(K[-1]))
    for j in range(1, 5):
        Xspace = np.hstack([S.precond(k) for k in K[:j]])
        AX = S.A @ Xspace
        Qb, _ = np.linalg.qr(AX)
        res = Q - Qb @ (Qb.conj().T @ Q)
        ref = np.linalg.norm(res, axis=0) / np.linalg.norm(Q, axis=0)
        np.testing.assert_allclose(info.history[j - 1], ref, rtol=1e-6, atol=1e-14)


def test_fgmres_arnoldi_relation_and_orthonormality():
    rng = np.random.default_rng(13)
    W = crand(rng, 50, 4)
    V, _ = np.linalg.qr(crand(rng, 50, 3))
    Q, R, dep = O.orthonormalize(W - V @ (V.conj().T @ W), [V],
                                 np.linalg.norm(W, axis=0), rng)
    assert dep == []
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(4), atol=1e-13)
    assert np.abs(V.conj().T @ Q).max() < 1e-13
    np.testing.assert_allclose(Q @ R, W - V @ (V.conj().T @ W), atol=1e-12)
    assert np.all(np.diag(R).real > 0) and np.all(np.diag(R).imag == 0)
    # QR with real positive diagonal is unique: equals phase-fixed Householder
    Qh, Rh = np.linalg.qr(W - V @ (V.conj().T @ W))
    ph = np.diag(Rh) / np.abs(np.diag(Rh))
    np.testing.assert_allclose(R, (Rh.T * ph.conj()).T, atol=1e-12)


def test_orthonormalize_rank_deficient_column():
    rng = np.random.default_rng(14)
    W = crand(rng, 40, 3)
    W[:, 2] = 2.0 * W[:, 0] - 1j * W[:, 1]
    Q, R, dep = O.orthonormalize(W, [], np.linalg.norm(W, axis=0), rng)
    assert dep == [2]
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(3), atol=1e-13)
    np.testing.assert_allclose(Q @ R, W, atol=1e-12)
    assert R[2, 2] == 0


def test_manufactured_solution_2d():
    p = small_problem((32, 16), seed=1)
    S = O.Solver(p["m"], p["gamma"], p["omega"], p["h"], levels=3)
    rng = np.random.default_rng(15)
    Uk = crand(rng, S.A.shape[0], 4)
    Q = S.A @ Uk
    U, infos = S.solve(Q, tol=1e-11, restart=10, block=4)
    assert infos[0].converged
    assert np.all(O.relres(S.A, U, Q) <= 1e-11)
    assert np.linalg.norm(U - Uk) <= 1e-7 * np.linalg.norm(Uk)


def test_dense_lu_tiny_grids_against_fgmres():
    for cells, lv in (((8, 4), 2), ((16, 8), 3), ((8, 8, 4), 2)):
        shape = I.node_shape(cells)
        g = I.absorbing_gamma(shape, 2)
        rng = np.random.default_rng(16)
        m = rng.uniform(0.5, 1.5, shape)
        S = O.Solver(m, g, 1.2, 1.0, levels=lv)
        Q = crand(rng, S.A.shape[0], 2)
        U, infos = S.solve(Q, tol=1e-12, restart=8, block=2)
        Ud = O.dense_solve(S.A, Q)
        assert np.linalg.norm(U - Ud) <= 1e-9 * np.linalg.norm(Ud)


def test_reciprocity():
    """A complex symmetric => (A^{-1} e_a)[b] = (A^{-1} e_b)[a]."""
    p = small_problem((32, 16), seed=2)
    S = O.Solver(p["m"], p["gamma"], p["omega"], p["h"], levels=3)
    N = S.A.shape[0]
    a, b = 40, N - 77
    Q = np.zeros((N, 2), dtype=complex)
    Q[a, 0] = Q[b, 1] = 1.0
    U, infos = S.solve(Q, tol=1e-12, restart=10, block=2)
    assert abs(U[b, 0] - U[a, 1]) <= 1e-9 * abs(U[b, 0])


def test_adjoint_solve():
    p = small_problem((32, 16), seed=3)
    S = O.Solver(p["m"], p["gamma"], p["omega"], p["h"], levels=3)
    rng = np.random.default_rng(17)
    B = crand(rng, S.A.shape[0], 2)
    L, _ = S.adjoint(B, tol=1e-11, block=2)
    AH = S.A.conj().T
    assert np.linalg.norm(AH @ L - B) <= 1e-10 * np.linalg.norm(B)
    X, _ = S.solve(B, tol=1e-11, block=2)
    # <A^{-1} x, y> = <x, A^{-H} y> (sesquilinear)
    lhs = np.vdot(B[:, 1], X[:, 0])
    rhs = np.vdot(L[:, 1], B[:, 0])
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_zero_and_duplicate_columns():
    p = small_problem((16, 8), seed=4)
    S = O.Solver(p["m"], p["gamma"], p["omega"], p["h"], levels=2)
    rng = np.random.default_rng(18)
    q = crand(rng, S.A.shape[0])
    Q = np.stack([q, np.zeros_like(q), q, 2 * q], axis=1)
    U, infos = S.solve(Q, tol=1e-10, block=4)
    assert infos[0].converged
    assert np.all(U[:, 1] == 0)
    np.testing.assert_allclose(U[:, 2], U[:, 0], rtol=1e-8)
    np.testing.assert_allclose(U[:, 3], 2 * U[:, 0], rtol=1e-8)
    assert np.all(O.relres(S.A, U, Q) <= 1e-10)


# --------------------------------------------------------------------------
# block BiCGSTAB with W-cycles (Sec. 5.3 "W-BiCG")
# --------------------------------------------------------------------------

def test_wcycle_is_linear_and_better_than_vcycle_on_poisson():
    shape = I.node_shape((32, 32))
    M = O.helmholtz_matrix(np.ones(shape), np.zeros(shape), 0.0, 1.0)
    H = O.Hierarchy(M, shape, 4)
    rng = np.random.default_rng(30)
    f1, f2 = crand(rng, M.shape[0], 1), crand(rng, M.shape[0], 1)
    np.testing.assert_allclose(O.vcycle(H, 2 * f1 - 1j * f2, gamma=2),
                               2 * O.vcycle(H, f1, gamma=2) - 1j * O.vcycle(H, f2, gamma=2),
                               rtol=1e-11)
    e_v = np.linalg.norm(f1 - M @ O.vcycle(H, f1, gamma=1))
    e_w = np.linalg.norm(f1 - M @ O.vcycle(H, f1, gamma=2))
    assert e_w < e_v


def scalar_bicgstab(A, Mp, b, iters):
    """van der Vorst's BiCGSTAB for one right-hand side (complex, r_hat^H
    products), right-preconditioned: the s = 1 case of the block method."""
    x = np.zeros_like(b)
    r = b.copy()
    rh = r.copy()
    rho = alpha = omega = 1.0
    v = p = np.zeros_like(b)
    hist = []
    for _ in range(iters):
        rho_new = np.vdot(rh, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = Mp(p)
        v = A @ ph
        alpha = rho_new / np.vdot(rh, v)
        s = r - alpha * v
        sh = Mp(s)
        t = A @ sh
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho = rho_new
        hist.append(np.linalg.norm(r))
    return x, hist


def test_block_bicgstab_single_column_is_scalar_bicgstab():
    p = small_problem((16, 16), seed=5)
    S = O.Solver(p["m"], p["gamma"], p["omega"], p["h"], levels=2)
    rng = np.random.default_rng(31)
    b = crand(rng, S.A.shape[0])
    Mp = lambda v: S.precond(v[:, None], 2)[:, 0]
    xs, hist = scalar_bicgstab(S.A, Mp, b, 4)
    X, info = O.block_bicgstab(S.A, lambda V: S.precond(V, 2), b[:, None], tol=1e-300, maxit=4,
                               max_restarts=1)
    np.testing.assert_allclose(np.array(info.history)[:, 0] * np.linalg.norm(b), hist, rtol=1e-8)
    np.testing.assert_allclose(X[:, 0], xs, rtol=1e-8, atol=1e-12 * np.abs(xs).max())


def test_block_bicgstab_converges_and_keeps_biorthogonality():
    for cells, lv in (((16, 8), 2), ((32, 16), 3), ((8, 8, 4), 2)):
        shape = I.node_shape(cells)
        g = I.absorbing_gamma(shape, 2)
        rng = np.random.default_rng(32)
        S = O.Solver(rng.uniform(0.5, 1.5, shape), g, 1.2, 1.0, levels=lv)
        Q = crand(rng, S.A.shape[0], 3)
        U, infos = S.solve_bicgstab(Q, tol=1e-11, block=3, gamma=2)
        assert infos[0].converged
        Ud = O.dense_solve(S.A, Q)
        assert np.linalg.norm(U - Ud) <= 1e-8 * np.linalg.norm(Ud)
        # alpha makes S orthogonal to the shadow block (while S is above rounding)
        assert max(infos[0].biortho[:3]) < 1e-10


# --------------------------------------------------------------------------
# FWI sensitivities (Sec. 2.4 Eq. fwisens)
# --------------------------------------------------------------------------

def fwi_setup(seed=50):
    cells = (8, 6)
    shape = I.node_shape(cells)
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.8, 1.2, shape)
    g = I.absorbing_gamma(shape, 2) + 0.05
    omega, h = 1.3, 1.0
    N = int(np.prod(shape))
    Q = np.zeros((N, 2), dtype=complex)
    Q[3, 0] = Q[5, 1] = 1.0
    recv = np.arange(0, shape[1])                 # top row
    return m, g, omega, h, Q, recv, rng


def test_fwi_gradient_finite_differences():
    m, g, omega, h, Q, recv, rng = fwi_setup()

    def solvers(mm):
        A = O.helmholtz_matrix(mm, g, omega, h)
        return (lambda B: O.dense_solve(A, B)), (lambda B: O.dense_solve(A.conj().T, B))

    d_obs = crand(rng, recv.size, 2)
    s, a = solvers(m)
    phi, grad, _ = O.fwi_misfit_gradient(s, a, g, omega, Q, recv, d_obs)
    eps = 1e-6
    for k in rng.choice(m.size, 6, replace=False):
        mp, mm_ = m.copy().ravel(), m.copy().ravel()
        mp[k] += eps
        mm_[k] -= eps
        sp_, ap_ = solvers(mp.reshape(m.shape))
        sm_, am_ = solvers(mm_.reshape(m.shape))
        fp = O.fwi_misfit_gradient(sp_, ap_, g, omega, Q, recv, d_obs)[0]
        fm = O.fwi_misfit_gradient(sm_, am_, g, omega, Q, recv, d_obs)[0]
        num = (fp - fm) / (2 * eps)
        assert abs(num - grad[k]) <= 1e-6 * max(1.0, abs(num)), (k, num, grad[k])


def test_fwi_jv_jtw_dot_product():
    """<J v, w>_R = v . J^T w for the real-to-complex linear map J."""
    m, g, omega, h, Q, recv, rng = fwi_setup(51)
    A = O.helmholtz_matrix(m, g, omega, h)
    solve = lambda B: O.dense_solve(A, B)
    adjoint = lambda B: O.dense_solve(A.conj().T, B)
    U = solve(Q)
    v = rng.standard_normal(m.size)
    W = crand(rng, recv.size, 2)
    Jv = O.fwi_jv(solve, g, omega, U, v, recv)
    lhs = float(np.sum(np.real(np.conj(W) * Jv)))
    rhs = float(v @ O.fwi_jtw(adjoint, g, omega, U, W, recv))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    # J v is the derivative of the sampled field along v
    eps = 1e-6
    Ap = O.helmholtz_matrix(m + eps * v.reshape(m.shape), g, omega, h)
    Am = O.helmholtz_matrix(m - eps * v.reshape(m.shape), g, omega, h)
    num = (O.dense_solve(Ap, Q) - O.dense_solve(Am, Q))[recv] / (2 * eps)
    np.testing.assert_allclose(Jv, num, rtol=1e-6, atol=1e-9 * np.abs(num).max())


def test_kcycle_coarse_correction_minimises_the_residual():
    """The K-cycle's coarse correction is the minimal-residual combination of
    the two preconditioned directions: brute-force least squares over
    span{z1, z2} gives the same residual."""
    p = small_problem((32, 32), seed=6)
    shape = p["m"].shape
    M = O.helmholtz_matrix(p["m"], p["gamma"], p["omega"], p["h"], 0.5)
    H = O.Hierarchy(M, shape, 4)
    rng = np.random.default_rng(33)
    r = crand(rng, H.M[1].shape[0], 2)
    e = O._kcycle_correction(H, r, 1, 2, 2, 0.8)
    Mc = H.M[1]
    z1 = O.vcycle(H, r, 1, gamma=3)
    for j in range(2):
        r2 = r[:, j] - Mc @ (z1[:, j] * (np.vdot(Mc @ z1[:, j], r[:, j]) / np.vdot(Mc @ z1[:, j], Mc @ z1[:, j])))
        z2 = O.vcycle(H, r2[:, None], 1, gamma=3)[:, 0]
        Z = np.stack([z1[:, j], z2], axis=1)
        c, *_ = np.linalg.lstsq(Mc @ Z, r[:, j], rcond=None)
        best = np.linalg.norm(r[:, j] - Mc @ (Z @ c))
        got = np.linalg.norm(r[:, j] - Mc @ e[:, j])
        assert got <= best * (1 + 1e-8) + 1e-12


def test_kcycle_fgmres_converges():
    p = small_problem((32, 32), seed=7)
    S = O.Solver(p["m"], p["gamma"], p["omega"], p["h"], levels=4)
    rng = np.random.default_rng(34)
    Q = crand(rng, S.A.shape[0], 2)
    X, info = O.block_fgmres(S.A, lambda V: S.precond(V, 3), Q, tol=1e-10, restart=10)
    assert info.converged
    assert np.linalg.norm(X - O.dense_solve(S.A, Q)) <= 1e-7 * np.linalg.norm(X)
