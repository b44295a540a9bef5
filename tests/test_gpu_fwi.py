"""FWI sensitivity products on the GPU (helm_fwi_gradient, helm_fwi_jv,
helm_fwi_jtw) against the FP64 oracle (oracle.helmholtz.fwi_*, pinned by
finite differences and the dot-product test)."""
import numpy as np
import pytest

from oracle import helmholtz as O
from paper_1607_00968_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00968_gb300 import helm
    cells = (32, 16)
    v = I.layered_velocity_2d(3, cells)
    shape = I.node_shape(cells)
    m, g, h = 1.0 / v ** 2, I.absorbing_gamma(shape, 4) + 0.01, 25.0
    om = I.omega_for_ppw(h)
    S = helm.Solver(m, g, h, om, levels=2, block=3, prec="c64")
    A = O.helmholtz_matrix(m, g, om, h)
    solve = lambda B: O.dense_solve(A, B)
    adjoint = lambda B: O.dense_solve(A.conj().T, B)
    Q = I.point_sources(shape, I.line_positions(shape, 3, 1, 4), h)      # (s, N)
    recv = np.arange(2, shape[1] - 2)                                     # top row
    rng = np.random.default_rng(60)
    d_obs = 0.1 * (rng.standard_normal((3, recv.size)) + 1j * rng.standard_normal((3, recv.size)))
    return helm, S, m, g, om, Q, recv, d_obs, solve, adjoint, rng


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_gradient_matches_oracle(case):
    helm, S, m, g, om, Q, recv, d_obs, solve, adjoint, rng = case
    phi, grad, U = S.fwi_gradient(torch.as_tensor(Q).cuda(), d_obs, recv, tol=1e-11)
    phi_o, grad_o, U_o = O.fwi_misfit_gradient(solve, adjoint, g, om, Q.T, recv, d_obs.T)
    assert abs(phi - phi_o) <= 1e-8 * phi_o
    assert rel(grad.cpu().numpy(), grad_o) <= 1e-7
    assert rel(U.cpu().numpy().T, U_o) <= 1e-9
    # forward fields kept in 16 bits (Sec. 2.4): the gradient to about 1e-3
    phi_h, grad_h, _ = S.fwi_gradient(torch.as_tensor(Q).cuda(), d_obs, recv, tol=1e-11, store_half=True)
    assert rel(grad_h.cpu().numpy(), grad_o) <= 5e-3


def test_jv_jtw_match_oracle_and_are_adjoint(case):
    helm, S, m, g, om, Q, recv, d_obs, solve, adjoint, rng = case
    U = solve(Q.T)                                          # (N, s)
    Ud = torch.as_tensor(U.T.copy()).cuda()                 # (s, N) ABI
    v = rng.standard_normal(U.shape[0])
    W = rng.standard_normal((3, recv.size)) + 1j * rng.standard_normal((3, recv.size))
    jv = S.fwi_jv(Ud, v, recv, tol=1e-11).cpu().numpy()     # (s, nrec)
    jtw = S.fwi_jtw(Ud, W, recv, tol=1e-11).cpu().numpy()
    assert rel(jv.T, O.fwi_jv(solve, g, om, U, v, recv)) <= 1e-8
    assert rel(jtw, O.fwi_jtw(adjoint, g, om, U, W.T, recv)) <= 1e-8
    lhs = float(np.sum(np.real(np.conj(W) * jv)))
    assert abs(lhs - float(v @ jtw)) <= 1e-8 * abs(lhs)
    # 16-bit fields give the same products to about 1e-3
    U16 = S.fields_to_half(Ud)
    jv16 = S.fwi_jv(U16, v, recv, tol=1e-11, half=True).cpu().numpy()
    assert rel(jv16, jv) <= 5e-3
