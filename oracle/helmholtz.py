"""FP64 oracle: Helmholtz operator, shifted-Laplacian multigrid, block FGMRES.

Test infrastructure only (see the package docstring).  Notation follows the
paper with the sign convention of the solver library:

    A u := -Lap_h u - omega^2 m (1 - i gamma) u,

with ``gamma`` dimensionless.  The paper writes Lap_h u + omega^2
(1 - i gamma_p/omega) m u = q (Sec. 2.1, Eq. helm); so gamma = gamma_p/omega
and A = -A_paper (u = -u_paper for the same q).  The shifted operator used by
the preconditioner is M := A with gamma -> gamma + beta (Sec. 4: a positive
constant added to gamma).

Vectors are numpy arrays of shape (N, s) (node-major, one column per right
hand side); the node index is the C-order ravel of the node grid with x1
fastest (see ``paper_1607_00968_gb300.inputs``).  Dirichlet zero is imposed
beyond the node grid on every side.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp

# --------------------------------------------------------------------------
# Operator (Sec. 2.1 Eq. helm, Sec. 2.4 Eq. LinearSystem)
# --------------------------------------------------------------------------


def laplacian_1d(n: int, h: float) -> sp.csr_matrix:
    """Second-order FD  (u[i-1] - 2u[i] + u[i+1]) / h^2  on n nodes, zero
    beyond both ends (Sec. 2.4: second-order finite differences)."""
    main = -2.0 * np.ones(n)
    off = np.ones(n - 1)
    return (sp.diags([off, main, off], [-1, 0, 1]) / (h * h)).tocsr()


def laplacian(shape, h: float) -> sp.csr_matrix:
    """Lap_h on the node grid ``shape`` (numpy order, x1 last = fastest):
    the sum over axes of the 1D operator, as Kronecker products."""
    d = len(shape)
    L = None
    for ax in range(d):
        factors = [sp.identity(shape[k], format="csr") for k in range(d)]
        factors[ax] = laplacian_1d(shape[ax], h)
        term = factors[0]
        for f in factors[1:]:
            term = sp.kron(term, f, format="csr")
        L = term if L is None else L + term
    return L.tocsr()


def mass_coefficient(m, gamma, omega: float, shift: float = 0.0) -> np.ndarray:
    """c = omega^2 m (1 - i (gamma + shift)), flattened (Sec. 2.1 Eq. helm;
    the shift is the shifted-Laplacian imaginary shift of Sec. 4)."""
    m = np.asarray(m, dtype=np.float64).ravel()
    g = np.asarray(gamma, dtype=np.float64).ravel()
    return omega * omega * m * (1.0 - 1j * (g + shift))


def helmholtz_matrix(m, gamma, omega: float, h: float,
                     shift: float = 0.0) -> sp.csr_matrix:
    """Sparse A (shift = 0) or M (shift = beta): -Lap_h - diag(c)."""
    shape = np.shape(m)
    L = laplacian(shape, h)
    c = mass_coefficient(m, gamma, omega, shift)
    return (-L - sp.diags(c)).tocsr().astype(np.complex128)


def apply(Amat: sp.csr_matrix, U: np.ndarray) -> np.ndarray:
    """y = A U for a block U of shape (N, s)."""
    return np.asarray(Amat @ U)


# --------------------------------------------------------------------------
# Grid transfers (Sec. 4: bilinear interpolation, R = P^T)
# --------------------------------------------------------------------------


def prolongation_1d(nc: int) -> sp.csr_matrix:
    """Linear interpolation from nc coarse nodes to 2(nc-1)+1 fine nodes:
    coarse node J -> fine node 2J with weight 1 and fine nodes 2J+-1 with
    weight 1/2."""
    nf = 2 * (nc - 1) + 1
    rows, cols, vals = [], [], []
    for J in range(nc):
        for off, w in ((-1, 0.5), (0, 1.0), (1, 0.5)):
            i = 2 * J + off
            if 0 <= i < nf:
                rows.append(i)
                cols.append(J)
                vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def coarse_shape(shape):
    """Node shape of the next coarser grid (cells halved per axis)."""
    for n in shape:
        if (n - 1) % 2:
            raise ValueError("cells per axis must be even to coarsen: %r" % (shape,))
    return tuple((n - 1) // 2 + 1 for n in shape)


def prolongation(shape_fine) -> sp.csr_matrix:
    """Bi/trilinear interpolation P (tensor product of the 1D operators)."""
    cs = coarse_shape(shape_fine)
    P = prolongation_1d(cs[0])
    for n in cs[1:]:
        P = sp.kron(P, prolongation_1d(n), format="csr")
    return P.tocsr()


# --------------------------------------------------------------------------
# Dense LU with partial pivoting (coarsest solve, Sec. 4 last paragraph)
# --------------------------------------------------------------------------


def lu_factor(A: np.ndarray):
    """Gaussian elimination with partial pivoting, P A = L U.

    Returns (LU, piv): unit-lower L below the diagonal and U on and above it,
    ``piv[k]`` the row swapped with row k at step k."""
    LU = np.array(A, dtype=np.complex128, copy=True)
    n = LU.shape[0]
    piv = np.zeros(n, dtype=np.int64)
    for k in range(n):
        p = k + int(np.argmax(np.abs(LU[k:, k])))
        piv[k] = p
        if p != k:
            LU[[k, p], :] = LU[[p, k], :]
        if LU[k, k] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        LU[k + 1:, k] /= LU[k, k]
        LU[k + 1:, k + 1:] -= np.outer(LU[k + 1:, k], LU[k, k + 1:])
    return LU, piv


def lu_solve(fac, B: np.ndarray) -> np.ndarray:
    """Solve A X = B from ``lu_factor`` output (row swaps, then forward and
    back substitution)."""
    LU, piv = fac
    X = np.array(B, dtype=np.complex128, copy=True)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    n = LU.shape[0]
    for k in range(n):
        if piv[k] != k:
            X[[k, piv[k]], :] = X[[piv[k], k], :]
    for k in range(n):
        X[k + 1:, :] -= np.outer(LU[k + 1:, k], X[k, :])
    for k in range(n - 1, -1, -1):
        X[k, :] /= LU[k, k]
        X[:k, :] -= np.outer(LU[:k, k], X[k, :])
    return X[:, 0] if vec else X


def dense_solve(Amat, B: np.ndarray) -> np.ndarray:
    """u = A^{-1} q by the oracle's own LU (tiny grids only)."""
    Ad = Amat.toarray() if sp.issparse(Amat) else np.asarray(Amat)
    return lu_solve(lu_factor(Ad), B)


# --------------------------------------------------------------------------
# Shifted-Laplacian multigrid (Sec. 4, Alg. "Two-grid cycle")
# --------------------------------------------------------------------------


class Hierarchy:
    """Galerkin hierarchy M_0 = M, M_{l+1} = P_l^T M_l P_l (Sec. 4), with a
    dense LU of the coarsest operator (Sec. 4: LU for a block of right-hand
    sides on the coarsest grid).  The coarsest LU is LAPACK's partial-pivoting
    factorisation (scipy.linalg.lu_factor, a library primitive; the oracle's
    own ``lu_factor`` restates it for the tiny-grid dense solves and both are
    pinned against numpy.linalg.solve)."""

    def __init__(self, M0: sp.csr_matrix, shape, levels: int):
        self.M = [M0.tocsr()]
        self.P = []
        self.shapes = [tuple(shape)]
        for _ in range(levels - 1):
            P = prolongation(self.shapes[-1])
            self.P.append(P)
            self.M.append((P.T @ self.M[-1] @ P).tocsr())
            self.shapes.append(coarse_shape(self.shapes[-1]))
        self.diag = [Ml.diagonal() for Ml in self.M]
        self.coarse_lu = scipy.linalg.lu_factor(self.M[-1].toarray())

    def coarse_solve(self, f):
        """M_L^{-1} f on the coarsest level."""
        return scipy.linalg.lu_solve(self.coarse_lu, f)

    @property
    def levels(self):
        return len(self.M)


def jacobi(M: sp.csr_matrix, diag: np.ndarray, u, f, w: float, sweeps: int):
    """Damped Jacobi u <- u + w D^{-1} (f - M u), ``sweeps`` times
    (Sec. 5.3: weighted Jacobi, weight 0.8)."""
    dinv = (1.0 / diag)[:, None]
    for _ in range(sweeps):
        u = u + w * dinv * (f - M @ u)
    return u


def _kcycle_correction(H: Hierarchy, r: np.ndarray, level: int, pre, post, w):
    """K-cycle coarse correction (Sec. 5.3 "K-cycles": the coarse system is
    solved by two iterations of a flexible Krylov method preconditioned by the
    cycle one level down), per column: two steps of flexible GMRES, written
    as GCR(2):  z1 = C(r), w1 = M z1, a1 = w1^H r / w1^H w1, r2 = r - a1 w1;
    z2 = C(r2), w2 = M z2, b = w1^H w2 / w1^H w1, w2 -= b w1, z2 -= b z1,
    a2 = w2^H r2 / w2^H w2;  e = a1 z1 + a2 z2  (C = this level's K-cycle)."""
    M = H.M[level]

    def dots(a, b):
        return np.sum(np.conj(a) * b, axis=0)

    def ratio(num, den):
        return np.where(den != 0, num / np.where(den != 0, den, 1), 0)

    z1 = vcycle(H, r, level, pre, post, w, 3)
    w1 = M @ z1
    n1 = dots(w1, w1)
    a1 = ratio(dots(w1, r), n1)
    r2 = r - w1 * a1
    z2 = vcycle(H, r2, level, pre, post, w, 3)
    w2 = M @ z2
    b = ratio(dots(w1, w2), n1)
    w2 = w2 - w1 * b
    z2 = z2 - z1 * b
    a2 = ratio(dots(w2, r2), dots(w2, w2))
    return z1 * a1 + z2 * a2


def vcycle(H: Hierarchy, f: np.ndarray, level: int = 0, pre: int = 2,
           post: int = 2, w: float = 0.8, gamma: int = 1) -> np.ndarray:
    """Multigrid cycle for M_level e = f from a zero initial guess, following
    Alg. "Two-grid cycle": pre-relax, restrict the residual with P^T, solve
    the coarse problem recursively (``gamma`` = 1 gives the V-cycle, 2 the
    W-cycle: two recursive calls, the second on the residual of the first; 3
    the K-cycle of Sec. 5.3, see ``_kcycle_correction``), prolong and
    correct, post-relax.  The coarsest level is solved with the dense LU, once
    per visit."""
    if level == H.levels - 1:
        return H.coarse_solve(f)
    M, d, P = H.M[level], H.diag[level], H.P[level]
    u = np.zeros_like(f)
    u = jacobi(M, d, u, f, w, pre)
    rc = P.T @ (f - M @ u)
    Mc = H.M[level + 1]
    if gamma == 3 and level + 1 < H.levels - 1:
        ec = _kcycle_correction(H, rc, level + 1, pre, post, w)
    else:
        ec = vcycle(H, rc, level + 1, pre, post, w, min(gamma, 2))
        if gamma == 2 and level + 1 < H.levels - 1:
            ec = ec + vcycle(H, rc - Mc @ ec, level + 1, pre, post, w, gamma)
    u = u + P @ ec
    u = jacobi(M, d, u, f, w, post)
    return u


# --------------------------------------------------------------------------
# Block flexible GMRES (Sec. 4; Sec. 5.3 "block FGMRES", Calandra et al.)
# --------------------------------------------------------------------------

DEP_ANGLE = 1e-7     # a block column within this sine of the span of the
                     # columns before it counts as dependent
DEP_ROUNDOFF = 1e-12  # ... and so does one this small against its norm
                      # before orthogonalisation


def _dot(q, w):
    return np.vdot(q, w)


def orthonormalize(W: np.ndarray, basis: list, ref: np.ndarray, rng):
    """Gram-Schmidt QR of the block W (N x s) against ``basis`` (a list of
    orthonormal blocks) and its own earlier columns, each column projected
    twice: W = Q R with Q orthonormal and orthogonal to the basis, R upper
    triangular with a real, non-negative diagonal.

    Reading of the paper (silent on rank deficiency): a column within
    ``DEP_ANGLE`` of the span of the columns before it, or smaller than
    ``DEP_ROUNDOFF * ref[k]`` (``ref`` = column norms before any
    orthogonalisation), is dependent: its R diagonal entry is 0 and its Q
    column is a random direction orthogonal to everything before it.
    Returns (Q, R, dependent column indices)."""
    N, s = W.shape
    Q = np.zeros_like(W)
    R = np.zeros((s, s), dtype=np.complex128)
    dep = []
    prev = [b[:, i] for b in basis for i in range(b.shape[1])]
    for k in range(s):
        w = W[:, k].copy()
        before = np.linalg.norm(w)
        for _ in range(2):
            for q in prev:
                w = w - _dot(q, w) * q
            for i in range(k):
                c = _dot(Q[:, i], w)
                R[i, k] += c
                w = w - c * Q[:, i]
        nrm = np.linalg.norm(w)
        if nrm <= DEP_ANGLE * before or nrm <= DEP_ROUNDOFF * ref[k] or nrm == 0.0:
            dep.append(k)
            z = rng.standard_normal(N) + 1j * rng.standard_normal(N)
            for _ in range(2):
                for q in prev + [Q[:, i] for i in range(k)]:
                    z = z - _dot(q, z) * q
            Q[:, k] = z / np.linalg.norm(z)
        else:
            R[k, k] = nrm
            Q[:, k] = w / nrm
    return Q, R, dep


class FGMRESInfo:
    def __init__(self, s):
        self.iters = 0             # preconditioner applications (block steps)
        self.restarts = 0
        self.relres = np.zeros(s)  # true relative residuals at exit
        self.converged = False
        self.history = []          # per step: LS residual estimates / ||b||


def block_fgmres(Amat, precond, B: np.ndarray, tol: float = 1e-6,
                 restart: int = 10, max_restarts: int = 50, seed: int = 0):
    """Block flexible GMRES(m) for A X = B, X_0 = 0 (Sec. 5.3; the flexible
    variant stores Z_j = precond(V_j), so the preconditioner may vary).

    Each restart cycle: R = B - A X; R = V_1 Lambda (QR); for j = 1..m:
    Z_j = precond(V_j), W = A Z_j, block Gram-Schmidt against V_1..V_j
    (two passes) giving H_{i,j}, W = V_{j+1} H_{j+1,j} (QR); the least-squares
    problem min ||E_1 Lambda - Hbar_j Y|| is solved column by column and the
    cycle stops when every column's residual estimate is <= tol ||b_i||.
    Then X += [Z_1 .. Z_j] Y and the true residual is checked.  Columns with
    b_i = 0 give x_i = 0."""
    B = np.asarray(B, dtype=np.complex128)
    N, s = B.shape
    rng = np.random.Generator(np.random.PCG64(seed))
    info = FGMRESInfo(s)
    X = np.zeros_like(B)
    bnorm = np.linalg.norm(B, axis=0)
    live = np.nonzero(bnorm > 0)[0]
    if live.size == 0:
        info.converged = True
        return X, info
    Bl = B[:, live]
    bl = bnorm[live]
    Xl = np.zeros_like(Bl)
    sl = live.size
    for cycle in range(max_restarts + 1):
        Rr = Bl - apply(Amat, Xl)
        rel = np.linalg.norm(Rr, axis=0) / bl
        if np.all(rel <= tol) or cycle == max_restarts:
            info.relres[live] = rel
            info.converged = bool(np.all(rel <= tol))
            break
        info.restarts = cycle
        V1, Lam, _ = orthonormalize(Rr, [], np.linalg.norm(Rr, axis=0), rng)
        Vs, Zs = [V1], []
        H = np.zeros(((restart + 1) * sl, restart * sl), dtype=np.complex128)
        E = np.zeros(((restart + 1) * sl, sl), dtype=np.complex128)
        E[:sl] = Lam
        Y = None
        for j in range(restart):
            Z = precond(Vs[j])
            Zs.append(Z)
            W = apply(Amat, Z)
            ref = np.linalg.norm(W, axis=0)
            for _ in range(2):
                for i in range(j + 1):
                    Hij = Vs[i].conj().T @ W
                    W = W - Vs[i] @ Hij
                    H[i * sl:(i + 1) * sl, j * sl:(j + 1) * sl] += Hij
            Vn, Rn, _ = orthonormalize(W, Vs, ref, rng)
            H[(j + 1) * sl:(j + 2) * sl, j * sl:(j + 1) * sl] = Rn
            Vs.append(Vn)
            info.iters += 1
            Hj = H[:(j + 2) * sl, :(j + 1) * sl]
            Ej = E[:(j + 2) * sl]
            Y = np.linalg.lstsq(Hj, Ej, rcond=None)[0]
            est = np.linalg.norm(Ej - Hj @ Y, axis=0)
            info.history.append(est / bl)
            if np.all(est <= tol * bl):
                break
        Xl = Xl + np.hstack(Zs) @ Y
    X[:, live] = Xl
    return X, info


# --------------------------------------------------------------------------
# Block BiCGSTAB (Sec. 5.3 "W-BiCG": block BiCGSTAB of El Guennouni et al.
# with a stationary W-cycle preconditioner)
# --------------------------------------------------------------------------


def _small_solve(G, Rhs, rel=1e-14):
    """Solve G Y = Rhs (s x s, s x s) by Gaussian elimination with partial
    pivoting; a pivot below rel * max|G| makes its row of Y zero (the block
    direction it stands for has collapsed)."""
    n = G.shape[0]
    Ga = np.array(G, dtype=np.complex128)
    Y = np.array(Rhs, dtype=np.complex128)
    scale = np.abs(Ga).max() if Ga.size else 0.0
    perm = np.arange(n)
    dead = np.zeros(n, dtype=bool)
    for k in range(n):
        p = k + int(np.argmax(np.abs(Ga[k:, k])))
        if p != k:
            Ga[[k, p]] = Ga[[p, k]]
            Y[[k, p]] = Y[[p, k]]
        if abs(Ga[k, k]) <= rel * scale:
            dead[k] = True
            continue
        f = Ga[k + 1:, k] / Ga[k, k]
        Ga[k + 1:, k:] -= np.outer(f, Ga[k, k:])
        Y[k + 1:] -= np.outer(f, Y[k])
    for k in range(n - 1, -1, -1):
        if dead[k]:
            Y[k] = 0
            continue
        Y[k] = (Y[k] - Ga[k, k + 1:] @ Y[k + 1:]) / Ga[k, k]
    return Y


class BiCGInfo(FGMRESInfo):
    def __init__(self, s):
        super().__init__(s)
        self.biortho = []    # per iteration: max |Rt^H S| / (|Rt| |S|)


def block_bicgstab(Amat, precond, B: np.ndarray, tol: float = 1e-6, maxit: int = 500,
                   max_restarts: int = 5):
    """Block BiCGSTAB, right-preconditioned, X_0 = 0, shadow block Rt = R_0:

        P_0 = R_0;  for k:  Ph = M P_k, V = A Ph,  alpha = (Rt^H V)^{-1} Rt^H R_k,
                            S = R_k - V alpha,  Sh = M S,  T = A Sh,
                            omega = <T, S>_F / <T, T>_F,
                            X += Ph alpha + omega Sh,  R_{k+1} = S - omega T,
                            beta = -(Rt^H V)^{-1} Rt^H T,  P_{k+1} = R_{k+1} + (P_k - omega V) beta

    (<X, Y>_F = trace(X^H Y)).  Stops when every column's recursive residual
    is <= tol ||b_i||, then checks the true residual and restarts from it if
    needed.  The preconditioner must be fixed and linear (Sec. 5.3: W-BiCG
    uses W-cycles).  ``iters`` counts preconditioner applications (two per
    iteration)."""
    B = np.asarray(B, dtype=np.complex128)
    N, s = B.shape
    info = BiCGInfo(s)
    X = np.zeros_like(B)
    bnorm = np.linalg.norm(B, axis=0)
    live = np.nonzero(bnorm > 0)[0]
    if live.size == 0:
        info.converged = True
        return X, info
    Bl, bl = B[:, live], bnorm[live]
    Xl = np.zeros_like(Bl)
    for restart in range(max_restarts + 1):
        R = Bl - apply(Amat, Xl)
        rel = np.linalg.norm(R, axis=0) / bl
        if np.all(rel <= tol) or restart == max_restarts:
            break
        info.restarts = restart
        Rt = R.copy()
        P = R.copy()
        for k in range(maxit):
            Ph = precond(P)
            V = apply(Amat, Ph)
            G = Rt.conj().T @ V
            alpha = _small_solve(G, Rt.conj().T @ R)
            S = R - V @ alpha
            nS = np.linalg.norm(S)
            if nS > 0:
                info.biortho.append(np.abs(Rt.conj().T @ S).max()
                                    / (np.linalg.norm(Rt) * nS))
            Sh = precond(S)
            T = apply(Amat, Sh)
            tt = np.vdot(T, T)
            omega = np.vdot(T, S) / tt if tt != 0 else 0.0
            Xl = Xl + Ph @ alpha + omega * Sh
            R = S - omega * T
            info.iters += 2
            est = np.linalg.norm(R, axis=0) / bl
            info.history.append(est)
            if np.all(est <= tol):
                break
            beta = _small_solve(G, -(Rt.conj().T @ T))
            P = R + (P - omega * V) @ beta
    R = Bl - apply(Amat, Xl)
    rel = np.linalg.norm(R, axis=0) / bl
    info.relres[live] = rel
    info.converged = bool(np.all(rel <= tol))
    X[:, live] = Xl
    return X, info


# --------------------------------------------------------------------------
# Whole solve (the method end to end)
# --------------------------------------------------------------------------


class Solver:
    """Set-up once per (m, gamma, omega) (Sec. 4: the hierarchy is built once
    and reused by all right-hand sides and by the adjoint solve)."""

    def __init__(self, m, gamma, omega: float, h: float, levels: int = 3,
                 shift: float = 0.5, pre: int = 2, post: int = 2,
                 w: float = 0.8):
        self.shape = np.shape(m)
        self.A = helmholtz_matrix(m, gamma, omega, h)
        self.M = helmholtz_matrix(m, gamma, omega, h, shift)
        self.H = Hierarchy(self.M, self.shape, levels)
        self.pre, self.post, self.w = pre, post, w

    def precond(self, V, gamma: int = 1):
        return vcycle(self.H, V, 0, self.pre, self.post, self.w, gamma)

    def solve_bicgstab(self, Q_cols: np.ndarray, tol=1e-6, block=None, gamma: int = 2,
                       maxit=500):
        """Block BiCGSTAB with W-cycles (gamma = 2) in groups of ``block``."""
        N, s = Q_cols.shape
        block = s if block is None else block
        U = np.zeros_like(Q_cols, dtype=np.complex128)
        infos = []
        for g0 in range(0, s, block):
            sl = slice(g0, min(s, g0 + block))
            U[:, sl], inf = block_bicgstab(self.A, lambda V: self.precond(V, gamma),
                                           Q_cols[:, sl], tol, maxit)
            infos.append(inf)
        return U, infos

    def solve(self, Q_cols: np.ndarray, tol=1e-6, restart=10, block=None,
              max_restarts=50, gamma: int = 1):
        """Q_cols: (N, s).  Columns are solved in groups of ``block``
        (independent block-FGMRES runs); returns (U, [info per group]).
        ``gamma`` picks the cycle: 1 V, 2 W, 3 K."""
        N, s = Q_cols.shape
        block = s if block is None else block
        U = np.zeros_like(Q_cols, dtype=np.complex128)
        infos = []
        for g0 in range(0, s, block):
            sl = slice(g0, min(s, g0 + block))
            U[:, sl], inf = block_fgmres(self.A, lambda V: self.precond(V, gamma), Q_cols[:, sl],
                                         tol, restart, max_restarts)
            infos.append(inf)
        return U, infos

    def adjoint(self, B_cols, **kw):
        """Solve A^H L = B.  A is complex symmetric (A = A^T: symmetric
        stencil, diagonal mass term), so L = conj(A^{-1} conj(B)) and the
        same hierarchy serves (Sec. 4: transposed hierarchy)."""
        U, infos = self.solve(np.conj(B_cols), **kw)
        return np.conj(U), infos


# --------------------------------------------------------------------------
# FWI sensitivities (Sec. 2.4 Eq. fwisens; data Eq. data; misfit Eq. minp)
# --------------------------------------------------------------------------
#
# In this sign convention A(m) = -Lap_h - w^2 diag(m (1 - i g)), so
# dA/dm_k = -w^2 (1 - i g_k) e_k e_k^T and differentiating A u = q gives
#     J = du/dm = w^2 A^{-1} diag((1 - i g) u)
# (the paper's J up to the sign of u).  With receivers R (node indices) the
# data are P^T u = u[R]; for real m, J^T w = Re(J^H P w) =
#     w^2 Re(conj((1 - i g) u) lambda),  lambda = A^{-H} P w,
# and the gradient of Phi = 1/2 sum_s ||u_s[R] - d_s||^2 is J^T (P^T u - d),
# summed over the sources.


def dA_dm(gamma, omega: float) -> np.ndarray:
    """w^2 (1 - i g): minus the derivative of A's diagonal w.r.t. m."""
    return omega * omega * (1.0 - 1j * np.asarray(gamma, dtype=np.float64).ravel())


def fwi_jv(solve, gamma, omega, U, v, recv):
    """P^T J v for every source: w^2 A^{-1} (dA_dm * U * v) sampled at recv.
    solve(B) returns A^{-1} B for B of shape (N, s)."""
    rhs = dA_dm(gamma, omega)[:, None] * U * np.asarray(v, dtype=np.float64).ravel()[:, None]
    return solve(rhs)[recv, :]


def fwi_jtw(adjoint, gamma, omega, U, W, recv):
    """J^T w summed over sources (real, length N): lambda = A^{-H} P w,
    sum_s Re(conj(dA_dm * u_s) lambda_s).  adjoint(B) returns A^{-H} B."""
    N = U.shape[0]
    PW = np.zeros((N, W.shape[1]), dtype=np.complex128)
    PW[recv, :] = W
    Lam = adjoint(PW)
    return np.sum(np.real(np.conj(dA_dm(gamma, omega)[:, None] * U) * Lam), axis=1)


def fwi_misfit_gradient(solve, adjoint, gamma, omega, Q, recv, d_obs):
    """(Phi, grad, U): Phi = 1/2 sum_s ||u_s[recv] - d_s||^2 and its gradient
    with respect to m (Eq. minp without regularisation, unit covariance)."""
    U = solve(Q)
    D = U[recv, :] - d_obs
    phi = 0.5 * float(np.sum(np.abs(D) ** 2))
    return phi, fwi_jtw(adjoint, gamma, omega, U, D, recv), U


def relres(Amat, U, Q) -> np.ndarray:
    """Per-column true relative residual ||q_i - A u_i|| / ||q_i|| in FP64."""
    R = Q - apply(Amat, U)
    qn = np.linalg.norm(Q, axis=0)
    rn = np.linalg.norm(R, axis=0)
    return np.where(qn > 0, rn / np.where(qn > 0, qn, 1.0), rn)
