"""Factored eikonal equation, fast marching and its sensitivities (Sec. 2.5).

TEST INFRASTRUCTURE ONLY: a plain, slow FP64 restatement of the method for
checking the CUDA path.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import it; the product path never does.

What is computed (paper Sec. 2.5, Eq. eik, Eq. factoredeikonal, Eq. Gudonov,
Eq. FOfactoredD, Algorithm "Fast Marching", Eq. Sensitivity / Sensitivity2):

* tau = tau0 * tau1 with tau0 = |x - x_s| and p0 = grad tau0 = (x - x_s)/|x - x_s|
  known analytically (0 at the source);
* first-order factored upwind derivatives along each axis a at node i:
      backward  D-_a tau1 = tau0_i (tau1_i - tau1_{i-e_a}) / h + p0_{a,i} tau1_i
      forward   D+_a tau1 = tau0_i (tau1_{i+e_a} - tau1_i) / h + p0_{a,i} tau1_i
  and the Godunov equation  sum_a max{D-_a tau1, -D+_a tau1, 0}^2 = m_i;
* fast marching: accept the front node of least tau (ties: lower node index),
  then re-solve the Godunov equation at each of its not-yet-accepted
  neighbours from the accepted ("known") values only;
* the sensitivity of tau1 to m: with the derivative chosen by fast marching
  at each node (a zero row where none), J = (sum_a diag(2 D_a tau1) D_a)^{-1},
  lower triangular in fast-marching order: J v by forward substitution,
  J^T w by backward substitution.

Readings (the paper leaves these open; the CUDA path takes the same ones):
  E1  the source node is known from the start with tau1 = sqrt(m_s), i.e. its
      row is tau1_s^2 = m_s (derivative row 2 tau1_s);
  E2  the local solve is the Godunov equation solved exactly for the node's
      value: every choice per axis (none, backward, forward; known neighbours
      only) gives a quadratic whose larger root is a candidate; a candidate is
      consistent when each chosen term is >= 0 and >= the axis' other known
      term, and each unchosen axis has no positive known term.  The least
      consistent candidate is taken (ties: first choice in the enumeration,
      axis 0 slowest, none < backward < forward); with none consistent (only
      through rounding) the least root with all chosen terms >= 0;
  E3  the key of the heap is tau = tau0 * tau1 (the paper's "minimal value of
      tau"); a node's value and direction change only when a new solve gives a
      strictly smaller tau1;
  E4  the derivative factor D_a tau1 in the sensitivity is evaluated from the
      stored tau1, which the paper keeps in single precision; the caller passes
      the rounded values.

Grids: numpy arrays of the node shape (x1 last, as the Helmholtz oracle),
flattened C order; axis a of the numpy array has spacing h.  Arithmetic is
plain IEEE double (products, sums, sqrt and divisions rounded once each, in
the order written here).
"""
from __future__ import annotations

import heapq
import itertools
import math

import numpy as np

FAR, FRONT, KNOWN = 0, 1, 2


def tau0_p0(shape, h: float, src):
    """tau0 = h |k - k_s| and p0 per numpy axis at every node (Sec. 2.5:
    distance from the source and its gradient, 0 at the source)."""
    d = len(shape)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    diff = [h * (grids[a] - float(src[a])) for a in range(d)]
    r2 = np.zeros(shape)
    for a in range(d):
        r2 = r2 + diff[a] * diff[a]
    t0 = np.sqrt(r2)
    p0 = np.zeros((d,) + tuple(shape))
    nz = t0 > 0
    for a in range(d):
        p0[a][nz] = diff[a][nz] / t0[nz]
    return t0, p0


def _choices(d):
    """Per-axis choices (0 none, 1 backward, 2 forward), axis 0 slowest."""
    return list(itertools.product((0, 1, 2), repeat=d))


def _strides(shape):
    return [int(np.prod(shape[a + 1:])) for a in range(len(shape))]


def local_solve(i, multi, shape, h, t0, p0, m, tau1, known, choices, strides=None):
    """Godunov solve at flat node i from known neighbours (reading E2).
    Returns (tau1_i, choice tuple) or (inf, None) when no neighbour is known."""
    d = len(shape)
    t0h = t0[i] / h
    # candidate terms alpha * x - beta per axis and direction:
    # alpha = tau0_i / h +- p0, beta = (tau0_i / h) tau1_nb
    cand = [[None, None, None] for _ in range(d)]
    if strides is None:
        strides = _strides(shape)
    for a in range(d):
        k = multi[a]
        pa = p0[a][i]
        if k > 0 and known[i - strides[a]]:
            nb = i - strides[a]
            cand[a][1] = (t0h + pa, t0h * tau1[nb])
        if k < shape[a] - 1 and known[i + strides[a]]:
            nb = i + strides[a]
            cand[a][2] = (t0h - pa, t0h * tau1[nb])
    if all(cand[a][1] is None and cand[a][2] is None for a in range(d)):
        return math.inf, None
    mi = m[i]
    best, best_c = math.inf, None
    fb, fb_c = math.inf, None
    for ch in choices:
        if all(c == 0 for c in ch):
            continue
        if any(c != 0 and cand[a][c] is None for a, c in enumerate(ch)):
            continue
        A = 0.0
        B = 0.0
        C = 0.0
        for a, c in enumerate(ch):
            if c:
                al, be = cand[a][c]
                A = A + al * al
                B = B + al * be
                C = C + be * be
        C = C - mi
        if A <= 0.0:
            continue
        disc = B * B - A * C
        if disc < 0.0:
            continue
        x = (B + math.sqrt(disc)) / A
        ok_pos = True
        ok = True
        for a, c in enumerate(ch):
            if c:
                al, be = cand[a][c]
                f = al * x - be
                if f < 0.0:
                    ok_pos = False
                    ok = False
                o = cand[a][3 - c]
                if o is not None and o[0] * x - o[1] > f:
                    ok = False
            else:
                for o in (cand[a][1], cand[a][2]):
                    if o is not None and o[0] * x - o[1] > 0.0:
                        ok = False
        if ok and x < best:
            best, best_c = x, ch
        if ok_pos and x < fb:
            fb, fb_c = x, ch
    if best_c is not None:
        return best, best_c
    return fb, fb_c


def encode_dir(ch):
    """Choice tuple -> byte: 2 bits per numpy axis (axis a in bits 2a, 2a+1)."""
    v = 0
    for a, c in enumerate(ch):
        v |= c << (2 * a)
    return v


def fast_marching(m, h: float, src):
    """Algorithm "Fast Marching" for the factored equation.

    m: node array (squared slowness); src: node multi-index (numpy axis
    order).  Returns dict(tau1, tau, t0, p0, order, dir, level) with flat
    arrays: order = nodes in acceptance order, dir = encoded choice per node
    (0xFF at the source), level = 1 + max level of the chosen neighbours (0 at
    the source): the wavefront depth of the triangular system."""
    shape = m.shape
    d = len(shape)
    N = m.size
    mf = m.reshape(-1).astype(np.float64)
    t0, p0 = tau0_p0(shape, h, src)
    t0f = t0.reshape(-1)
    p0f = p0.reshape(d, -1)
    tau1 = np.full(N, math.inf)
    state = np.zeros(N, dtype=np.int8)
    direction = np.zeros(N, dtype=np.uint8)
    level = np.zeros(N, dtype=np.int64)
    known = np.zeros(N, dtype=bool)
    s = int(np.ravel_multi_index(tuple(src), shape))
    tau1[s] = math.sqrt(mf[s])
    direction[s] = 0xFF
    heap = [(0.0, s)]
    state[s] = FRONT
    order = []
    choices = _choices(d)
    strides = _strides(shape)
    while heap:
        key, i = heapq.heappop(heap)
        if state[i] == KNOWN or key != t0f[i] * tau1[i]:
            continue                                   # stale entry
        state[i] = KNOWN
        known[i] = True
        order.append(i)
        multi = np.unravel_index(i, shape)
        for a in range(d):
            for step in (-1, 1):
                k = multi[a] + step
                if k < 0 or k >= shape[a]:
                    continue
                q = i + step * strides[a]
                if state[q] == KNOWN:
                    continue
                qm = np.unravel_index(q, shape)
                x, ch = local_solve(q, qm, shape, h, t0f, p0f, mf, tau1, known, choices, strides)
                if x < tau1[q]:
                    tau1[q] = x
                    direction[q] = encode_dir(ch)
                    lv = 0
                    for b, c in enumerate(ch):
                        if c:
                            nb = q + (-1 if c == 1 else 1) * strides[b]
                            lv = max(lv, level[nb])
                    level[q] = lv + 1
                    state[q] = FRONT
                    heapq.heappush(heap, (t0f[q] * tau1[q], q))
    return dict(tau1=tau1, tau=t0f * tau1, t0=t0f, p0=p0f, order=np.array(order, dtype=np.int64),
                dir=direction, level=level, shape=shape, h=h, src=s)


def _rows(fm, tau1_used):
    """Per node: diagonal and (neighbour, coefficient) pairs of the matrix
    M = sum_a diag(2 D_a tau1) D_a (Eq. Sensitivity2), D_a as chosen by FM;
    the source row is 2 tau1_s (reading E1)."""
    shape, h = fm["shape"], fm["h"]
    d = len(shape)
    strides = [int(np.prod(shape[a + 1:])) for a in range(d)]
    t0, p0 = fm["t0"], fm["p0"]
    N = t0.size
    diag = np.zeros(N)
    off = [[] for _ in range(N)]
    for i in range(N):
        dv = int(fm["dir"][i])
        if dv == 0xFF:
            diag[i] = 2.0 * tau1_used[i]
            continue
        for a in range(d):
            c = (dv >> (2 * a)) & 3
            if c == 0:
                continue
            nb = i + (-1 if c == 1 else 1) * strides[a]
            # D_a z = alpha z_i - (tau0_i / h) z_nb, alpha = tau0_i/h +- p0
            al = t0[i] / h + p0[a][i] if c == 1 else t0[i] / h - p0[a][i]
            cn = t0[i] / h
            g = al * tau1_used[i] - cn * tau1_used[nb]       # D_a tau1 (sign of the chosen term)
            diag[i] = diag[i] + 2.0 * g * al
            off[i].append((nb, -2.0 * g * cn))
    return diag, off


def sens_matrix(fm, tau1_used=None):
    """Dense M of Eq. Sensitivity2 (small grids): J = M^{-1}."""
    t1 = fm["tau1"] if tau1_used is None else tau1_used
    diag, off = _rows(fm, t1)
    N = diag.size
    M = np.diag(diag)
    for i in range(N):
        for nb, c in off[i]:
            M[i, nb] += c
    return M


def sens_jv(fm, v, tau1_used=None):
    """z = J v: forward substitution in fast-marching order (Eq. Sensitivity2)."""
    t1 = fm["tau1"] if tau1_used is None else tau1_used
    diag, off = _rows(fm, t1)
    z = np.zeros(diag.size)
    for i in fm["order"]:
        acc = v[i]
        for nb, c in off[i]:
            acc = acc - c * z[nb]
        z[i] = acc / diag[i]
    return z


def sens_jtw(fm, w, tau1_used=None):
    """y = J^T w: backward substitution in reverse fast-marching order."""
    t1 = fm["tau1"] if tau1_used is None else tau1_used
    diag, off = _rows(fm, t1)
    y = np.zeros(diag.size)
    acc = np.array(w, dtype=np.float64).copy()
    for i in fm["order"][::-1]:
        y[i] = acc[i] / diag[i]
        for nb, c in off[i]:
            acc[nb] = acc[nb] - c * y[i]
    return y
