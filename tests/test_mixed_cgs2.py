"""The arithmetic argument behind the complex64 path's block Gram-Schmidt
(block CGS2 against an orthonormal basis V, Sec. 5.3 block FGMRES), checked
on the CPU with numpy in plain IEEE arithmetic:

* the first pass may take its coefficients H1 in FP32 from the FP32-rounded
  operands (the hi parts of the float pairs), because the second pass, with
  accurate coefficients H2 = V^H (W - V H1), removes that error: H1 + H2
  equals V^H W to FP64-class accuracy and the result is orthogonal to V at
  the level of an accurate single pass;
* the second update V H2 may be formed in FP32 and added to the accurate
  W - V H1, because |H2| is the first pass's small error: the update error
  is ~1e-7 of a term ~1e-6 of |W|;
* a second QR factor T2 within 1e-7 of the identity may be applied as
  W2 + W2 (T2 - I) with the correction in FP32.

The GPU kernels implement these steps in double-float arithmetic; this file
pins the claim that the FP32 pieces cost no FP64-class accuracy.
"""
import numpy as np
import pytest


def orthonormal(rng, n, k):
    q, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    return q


def f32(a):
    return a.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("sine", [1.0, 1e-3, 1e-6])
def test_fp32_first_pass_is_corrected_by_the_second(sine):
    rng = np.random.default_rng(0)
    n, k, s = 4000, 12, 4
    V = orthonormal(rng, n, k)
    C = rng.standard_normal((k, s)) + 1j * rng.standard_normal((k, s))
    P = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
    P -= V @ (V.conj().T @ P)
    P -= V @ (V.conj().T @ P)
    W = V @ C + sine * np.linalg.norm(V @ C) / np.linalg.norm(P) * P   # angle ~ sine to span(V)
    # pass 1: FP32 products of FP32-rounded operands, FP32 accumulation
    H1 = (f32(V).conj().T.astype(np.complex64) @ f32(W).astype(np.complex64)).astype(np.complex128)
    W1 = W - V @ H1                                     # accurate update
    # pass 2: accurate coefficients; the update in FP32 from the hi parts
    H2 = V.conj().T @ W1
    upd = (f32(V).astype(np.complex64) @ f32(H2).astype(np.complex64)).astype(np.complex128)
    W2 = W1 - upd
    exact_H = V.conj().T @ W
    nW = np.linalg.norm(W)
    assert np.linalg.norm(H1 + H2 - exact_H) <= 1e-14 * nW
    assert np.linalg.norm(H2) <= 1e-5 * nW                       # the first pass's error is small
    # orthogonality at the level of one accurate pass: eps * |W| / |W_perp|
    w_perp = np.linalg.norm(W - V @ exact_H)
    assert np.linalg.norm(V.conj().T @ W2) <= 1e-13 * nW
    # the result is the exact projection up to a tiny fraction of |W|
    assert np.linalg.norm(W2 - (W - V @ exact_H)) <= 1e-13 * nW
    assert w_perp > 0


def test_second_qr_factor_as_fp32_correction():
    rng = np.random.default_rng(1)
    n, s = 5000, 4
    Q = orthonormal(rng, n, s)
    E = 1e-9 * (rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s)))
    W2 = Q @ (np.eye(s) + E)                           # nearly orthonormal, as after a first CholQR
    G = W2.conj().T @ W2
    R2 = np.linalg.cholesky(G).conj().T
    T2 = np.linalg.inv(R2)
    assert np.max(np.abs(T2 - np.eye(s))) <= 1e-7
    exact = W2 @ T2
    corr = (f32(W2).astype(np.complex64) @ (T2 - np.eye(s)).astype(np.complex64)).astype(np.complex128)
    got = W2 + corr
    assert np.linalg.norm(got - exact) <= 1e-14 * np.linalg.norm(exact)
    assert np.linalg.norm(got.conj().T @ got - np.eye(s)) <= 1e-13
