"""helm_vcycle_noalloc against helm_vcycle, through the C-ABI.

helm_vcycle_noalloc serves callers that cannot allocate device memory when
they run the preconditioner (latency-bound loops that cannot afford the
synchronisation an allocation may cause, or a framework allocator that owns
the device): its level buffers live in a fixed device array inside libhelm.  Its result must
equal helm_vcycle's on the same context and input, on consecutive calls (the
array keeps the previous call's contents), and it must refuse a block that
needs more than the array holds.  This file is named to run last.
"""
import ctypes

import numpy as np
import pytest

from paper_1607_00968_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _solver(cells=(64, 32), levels=3):
    from paper_1607_00968_gb300 import helm
    v = I.layered_velocity_2d(0, cells)
    shape = I.node_shape(cells)
    return helm, helm.Solver(1.0 / v ** 2, I.absorbing_gamma(shape, 6), 25.0,
                             I.omega_for_ppw(25.0), levels=levels)


def _noalloc(helm, S, f, prec):
    z = torch.empty(f.shape, device=f.device,
                    dtype=torch.complex128 if prec == 0 else torch.complex64)
    st = S.lib.helm_vcycle_noalloc(S.ctx, prec, ctypes.c_void_p(f.data_ptr()),
                                   ctypes.c_void_p(z.data_ptr()), f.shape[1])
    return st, z


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-5)])
def test_noalloc_vcycle_matches_vcycle_twice(prec, tol):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    helm, S = _solver()
    rng = np.random.default_rng(20)
    for call in range(2):
        s = 6 if call == 0 else 3          # second call: different block, stale array contents
        f = torch.as_tensor(rng.standard_normal((S.N, s)) + 1j * rng.standard_normal((S.N, s))).cuda()
        ref = S.vcycle(f, "c128" if prec == 0 else "c64").cpu().numpy()
        st, z = _noalloc(helm, S, f, prec)
        assert st == helm.HELM_OK, S.lib.helm_last_error(S.ctx)
        got = z.cpu().numpy()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    S.close()


def test_noalloc_rejects_oversized_block():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    helm, S = _solver(cells=(512, 256), levels=4)
    s = 64                                   # 2 x 131841 x 64 x 16 B alone exceed 64 MiB
    f = torch.zeros((S.N, s), dtype=torch.complex128, device="cuda")
    st, _ = _noalloc(helm, S, f, 0)
    assert st == helm.HELM_ERR_ARG
    assert b"64 MiB" in S.lib.helm_last_error(S.ctx) or b"scratch" in S.lib.helm_last_error(S.ctx)
    S.close()
