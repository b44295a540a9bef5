"""libhelm's C-ABI without a GPU: the library builds, loads, exports every
function include/helm.h declares, and its host-side argument checks work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1607_00968_gb300 import build, helm
    build.build()
    return helm.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "helm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(helm_[a-z_0-9]+)\s*\(", text)))


def test_exports_match_header(lib):
    from paper_1607_00968_gb300 import helm
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []
    assert sorted(helm.EXPORTS) == names


def test_default_params(lib):
    from paper_1607_00968_gb300.helm import HelmParams
    p = HelmParams()
    lib.helm_default_params(ctypes.byref(p))
    assert (p.levels, p.pre, p.post, p.restart) == (3, 2, 2, 10)
    assert p.jacobi_w == pytest.approx(0.8) and p.shift == pytest.approx(0.5)


def test_setup_rejects_bad_arguments_on_host(lib):
    from paper_1607_00968_gb300.helm import HelmParams, HELM_ERR_ARG
    p = HelmParams()
    lib.helm_default_params(ctypes.byref(p))
    p.dim, p.h, p.omega = 2, 1.0, 1.0
    p.n[0], p.n[1] = 30, 16        # 30 not divisible by 2^(3-1)
    ctx = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    st = lib.helm_setup(dummy, dummy, ctypes.byref(p), None, ctypes.byref(ctx))
    assert st == HELM_ERR_ARG and not ctx.value
    assert b"divisible" in lib.helm_last_error(None)
    p.n[0], p.dim = 32, 4
    assert lib.helm_setup(dummy, dummy, ctypes.byref(p), None, ctypes.byref(ctx)) == HELM_ERR_ARG
    p.dim, p.block = 2, 0
    assert lib.helm_setup(dummy, dummy, ctypes.byref(p), None, ctypes.byref(ctx)) == HELM_ERR_ARG
    assert lib.helm_setup(None, dummy, ctypes.byref(p), None, ctypes.byref(ctx)) == HELM_ERR_ARG


def test_null_context_calls_fail_cleanly(lib):
    from paper_1607_00968_gb300.helm import HELM_ERR_ARG
    assert lib.helm_solve(None, None, 1, 1e-6, None, None) == HELM_ERR_ARG
    assert lib.helm_kernel_launches(None) == 0
    lib.helm_destroy(None)


def test_setup_rejects_unsupported_method_combinations(lib):
    from paper_1607_00968_gb300.helm import HelmParams, HELM_ERR_ARG
    p = HelmParams()
    lib.helm_default_params(ctypes.byref(p))
    p.dim, p.h, p.omega = 2, 1.0, 1.0
    p.n[0], p.n[1] = 32, 16
    ctx = ctypes.c_void_p()
    dummy = ctypes.c_void_p(16)
    p.cycle_gamma, p.krylov = 3, 1          # the K-cycle is nonlinear: FGMRES only
    assert lib.helm_setup(dummy, dummy, ctypes.byref(p), None, ctypes.byref(ctx)) == HELM_ERR_ARG
    p.cycle_gamma, p.krylov = 4, 0
    assert lib.helm_setup(dummy, dummy, ctypes.byref(p), None, ctypes.byref(ctx)) == HELM_ERR_ARG
    p.cycle_gamma, p.krylov, p.prec, p.block = 2, 1, 1, 4   # complex64 BiCGSTAB needs block <= 2
    assert lib.helm_setup(dummy, dummy, ctypes.byref(p), None, ctypes.byref(ctx)) == HELM_ERR_ARG
    p.cycle_gamma, p.krylov, p.prec, p.block = 1, 0, 2, 4   # learned stage without weights
    assert lib.helm_setup(dummy, dummy, ctypes.byref(p), None, ctypes.byref(ctx)) == HELM_ERR_ARG
    assert not ctx.value


def test_eikonal_and_profiler_argument_checks(lib):
    from paper_1607_00968_gb300.helm import HELM_ERR_ARG
    e = ctypes.c_void_p()
    n = (ctypes.c_int * 3)(16, 8, 0)
    assert lib.helm_eik_create(4, n, 10.0, 1, None, ctypes.byref(e)) == HELM_ERR_ARG
    assert lib.helm_eik_create(2, None, 10.0, 1, None, ctypes.byref(e)) == HELM_ERR_ARG
    assert lib.helm_eik_create(2, n, 0.0, 1, None, ctypes.byref(e)) == HELM_ERR_ARG
    assert lib.helm_eik_create(2, n, 10.0, 0, None, ctypes.byref(e)) == HELM_ERR_ARG
    bad = (ctypes.c_int * 3)(16, 0, 0)
    assert lib.helm_eik_create(2, bad, 10.0, 1, None, ctypes.byref(e)) == HELM_ERR_ARG
    assert not e.value
    assert lib.helm_eik_forward(None, None, None, 1, None, None, None, None) == HELM_ERR_ARG
    assert lib.helm_eik_jv(None, None, None) == HELM_ERR_ARG
    assert lib.helm_eik_jtw(None, None, None) == HELM_ERR_ARG
    assert lib.helm_eik_last_error(None) == b""
    lib.helm_eik_destroy(None)
    assert lib.helm_profile_enable(None, 1) == HELM_ERR_ARG
    assert lib.helm_profile_select(None, 0) == HELM_ERR_ARG
