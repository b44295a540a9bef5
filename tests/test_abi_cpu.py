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


def test_every_context_call_rejects_a_null_context(lib):
    """Each entry point that takes a context returns HELM_ERR_ARG for NULL
    before any CUDA work (these run without a GPU)."""
    from paper_1607_00968_gb300.helm import HELM_ERR_ARG
    calls = {
        "helm_adjoint": (None, None, 1, 1e-6, None, None),
        "helm_solve_host": (None, None, 1, 1e-6, None, None),
        "helm_level_shape": (None, 0, None, None),
        "helm_apply": (None, 0, 1, 0, None, None, 1),
        "helm_smooth": (None, 0, 0, None, None, None, 1, 1),
        "helm_restrict_residual": (None, 0, 0, None, None, None, 1),
        "helm_prolong_add": (None, 0, 0, None, None, 1),
        "helm_coarse_solve": (None, 0, None, None, 1),
        "helm_vcycle": (None, 0, None, None, 1),
        "helm_vcycle_noalloc": (None, 0, None, None, 1),
        "helm_get_operator": (None, 0, None),
        "helm_orth_stats": (None, None, None, None),
        "helm_profile_read": (None, 0, None, None, None, None),
        "helm_learned_input": (None, None, None, 1, None, None),
        "helm_learned_residual_input": (None, None, None, 1, None, None, None, None),
        "helm_fwi_jv": (None, None, 0, 1, None, None, 1, 1e-6, None),
        "helm_fwi_jtw": (None, None, 0, 1, None, None, 1, 1e-6, None),
        "helm_fwi_gradient": (None, None, 1, None, None, 1, 1e-6, 0, None, None, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == HELM_ERR_ARG, name
    assert b"helm_fwi_gradient" in lib.helm_last_error(None)
    # batches: a negative count, missing arrays, a NULL context inside
    assert lib.helm_solve_batch(None, None, None, -1, 1e-6, None, None) == HELM_ERR_ARG
    assert lib.helm_solve_batch(None, None, None, 1, 1e-6, None, None) == HELM_ERR_ARG
    vp = ctypes.c_void_p
    ctxs, qs, us = (vp * 1)(None), (vp * 1)(None), (vp * 1)(None)
    ss = (ctypes.c_int * 1)(1)
    assert lib.helm_solve_batch(ctxs, qs, ss, 1, 1e-6, us, None) == HELM_ERR_ARG
    assert b"bad problem" in lib.helm_last_error(None)


def test_context_free_kernels_reject_null_pointers(lib):
    """The learned-stage, FWI-storage and layer-table entry points check their
    pointers and sizes on the host."""
    from paper_1607_00968_gb300.helm import HELM_ERR_ARG, HELM_OK
    assert lib.helm_conv3x3(None, 1, 8, 8, 16, None, None, 32, 1, None, None, 0, None) == HELM_ERR_ARG
    assert lib.helm_conv3x3_wgrad(None, None, 1, 8, 8, 16, 32, None, None, None) == HELM_ERR_ARG
    assert lib.helm_conv3x3_flip(None, 16, 32, None, 16, None) == HELM_ERR_ARG
    assert lib.helm_adam(None, None, None, None, None, 1, 1e-3, 0.9, 0.999, 1e-8, 1, None) == HELM_ERR_ARG
    assert lib.helm_learned_target(None, 1, 1, None, 1.0, None, None) == HELM_ERR_ARG
    assert lib.helm_learned_loss(None, None, 1, 1, None, None, None, None) == HELM_ERR_ARG
    assert lib.helm_learned_residual_loss(None, None, None, 1, 8, 8, None, None, None, None,
                                          None) == HELM_ERR_ARG
    assert lib.helm_learned_image_to_block(None, 1, 1, None, None) == HELM_ERR_ARG
    assert lib.helm_fields_to_half(None, 1, 1, None, None) == HELM_ERR_ARG
    # the layer table is host data
    n = lib.helm_learned_layers()
    assert n == 6
    for layer in (-1, n):
        assert lib.helm_learned_layer(layer, None, None, None, None, None) == HELM_ERR_ARG
    cin, cout, relu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    woff, boff = ctypes.c_longlong(), ctypes.c_longlong()
    ends = []
    for layer in range(n):
        assert lib.helm_learned_layer(layer, ctypes.byref(cin), ctypes.byref(cout), ctypes.byref(relu),
                                      ctypes.byref(woff), ctypes.byref(boff)) == HELM_OK
        assert cin.value >= 1 and cout.value >= 1
        assert relu.value == (1 if layer < n - 1 else 0)      # ReLU between layers only
        ends.append((woff.value, boff.value))
    assert all(a < b for a, b in zip(ends, ends[1:]))           # offsets increase through the blob
    assert lib.helm_profile_kernel_count() > 0
    assert lib.helm_profile_kernel_name(-1) == b""


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
