"""Host-side pieces of the benchmark and the binding, on CPU: the uneven
batch's level and cycle rule, the double-float peak, and the binding's
per-column result arrays (no GPU needed)."""
import numpy as np
import pytest

from paper_1607_00968_gb300 import inputs as I


def test_batch_levels_and_cycles():
    """The batch's grids get the fewest levels with a coarsest grid of at most
    9,000 nodes: never five (the 1024 x 512 grid stops at 129 x 65 = 8,385
    nodes), every coarsening even, and the K-cycle exactly from four levels."""
    for cells, want in (((256, 128), 2), ((512, 256), 3), ((1024, 512), 4)):
        lv = I.default_levels(cells, 9000)
        assert lv == want, (cells, lv)
        c = [n // 2 ** (lv - 1) for n in cells]
        assert all(n % 2 ** (lv - 1) == 0 for n in cells)
        assert np.prod([n + 1 for n in c]) <= 9000
        cycle = "K" if lv >= 4 else "V"
        assert (cycle == "K") == (cells == (1024, 512))


def test_double_float_peak_formula():
    import bench
    # 152 SMs x 128 lanes x 2070 MHz / 48 instructions per complex MAC x 8 flops
    assert abs(bench.dd_peak_tflops(152, 2070.0) - 6.7133) < 1e-3
    assert abs(bench.dd_peak_tflops(76, 2070.0) - bench.dd_peak_tflops(152, 2070.0) / 2) < 1e-12


def test_headline_convergence_rule():
    """The bench counts a solve only when every column ended at true relres
    <= tol with status OK; one column above tol, one non-OK status, or one
    column the library never reached withholds it."""
    import bench
    from paper_1607_00968_gb300 import helm
    tol = 1e-6
    ok = helm.Info(4)
    ok.iters[:] = 10
    ok.relres[:] = [1e-7, 5e-7, 1e-6, 0.0]       # tol itself and a zero column count
    ok.status[:] = 0
    assert bench.converged(ok, tol)
    above = helm.Info(4)
    above.relres[:] = [1e-7, 1.0000001e-6, 1e-7, 1e-7]
    above.status[:] = 0
    assert not bench.converged(above, tol)
    flagged = helm.Info(2)
    flagged.relres[:] = 1e-8
    flagged.status[:] = [0, 1]                   # HELM_NOT_CONVERGED on one column
    assert not bench.converged(flagged, tol)
    unreached = helm.Info(3)                     # NaN / -1 sentinels
    assert not bench.converged(unreached, tol)
    partial = helm.Info(3)
    partial.relres[:2] = 1e-8
    partial.status[:2] = 0                       # the third column never written
    assert not bench.converged(partial, tol)


def test_info_starts_unconverged():
    """A column the library never reached cannot pass for converged: the
    binding's result arrays start as iters -1, relres NaN, status -1."""
    from paper_1607_00968_gb300 import helm
    info = helm.Info(3)
    assert np.all(info.iters == -1)
    assert np.all(np.isnan(info.relres))
    assert np.all(info.status == -1)
    assert not np.any(info.relres <= 1e-6)
