"""GB300-native multi-source Helmholtz solver: shifted-Laplacian multigrid
preconditioned block FGMRES behind the C-ABI of ``include/helm.h``.

``paper_1607_00968_gb300.helm`` is the Python binding (ctypes) of libhelm;
``paper_1607_00968_gb300.inputs`` builds seeded synthetic problems;
``paper_1607_00968_gb300.build`` compiles libhelm for sm_103a.
"""
__all__ = ["helm", "inputs", "build"]
