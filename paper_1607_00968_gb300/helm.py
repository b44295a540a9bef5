"""Thin ctypes binding of libhelm (see include/helm.h).

Argument marshalling only: every step of a solve runs in libhelm's CUDA
kernels and its C++ driver.  PyTorch provides device memory and the CUDA
stream.  There is no CPU fallback: if libhelm.so is missing or no CUDA
device is present, constructing a :class:`Solver` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhelm.so")

HELM_OK, HELM_ERR_ARG, HELM_ERR_NOMEM, HELM_ERR_CUDA = 0, 1, 2, 3
HELM_NOT_CONVERGED, HELM_ERR_NONFINITE, HELM_ERR_BREAKDOWN = 4, 5, 6
STATUS_NAMES = {0: "HELM_OK", 1: "HELM_ERR_ARG", 2: "HELM_ERR_NOMEM", 3: "HELM_ERR_CUDA",
                4: "HELM_NOT_CONVERGED", 5: "HELM_ERR_NONFINITE", 6: "HELM_ERR_BREAKDOWN"}
PREC = {"c128": 0, "plain": 0, "c64": 1, "mixed": 1, "learned": 2}

# names the header declares (checked by the CPU tests)
EXPORTS = ["helm_default_params", "helm_setup", "helm_solve", "helm_adjoint", "helm_solve_host",
           "helm_solve_batch", "helm_destroy", "helm_last_error", "helm_level_shape",
           "helm_apply", "helm_smooth", "helm_restrict_residual", "helm_prolong_add",
           "helm_coarse_solve", "helm_vcycle", "helm_get_operator", "helm_kernel_launches",
           "helm_orth_stats",
           "helm_profile_enable", "helm_profile_select", "helm_profile_kernel_count",
           "helm_profile_kernel_name",
           "helm_profile_read", "helm_vcycle_noalloc", "helm_learned_layers",
           "helm_learned_blob_bytes", "helm_learned_layer", "helm_conv3x3", "helm_conv3x3_wgrad",
           "helm_conv3x3_flip", "helm_adam", "helm_learned_input", "helm_learned_target",
           "helm_learned_loss", "helm_learned_residual_input", "helm_learned_residual_loss",
           "helm_learned_image_to_block", "helm_fields_to_half", "helm_fwi_jv", "helm_fwi_jtw",
           "helm_fwi_gradient", "helm_eik_create", "helm_eik_forward", "helm_eik_jv", "helm_eik_jtw",
           "helm_eik_last_error", "helm_eik_destroy"]


class HelmParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double),
                ("omega", ctypes.c_double), ("shift", ctypes.c_double),
                ("levels", ctypes.c_int), ("pre", ctypes.c_int), ("post", ctypes.c_int),
                ("jacobi_w", ctypes.c_double), ("restart", ctypes.c_int),
                ("block", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("prec", ctypes.c_int), ("learned_weights", ctypes.c_void_p),
                ("coarse_tf32x3", ctypes.c_int), ("cycle_gamma", ctypes.c_int),
                ("krylov", ctypes.c_int), ("graphs", ctypes.c_int), ("orth", ctypes.c_int)]


class HelmInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.POINTER(ctypes.c_int)),
                ("relres", ctypes.POINTER(ctypes.c_double)),
                ("status", ctypes.POINTER(ctypes.c_int))]


class HelmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhelm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libhelm.so not built: run `python -c \"import __graft_entry__ as g; "
                          "g.build()\"` (expected at %s)" % path)
    lib = ctypes.CDLL(path)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    P = ctypes.POINTER
    sig = {
        "helm_default_params": (None, [P(HelmParams)]),
        "helm_setup": (i, [vp, vp, P(HelmParams), vp, P(vp)]),
        "helm_solve": (i, [vp, vp, i, d, vp, P(HelmInfo)]),
        "helm_adjoint": (i, [vp, vp, i, d, vp, P(HelmInfo)]),
        "helm_solve_host": (i, [vp, vp, i, d, vp, P(HelmInfo)]),
        "helm_solve_batch": (i, [P(vp), P(vp), P(i), i, d, P(vp), P(HelmInfo)]),
        "helm_destroy": (None, [vp]),
        "helm_last_error": (ctypes.c_char_p, [vp]),
        "helm_level_shape": (i, [vp, i, P(i), P(ll)]),
        "helm_apply": (i, [vp, i, i, i, vp, vp, i]),
        "helm_smooth": (i, [vp, i, i, vp, vp, vp, i, i]),
        "helm_restrict_residual": (i, [vp, i, i, vp, vp, vp, i]),
        "helm_prolong_add": (i, [vp, i, i, vp, vp, i]),
        "helm_coarse_solve": (i, [vp, i, vp, vp, i]),
        "helm_vcycle": (i, [vp, i, vp, vp, i]),
        "helm_vcycle_noalloc": (i, [vp, i, vp, vp, i]),
        "helm_get_operator": (i, [vp, i, vp]),
        "helm_kernel_launches": (ll, [vp]),
        "helm_orth_stats": (i, [vp, P(ll), P(ll), P(ll)]),
        "helm_profile_enable": (i, [vp, i]),
        "helm_profile_select": (i, [vp, i]),
        "helm_profile_kernel_count": (i, []),
        "helm_profile_kernel_name": (ctypes.c_char_p, [i]),
        "helm_profile_read": (i, [vp, i, P(d), P(ll), P(d), P(d)]),
        "helm_learned_layers": (i, []),
        "helm_learned_blob_bytes": (ll, []),
        "helm_learned_layer": (i, [i, P(i), P(i), P(i), P(ll), P(ll)]),
        "helm_conv3x3": (i, [vp, i, i, i, i, vp, vp, i, i, vp, vp, i, vp]),
        "helm_conv3x3_wgrad": (i, [vp, vp, i, i, i, i, i, vp, vp, vp]),
        "helm_conv3x3_flip": (i, [vp, i, i, vp, i, vp]),
        "helm_adam": (i, [vp, vp, vp, vp, vp, i, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                          ctypes.c_float, i, vp]),
        "helm_learned_input": (i, [vp, vp, vp, i, vp, vp]),
        "helm_learned_target": (i, [vp, ll, i, vp, ctypes.c_float, vp, vp]),
        "helm_learned_loss": (i, [vp, vp, i, ll, vp, vp, vp, vp]),
        "helm_learned_residual_input": (i, [vp, vp, vp, i, vp, vp, vp, vp]),
        "helm_learned_residual_loss": (i, [vp, vp, vp, i, i, i, vp, vp, vp, vp, vp]),
        "helm_learned_image_to_block": (i, [vp, ll, i, vp, vp]),
        "helm_fields_to_half": (i, [vp, ll, i, vp, vp]),
        "helm_fwi_jv": (i, [vp, vp, i, i, vp, vp, i, d, vp]),
        "helm_fwi_jtw": (i, [vp, vp, i, i, vp, vp, i, d, vp]),
        "helm_fwi_gradient": (i, [vp, vp, i, vp, vp, i, d, i, vp, P(d), vp]),
        "helm_eik_create": (i, [i, P(i), d, i, vp, P(vp)]),
        "helm_eik_forward": (i, [vp, vp, P(i), i, vp, vp, vp, vp]),
        "helm_eik_jv": (i, [vp, vp, vp]),
        "helm_eik_jtw": (i, [vp, vp, vp]),
        "helm_eik_last_error": (ctypes.c_char_p, [vp]),
        "helm_eik_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Info:
    """Per-column results of a solve (host numpy arrays).  They start as
    iters -1, relres NaN, status -1, so a column the library never reached
    (a call that failed before solving) cannot pass for converged."""

    def __init__(self, s):
        self.iters = np.full(s, -1, dtype=np.int32)
        self.relres = np.full(s, np.nan, dtype=np.float64)
        self.status = np.full(s, -1, dtype=np.int32)

    def c_struct(self):
        return HelmInfo(self.iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        self.relres.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        self.status.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))


def solve_batch(solvers, Qs, tol: float = 1e-6, check: bool = True):
    """helm_solve_batch over several Solvers (each ideally on its own stream).
    Qs: list of (s_k, N_k) complex128 device tensors.  Returns (Us, infos,
    status)."""
    import torch
    lib = load()
    n = len(solvers)
    Qs = [S._block(Q) for S, Q in zip(solvers, Qs)]
    Us = [torch.empty_like(Q) for Q in Qs]
    infos = [Info(Q.shape[0]) for Q in Qs]
    cinfo = (HelmInfo * n)(*[i.c_struct() for i in infos])
    ctxs = (ctypes.c_void_p * n)(*[S.ctx.value for S in solvers])
    qp = (ctypes.c_void_p * n)(*[Q.data_ptr() for Q in Qs])
    up = (ctypes.c_void_p * n)(*[U.data_ptr() for U in Us])
    ss = (ctypes.c_int * n)(*[Q.shape[0] for Q in Qs])
    for S in solvers:
        S.stream.synchronize()
    st = lib.helm_solve_batch(ctxs, qp, ss, n, float(tol), up, cinfo)
    if check and st != HELM_OK:
        raise HelmError(st, lib.helm_last_error(None).decode())
    return Us, infos, st


class Solver:
    """A set-up Helmholtz hierarchy on the current CUDA device.

    m, gamma: squared slowness and dimensionless attenuation on the nodes
    (numpy array or torch tensor of the node shape, numpy order with x1
    last).  The solve takes and returns torch complex128 tensors of shape
    (s, N) on the device (the ABI's column-major N x s block)."""

    def __init__(self, m, gamma, h: float, omega: float, *, shift: float = 0.5,
                 levels: int = 3, pre: int = 2, post: int = 2, jacobi_w: float = 0.8,
                 restart: int = 10, block: int = 8, max_restarts: int = 50,
                 prec: str = "c128", stream=None, coarse_tf32x3: bool = False,
                 coarse: str = "fp16",
                 learned_weights=None, cycle: str = "V", krylov: str = "fgmres",
                 graphs: str = "auto", orth: str = "selective"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libhelm needs a CUDA device")
        self.lib = load()
        self.torch = torch
        m_t = torch.as_tensor(np.ascontiguousarray(m) if isinstance(m, np.ndarray) else m)
        g_t = torch.as_tensor(np.ascontiguousarray(gamma) if isinstance(gamma, np.ndarray) else gamma)
        self.shape = tuple(m_t.shape)
        dim = len(self.shape)
        if dim not in (2, 3) or tuple(g_t.shape) != self.shape:
            raise ValueError("m and gamma must share a 2D or 3D node shape")
        dev = torch.device("cuda", torch.cuda.current_device())
        self.m = m_t.to(device=dev, dtype=torch.float64).contiguous()
        self.gamma = g_t.to(device=dev, dtype=torch.float64).contiguous()
        p = HelmParams()
        self.lib.helm_default_params(ctypes.byref(p))
        p.dim = dim
        cells = [n - 1 for n in reversed(self.shape)]
        for k in range(3):
            p.n[k] = cells[k] if k < dim else 0
        p.h, p.omega, p.shift = float(h), float(omega), float(shift)
        p.levels, p.pre, p.post, p.jacobi_w = int(levels), int(pre), int(post), float(jacobi_w)
        p.restart, p.block, p.max_restarts = int(restart), int(block), int(max_restarts)
        p.prec = PREC[prec]
        # complex64 coarsest product: "fp16" (tcgen05), "tf32x3", "fp16_mma_sync"
        p.coarse_tf32x3 = 1 if coarse_tf32x3 else {"fp16": 0, "tf32x3": 1, "fp16_mma_sync": 2}[coarse]
        p.cycle_gamma = {"V": 1, "W": 2, "K": 3}[cycle]
        p.krylov = {"fgmres": 0, "bicgstab": 1}[krylov]
        p.graphs = {"off": 0, "on": 1, "auto": 2}[graphs]
        p.orth = {"selective": 0, "twice": 1}[orth]
        self.learned_weights = learned_weights        # keeps the blob alive
        p.learned_weights = _ptr(learned_weights) if learned_weights is not None else None
        self.params = p
        self.prec = prec
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p()
        st = self.lib.helm_setup(_ptr(self.m), _ptr(self.gamma), ctypes.byref(p),
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if st != HELM_OK:
            raise HelmError(st, self.lib.helm_last_error(None).decode())
        self.ctx = ctx
        self.N = int(np.prod(self.shape))
        self.levels = int(levels)

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.helm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=(HELM_OK,)):
        if st not in allow:
            raise HelmError(st, self.lib.helm_last_error(self.ctx).decode())
        return st

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.helm_kernel_launches(self.ctx))

    def orth_stats(self) -> dict:
        """Block QRs factored since set-up, and how many needed a second
        Gram-Schmidt pass (reorth) or a second Cholesky QR pass (qr2)."""
        qr, re, q2 = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self.lib.helm_orth_stats(self.ctx, ctypes.byref(qr), ctypes.byref(re),
                                             ctypes.byref(q2)))
        return {"qr": qr.value, "reorth": re.value, "qr2": q2.value}

    # -- solves ----------------------------------------------------------
    def _block(self, Q):
        torch = self.torch
        Q = torch.as_tensor(Q)
        if Q.dim() == 1:
            Q = Q[None]
        if Q.shape[-1] != self.N:
            raise ValueError("right-hand sides must have shape (s, N)")
        return Q.to(device=self.m.device, dtype=torch.complex128).contiguous()

    def solve(self, Q, tol: float = 1e-6, adjoint: bool = False, check: bool = True):
        """U = A^{-1} Q (or A^{-H} Q).  Returns (U, Info, status)."""
        Q = self._block(Q)
        s = Q.shape[0]
        U = self.torch.empty_like(Q)
        info = Info(s)
        ci = info.c_struct()
        fn = self.lib.helm_adjoint if adjoint else self.lib.helm_solve
        st = fn(self.ctx, _ptr(Q), s, float(tol), _ptr(U), ctypes.byref(ci))
        if check:
            self._check(st, (HELM_OK,))
        return U, info, st

    def adjoint(self, B, tol: float = 1e-6, check: bool = True):
        return self.solve(B, tol, adjoint=True, check=check)

    def solve_host(self, Q_host, U_host, tol: float = 1e-6, check: bool = True):
        """Host complex128 buffers (torch CPU tensors, ideally pinned), shape (s, N)."""
        s = Q_host.shape[0]
        info = Info(s)
        ci = info.c_struct()
        st = self.lib.helm_solve_host(self.ctx, _ptr(Q_host), s, float(tol), _ptr(U_host),
                                      ctypes.byref(ci))
        if check:
            self._check(st, (HELM_OK,))
        return info, st

    # -- FWI sensitivities ----------------------------------------------------
    def fwi_gradient(self, Q, d_obs, recv, tol=1e-8, store_half=False):
        """(misfit, grad (N,) float64 device tensor, U (s, N)) for sources Q
        (s, N), data d_obs (s, nrec) and receiver node indices recv."""
        torch = self.torch
        Q = self._block(Q)
        s = Q.shape[0]
        recv = torch.as_tensor(recv, dtype=torch.int32, device=Q.device)
        d_obs = torch.as_tensor(d_obs).to(device=Q.device, dtype=torch.complex128).contiguous()
        grad = torch.empty(self.N, dtype=torch.float64, device=Q.device)
        U = torch.empty_like(Q)
        phi = ctypes.c_double()
        self._check(self.lib.helm_fwi_gradient(self.ctx, _ptr(Q), s, _ptr(d_obs), _ptr(recv),
                                               recv.numel(), float(tol), 1 if store_half else 0,
                                               _ptr(grad), ctypes.byref(phi), _ptr(U)))
        return phi.value, grad, U

    def fwi_jv(self, U, v, recv, tol=1e-8, half=False):
        torch = self.torch
        recv = torch.as_tensor(recv, dtype=torch.int32, device=U.device)
        v = torch.as_tensor(v).to(device=U.device, dtype=torch.float64).contiguous()
        s = U.shape[0]
        out = torch.empty((s, recv.numel()), dtype=torch.complex128, device=U.device)
        self._check(self.lib.helm_fwi_jv(self.ctx, _ptr(U), 1 if half else 0, s, _ptr(v), _ptr(recv),
                                         recv.numel(), float(tol), _ptr(out)))
        return out

    def fwi_jtw(self, U, W, recv, tol=1e-8, half=False):
        torch = self.torch
        recv = torch.as_tensor(recv, dtype=torch.int32, device=U.device)
        W = torch.as_tensor(W).to(device=U.device, dtype=torch.complex128).contiguous()
        s = U.shape[0]
        out = torch.empty(self.N, dtype=torch.float64, device=U.device)
        self._check(self.lib.helm_fwi_jtw(self.ctx, _ptr(U), 1 if half else 0, s, _ptr(W), _ptr(recv),
                                          recv.numel(), float(tol), _ptr(out)))
        return out

    def fields_to_half(self, U):
        torch = self.torch
        out = torch.empty(U.shape + (2,), dtype=torch.float16, device=U.device)
        self._check(self.lib.helm_fields_to_half(_ptr(U), self.N, U.shape[0], _ptr(out),
                                                 ctypes.c_void_p(self.stream.cuda_stream)))
        return out

    # -- profiler ----------------------------------------------------------
    def profile(self, enable: bool = True, only: str | None = None):
        """Enable (and reset) or disable the per-kernel profiler; `only`
        restricts the recording to one kernel class (a profile_read name)."""
        self._check(self.lib.helm_profile_enable(self.ctx, 1 if enable else 0))
        if enable and only is not None:
            names = [self.lib.helm_profile_kernel_name(k).decode()
                     for k in range(self.lib.helm_profile_kernel_count())]
            self._check(self.lib.helm_profile_select(self.ctx, names.index(only)))

    def profile_read(self) -> dict:
        """{kernel name: dict(time_ms, launches, bytes, flops)} since enabling."""
        out = {}
        for k in range(self.lib.helm_profile_kernel_count()):
            t, b, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            n = ctypes.c_longlong()
            self._check(self.lib.helm_profile_read(self.ctx, k, ctypes.byref(t), ctypes.byref(n),
                                                   ctypes.byref(b), ctypes.byref(f)))
            out[self.lib.helm_profile_kernel_name(k).decode()] = dict(
                time_ms=t.value, launches=n.value, bytes=b.value, flops=f.value)
        return out

    # -- components (internal layout (N_l, s)) ---------------------------
    def level_shape(self, level: int):
        nodes = (ctypes.c_int * 3)()
        cnt = ctypes.c_longlong()
        self._check(self.lib.helm_level_shape(self.ctx, level, nodes, ctypes.byref(cnt)))
        return tuple(nodes), int(cnt.value)

    def _prec(self, x):
        torch = self.torch
        if x.dtype == torch.complex128:
            return 0
        if x.dtype == torch.complex64:
            return 1
        raise TypeError("complex128 or complex64 tensors expected")

    def apply(self, x, level: int = 0, op: str = "A"):
        y = self.torch.empty_like(x)
        self._check(self.lib.helm_apply(self.ctx, level, 0 if op == "A" else 1, self._prec(x),
                                        _ptr(x), _ptr(y), x.shape[1]))
        return y

    def smooth(self, f, u=None, level: int = 0, sweeps: int = 1):
        out = self.torch.empty_like(f)
        self._check(self.lib.helm_smooth(self.ctx, level, self._prec(f), _ptr(u), _ptr(f),
                                         _ptr(out), f.shape[1], sweeps))
        return out

    def restrict_residual(self, u, f, level: int = 0):
        _, nc = self.level_shape(level + 1)
        rc = self.torch.empty((nc, f.shape[1]), dtype=f.dtype, device=f.device)
        self._check(self.lib.helm_restrict_residual(self.ctx, level, self._prec(f), _ptr(u),
                                                    _ptr(f), _ptr(rc), f.shape[1]))
        return rc

    def prolong_add(self, ec, u, level: int = 0):
        self._check(self.lib.helm_prolong_add(self.ctx, level, self._prec(u), _ptr(ec), _ptr(u),
                                              u.shape[1]))
        return u

    def coarse_solve(self, f):
        u = self.torch.empty_like(f)
        self._check(self.lib.helm_coarse_solve(self.ctx, self._prec(f), _ptr(f), _ptr(u),
                                               f.shape[1]))
        return u

    def vcycle(self, f, prec: str = "c128"):
        torch = self.torch
        f = f.to(torch.complex128).contiguous()
        z = torch.empty(f.shape, dtype=torch.complex128 if PREC[prec] == 0 else torch.complex64,
                        device=f.device)
        self._check(self.lib.helm_vcycle(self.ctx, PREC[prec], _ptr(f), _ptr(z), f.shape[1]))
        return z

    def operator(self, level: int):
        """FP64 K-point stencil of M_level, numpy (N_l, K)."""
        _, n = self.level_shape(level)
        K = 27 if len(self.shape) == 3 else 9
        out = np.zeros((n, K), dtype=np.complex128)
        self._check(self.lib.helm_get_operator(self.ctx, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out


class Eikonal:
    """Factored-eikonal fast marching and its sensitivities on the GPU
    (helm_eik_*).

    shape: node shape in numpy order (x1 last), as Solver's m; h: spacing;
    ns_max: most sources per forward call.  Sources are node multi-indices in
    numpy order; m is the squared slowness (numpy or torch, node shape)."""

    def __init__(self, shape, h: float, ns_max: int, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libhelm needs a CUDA device")
        self.lib = load()
        self.torch = torch
        self.shape = tuple(int(n) for n in shape)
        self.d = len(self.shape)
        if self.d not in (2, 3):
            raise ValueError("2D or 3D node shape")
        self.N = int(np.prod(self.shape))
        cells = (ctypes.c_int * 3)(*([n - 1 for n in reversed(self.shape)] + [0] * (3 - self.d)))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        e = ctypes.c_void_p()
        st = self.lib.helm_eik_create(self.d, cells, float(h), int(ns_max),
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(e))
        if st != HELM_OK:
            raise HelmError(st, self.lib.helm_last_error(None).decode())
        self.e = e
        self.ns = 0

    def _check(self, st):
        if st != HELM_OK:
            raise HelmError(st, self.lib.helm_eik_last_error(self.e).decode())

    def forward(self, m, sources, outputs=("tau", "tau1", "order", "dir")):
        """Fast marching for every source; returns a dict of the requested
        device outputs, each (ns, N): tau, tau1 (float64), order (int32),
        dir (uint8)."""
        torch = self.torch
        dev = torch.device("cuda", torch.cuda.current_device())
        mt = torch.as_tensor(np.ascontiguousarray(m) if isinstance(m, np.ndarray) else m)
        mt = mt.to(device=dev, dtype=torch.float64).contiguous().reshape(-1)
        if mt.numel() != self.N:
            raise ValueError("m must have the node shape")
        ns = len(sources)
        src = (ctypes.c_int * (ns * self.d))()
        for b, sidx in enumerate(sources):
            for k in range(self.d):                       # ABI order (x1, x2[, x3])
                src[b * self.d + k] = int(sidx[self.d - 1 - k])
        out = {}
        kinds = {"tau": torch.float64, "tau1": torch.float64, "order": torch.int32, "dir": torch.uint8}
        for k in outputs:
            out[k] = torch.empty((ns, self.N), dtype=kinds[k], device=dev)
        self._m = mt
        self._check(self.lib.helm_eik_forward(self.e, _ptr(mt), src, ns, _ptr(out.get("tau")),
                                              _ptr(out.get("tau1")), _ptr(out.get("order")),
                                              _ptr(out.get("dir"))))
        self.ns = ns
        return out

    def jv(self, v):
        """z (ns, N) = J_s v for the sources of the last forward call."""
        torch = self.torch
        vt = torch.as_tensor(v).to(device="cuda", dtype=torch.float64).contiguous().reshape(-1)
        z = torch.empty((self.ns, self.N), dtype=torch.float64, device=vt.device)
        self._check(self.lib.helm_eik_jv(self.e, _ptr(vt), _ptr(z)))
        return z

    def jtw(self, w):
        """y (ns, N) = J_s^T w_s, w of shape (ns, N)."""
        torch = self.torch
        wt = torch.as_tensor(w).to(device="cuda", dtype=torch.float64).contiguous()
        y = torch.empty((self.ns, self.N), dtype=torch.float64, device=wt.device)
        self._check(self.lib.helm_eik_jtw(self.e, _ptr(wt), _ptr(y)))
        return y

    def close(self):
        if getattr(self, "e", None):
            self.lib.helm_eik_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
