"""Learned preconditioning stage on the GPU against the FP64 oracle
(oracle/conv.py): convolution forward, data and weight gradients, the whole
network's forward/backward, Adam, a short training run, and the solve with
the stage switched on.

Inputs and weights are rounded to bf16 before both sides see them, so the
kernels' only differences from the oracle are FP32 accumulation and (for bf16
outputs) the final rounding: tolerances 2e-5 relative for float outputs,
1e-2 for bf16 activations.
"""
import ctypes

import numpy as np
import pytest

from oracle import conv as C
from oracle import helmholtz as O
from paper_1607_00968_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00968_gb300 import helm
    return helm.load()


def vp(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def bf(a):
    """numpy float -> (bf16 device tensor, its exact float64 values)"""
    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()
    return t, t.float().cpu().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16)])
def test_conv_forward_matches_oracle(lib, cin, cout):
    rng = np.random.default_rng(0)
    B, H, W = 2, 13, 21                    # ragged in both tile directions
    x, x64 = bf(rng.standard_normal((B, H, W, cin)))
    w, w64 = bf(rng.standard_normal((cout, 9, cin)) / np.sqrt(9 * cin))
    bias = torch.as_tensor(rng.standard_normal(cout).astype(np.float32)).cuda()
    y = torch.empty((B, H, W, cout), dtype=torch.float32, device="cuda")
    assert lib.helm_conv3x3(vp(x), B, H, W, cin, vp(w), vp(bias), cout, 0, None, vp(y), 1, stream()) == 0
    ref = C.conv3x3(x64, w64.reshape(cout, 3, 3, cin), bias.cpu().numpy().astype(np.float64))
    assert rel(y.cpu().numpy(), ref) < 2e-5
    yr = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device="cuda")
    assert lib.helm_conv3x3(vp(x), B, H, W, cin, vp(w), vp(bias), cout, 1, None, vp(yr), 0, stream()) == 0
    assert rel(yr.float().cpu().numpy(), np.maximum(ref, 0)) < 1e-2


def test_conv_backward_matches_oracle(lib):
    rng = np.random.default_rng(1)
    B, H, W, cin, cout = 2, 11, 19, 32, 16
    x, x64 = bf(np.maximum(rng.standard_normal((B, H, W, cin)), 0))   # a ReLU output
    w, w64 = bf(rng.standard_normal((cout, 9, cin)) / np.sqrt(9 * cin))
    gy, gy64 = bf(rng.standard_normal((B, H, W, cout)))
    W4 = w64.reshape(cout, 3, 3, cin)
    # data gradient through the flipped weights, masked by the input's ReLU
    wf = torch.empty(cin * 9 * cout, dtype=torch.bfloat16, device="cuda")
    assert lib.helm_conv3x3_flip(vp(w), cin, cout, vp(wf), cin, stream()) == 0
    gx = torch.empty((B, H, W, cin), dtype=torch.float32, device="cuda")
    assert lib.helm_conv3x3(vp(gy), B, H, W, cout, vp(wf), None, cin, 0, vp(x), vp(gx), 1, stream()) == 0
    ref = C.conv3x3_input_grad(gy64, W4) * (x64 > 0)
    assert rel(gx.cpu().numpy(), ref) < 2e-5
    # weight and bias gradients
    dw = torch.zeros(cout * 9 * cin, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    assert lib.helm_conv3x3_wgrad(vp(x), vp(gy), B, H, W, cin, cout, vp(dw), vp(db), stream()) == 0
    rdw, rdb = C.conv3x3_weight_grad(x64, gy64)
    assert rel(dw.cpu().numpy(), rdw.reshape(-1)) < 2e-5
    assert rel(db.cpu().numpy(), rdb) < 2e-5


def test_network_forward_backward_matches_oracle(lib):
    from paper_1607_00968_gb300 import learned
    net = learned.Network(seed=3)
    rng = np.random.default_rng(2)
    B, H, W = 2, 17, 33
    xin = np.zeros((B, H, W, 16))
    xin[..., :3] = rng.standard_normal((B, H, W, 3))
    x, x64 = bf(xin)
    params = []
    for l, t in enumerate(net.layers):
        Wl = net.wbf[l].float().cpu().numpy().astype(np.float64).reshape(t["cout"], 3, 3, t["cin"])
        params.append((Wl, net.b[l].cpu().numpy().astype(np.float64)))
    out, acts = net.forward(x, B, H, W, keep=True)

    def r16(a):   # the kernels store activations and gradients in bf16
        return torch.as_tensor(a.astype(np.float32)).to(torch.bfloat16).double().numpy()

    # oracle pass rounding at the same points as the kernels (the ReLU
    # decisions are then taken on the same values)
    ys = [x64]
    for l, (Wl, bl) in enumerate(params):
        z = C.conv3x3(ys[-1], Wl, bl)
        ys.append(r16(np.maximum(z, 0)) if l < len(params) - 1 else z)
    assert rel(out.cpu().numpy(), ys[-1]) < 5e-3
    assert rel(out.cpu().numpy(), C.forward(x64, params)[-1]) < 5e-2   # vs unrounded FP64
    g = np.zeros((B, H, W, 16))
    g[..., :2] = rng.standard_normal((B, H, W, 2))
    gt, g64 = bf(g)
    net.zero_grad()
    net.backward(acts, gt, B, H, W)
    gg = g64
    for l in range(len(params) - 1, -1, -1):
        rdw, rdb = C.conv3x3_weight_grad(ys[l], gg)
        assert rel(net.dw[l].cpu().numpy(), rdw.reshape(-1)) < 5e-3, l
        assert rel(net.db[l].cpu().numpy(), rdb) < 5e-3, l
        if l > 0:
            gg = r16(C.conv3x3_input_grad(gg, params[l][0]) * (ys[l] > 0))


def test_adam_step(lib):
    rng = np.random.default_rng(4)
    n = 1000
    p0, g0 = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
    p = torch.as_tensor(p0).cuda()
    g = torch.as_tensor(g0).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    pb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    for step in (1, 2):
        assert lib.helm_adam(vp(p), vp(g), vp(m), vp(v), vp(pb), n, 1e-2, 0.9, 0.999, 1e-8, step, stream()) == 0
    # Kingma & Ba: two steps with the same gradient
    mm, vv, pp = np.zeros(n), np.zeros(n), p0.astype(np.float64)
    for step in (1, 2):
        mm = 0.9 * mm + 0.1 * g0
        vv = 0.999 * vv + 0.001 * g0.astype(np.float64) ** 2
        pp = pp - 1e-2 * (mm / (1 - 0.9 ** step)) / (np.sqrt(vv / (1 - 0.999 ** step)) + 1e-8)
    np.testing.assert_allclose(p.cpu().numpy(), pp, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(pb.float().cpu().numpy(), pp, rtol=1e-2, atol=1e-2)


def test_error_loss_kernel_matches_oracle(lib):
    """helm_learned_target and helm_learned_loss (the error loss, kept in the
    ABI beside the residual loss) against oracle/conv.loss and loss_grad."""
    rng = np.random.default_rng(42)
    B, H, W, s = 2, 7, 11, 2
    N = H * W
    e = (rng.standard_normal((N, s)) + 1j * rng.standard_normal((N, s))).astype(np.complex64)
    rho = np.array([0.5, 2.0], dtype=np.float32)
    t = torch.empty((s, N, 2), dtype=torch.float32, device="cuda")
    e_d, rho_d = torch.as_tensor(e).cuda(), torch.as_tensor(rho).cuda()
    assert lib.helm_learned_target(vp(e_d), N, s, vp(rho_d), 0.25, vp(t), stream()) == 0
    tt = t.cpu().numpy().astype(np.float64)
    for j in range(s):
        np.testing.assert_allclose(tt[j, :, 0] + 1j * tt[j, :, 1], 0.25 * e[:, j] / rho[j], rtol=1e-6)
    pred = rng.standard_normal((B, N, 16)).astype(np.float32)
    sums = torch.empty(2 * B, dtype=torch.float32, device="cuda")
    grad = torch.empty((B, N, 16), dtype=torch.bfloat16, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    p_d = torch.as_tensor(pred).cuda()
    assert lib.helm_learned_loss(vp(p_d), vp(t), B, N, vp(sums), vp(grad), vp(loss), stream()) == 0
    pr = pred[..., :2].astype(np.float64).reshape(B, H, W, 2)
    tg = tt.reshape(B, H, W, 2)
    ref = C.loss(pr, tg)
    assert abs(float(loss.item()) - ref) <= 1e-5 * ref
    g = grad.float().cpu().numpy()
    assert rel(g[..., :2].reshape(B, H, W, 2), C.loss_grad(pr, tg)) < 1e-2
    assert not np.any(g[..., 2:])


# --------------------------------------------------------------------------
# residual loss of the corrected iterate
# --------------------------------------------------------------------------

def _pairs32(z):
    return np.stack([z.real, z.imag], axis=-1).astype(np.float32)


def test_residual_loss_kernel_matches_oracle(lib):
    """helm_learned_residual_loss against oracle/conv.residual_loss and its
    gradient on a ragged batch (FP32 loss, bf16 gradient)."""
    rng = np.random.default_rng(40)
    B, H, W = 2, 9, 13
    pred = rng.standard_normal((B, H, W, 16)).astype(np.float32)
    r = rng.standard_normal((B, H, W)) + 1j * rng.standard_normal((B, H, W))
    coef = rng.uniform(0.1, 0.6, (B, H, W)) * (1 - 1j * rng.uniform(0.0, 0.8, (B, H, W)))
    r32, c32 = _pairs32(r), _pairs32(coef)
    r64 = r32[..., 0].astype(np.float64) + 1j * r32[..., 1]
    c64 = c32[..., 0].astype(np.float64) + 1j * c32[..., 1]
    dev = lambda a: torch.as_tensor(a).cuda()
    p_d, r_d, c_d = dev(pred), dev(r32), dev(c32)
    q = torch.empty((B, H, W, 2), dtype=torch.float32, device="cuda")
    sums = torch.empty(2 * B, dtype=torch.float32, device="cuda")
    grad = torch.empty((B, H, W, 16), dtype=torch.bfloat16, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    assert lib.helm_learned_residual_loss(vp(p_d), vp(r_d), vp(c_d), B, H, W, vp(q), vp(sums), vp(grad),
                                          vp(loss), stream()) == 0
    ref = C.residual_loss(pred.astype(np.float64), r64, c64)
    assert abs(float(loss.item()) - ref) <= 1e-5 * ref
    gref = C.residual_loss_grad(pred.astype(np.float64), r64, c64)
    assert rel(grad.float().cpu().numpy(), gref) < 1e-2


def test_residual_input_and_chain_match_oracle(lib):
    """helm_learned_residual_input: r / rho against the oracle's FP64 r = f - A
    z (the kernel forms r in complex64 arithmetic), coef against h^2 omega^2 m
    (1 - i gamma), the network input's channels; helm_learned_image_to_block
    returns the image as the internal block exactly."""
    from paper_1607_00968_gb300 import helm
    m, g = 1.0 / I.layered_velocity_2d(3, (32, 16)) ** 2, None
    shape = m.shape
    g = I.absorbing_gamma(shape, 4)
    h, om = 25.0, I.omega_for_ppw(25.0)
    S = helm.Solver(m, g, h, om, levels=2, prec="c64")
    rng = np.random.default_rng(41)
    s, N = 3, S.N
    f = rng.standard_normal((N, s)) + 1j * rng.standard_normal((N, s))
    z = (rng.standard_normal((N, s)) + 1j * rng.standard_normal((N, s))).astype(np.complex64)
    H, W = shape
    x = torch.empty((s, H, W, 16), dtype=torch.bfloat16, device="cuda")
    rimg = torch.empty((s, H, W, 2), dtype=torch.float32, device="cuda")
    cimg = torch.empty((s, H, W, 2), dtype=torch.float32, device="cuda")
    rho = torch.empty(s, dtype=torch.float32, device="cuda")
    f_d = torch.as_tensor(f).cuda()
    z_d = torch.as_tensor(z).cuda()
    assert lib.helm_learned_residual_input(S.ctx, vp(f_d), vp(z_d), s, vp(x), vp(rho), vp(rimg), vp(cimg)) == 0
    A = O.helmholtz_matrix(m, g, om, h)
    rr = f - A @ z.astype(np.complex128)
    rho_ref = np.sqrt(np.mean(np.abs(rr) ** 2, axis=0))
    np.testing.assert_allclose(rho.cpu().numpy(), rho_ref, rtol=1e-5)
    ri = rimg.cpu().numpy()
    for j in range(s):
        got = (ri[j, ..., 0] + 1j * ri[j, ..., 1]).ravel()
        assert rel(got, rr[:, j] / rho_ref[j]) < 1e-5
    ci = cimg.cpu().numpy()
    cref = (h * h * om * om * m * (1 - 1j * g)).ravel()
    np.testing.assert_allclose((ci[0, ..., 0] + 1j * ci[0, ..., 1]).ravel(), cref, rtol=1e-6)
    xin = x.float().cpu().numpy()
    np.testing.assert_allclose(xin[1, ..., 0], ri[1, ..., 0], rtol=1e-2, atol=1e-2)
    np.testing.assert_allclose(xin[1, ..., 2], ci[1, ..., 0], rtol=1e-2)
    v = torch.empty((N, s), dtype=torch.complex128, device="cuda")
    assert lib.helm_learned_image_to_block(vp(rimg), N, s, vp(v), stream()) == 0
    vv = v.cpu().numpy()
    for j in range(s):
        np.testing.assert_array_equal(vv[:, j], (ri[j, ..., 0].astype(np.float64) + 1j * ri[j, ..., 1]).ravel())


def test_residual_training_lowers_heldout_residual_loss(lib):
    """A short online run on the residual loss (small seeded problems) makes
    the correction remove part of the held-out residual: loss below its
    starting value (1 = the correction removes nothing)."""
    from paper_1607_00968_gb300 import learned
    kw = dict(cells=(128, 64), h=25.0, nsrc=8, steps=6, width=10)
    net = learned.Network(seed=0)
    xv, rv, cv = learned.residual_pairs(21, 5.0, **kw)
    before = learned.evaluate_residual_loss(net, xv, rv, cv, batch=4)
    learned.train_residual(net, [(11, 4.0), (12, 5.0), (13, 6.0)], iters_per_config=60, batch=4, lr=2e-3,
                           buffer_configs=3, **kw)
    after = learned.evaluate_residual_loss(net, xv, rv, cv, batch=4)
    print("\nresidual loss (held out): %.4f -> %.4f" % (before, after))
    assert after < before, (before, after)


def test_committed_network_gain_on_heldout_model(lib):
    """The committed weights (residual loss, trained on seeded models
    101-110, disjoint from this one) on the benchmark's salt model (seed 0)
    at 5 Hz.  What the network gains: on vectors of the stationary
    iteration's chain from this model's sources it removes more than 10% of
    the residual energy the V-cycle leaves (residual loss < 0.9).  With the
    stage on, FGMRES still reaches 1e-6 (true residual of the oracle's
    operator) in at most 10% more cycles; the cycle counts and times of both
    solves are printed (measured: the same cycles at 5 Hz, at about five
    times the cost per cycle)."""
    import os
    import time
    from paper_1607_00968_gb300 import helm, learned
    path = os.path.join(os.path.dirname(learned.__file__), "weights", "learned_salt2d.bin")
    net = learned.Network.load(path)
    assert net.record.get("loss") == "residual of the corrected iterate"
    xv, rv, cv = learned.residual_pairs(0, 5.0, nsrc=16, steps=6)
    loss = learned.evaluate_residual_loss(net, xv, rv, cv)
    assert loss < 0.9, loss
    P = I.salt2d_problem(seed=0, freq_hz=5.0)
    Q = torch.as_tensor(P.rhs()).cuda()
    A = O.helmholtz_matrix(P.m, P.gamma, P.omega, P.h)
    res = {}
    for prec in ("c64", "learned"):
        kw = dict(learned_weights=net.blob) if prec == "learned" else {}
        S = helm.Solver(P.m, P.gamma, P.h, P.omega, shift=0.2, levels=3, block=4, restart=6, prec=prec,
                        max_restarts=100, **kw)
        S.solve(Q, 1e-6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U, info, _ = S.solve(Q, 1e-6)
        torch.cuda.synchronize()
        res[prec] = (int(info.iters.max()), time.perf_counter() - t0)
        assert np.all(O.relres(A, U.cpu().numpy().T, P.rhs().T) <= 1e-6)
        S.close()
    print("\nheld-out residual loss %.3f; cycles / seconds without the stage %s, with it %s"
          % (loss, res["c64"], res["learned"]))
    assert res["learned"][0] <= 1.1 * res["c64"][0], res
