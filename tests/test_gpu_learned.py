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


def test_training_lowers_loss_and_learned_solve_converges(lib):
    """A short training run on small seeded problems lowers the validation
    loss; the solve with the stage on reaches the tolerance (true FP64
    residual of the oracle's operator) and its cycle count is reported beside
    the plain cycle's."""
    from paper_1607_00968_gb300 import helm, learned
    cells, h = (128, 64), 25.0
    x, t = learned.make_pairs(seeds=(11, 12), freqs=(5.0,), cells=cells, h=h, nsrc=8, steps=2)
    xv, tv = learned.make_pairs(seeds=(21,), freqs=(5.0,), cells=cells, h=h, nsrc=8, steps=1)
    net = learned.Network(seed=0)
    before = learned.evaluate_loss(net, xv, tv, batch=4)
    learned.train(net, x, t, iters=150, batch=4, lr=2e-3)
    after = learned.evaluate_loss(net, xv, tv, batch=4)
    assert after < before, (before, after)
    P = I.random_problem_2d(31, cells, h, 5.0, 8, width=10, levels=3)
    Q = torch.as_tensor(P.rhs()).cuda()
    S0 = helm.Solver(P.m, P.gamma, P.h, P.omega, shift=0.2, levels=3, block=4, restart=6, prec="c64")
    S1 = helm.Solver(P.m, P.gamma, P.h, P.omega, shift=0.2, levels=3, block=4, restart=6,
                     prec="learned", learned_weights=net.blob)
    U0, i0, _ = S0.solve(Q, 1e-6)
    U1, i1, _ = S1.solve(Q, 1e-6)
    A = O.helmholtz_matrix(P.m, P.gamma, P.omega, P.h)
    assert np.all(O.relres(A, U1.cpu().numpy().T, P.rhs().T) <= 1e-6)
    print("\nlearned stage: val loss %.3f -> %.3f; cycles off %d, on %d"
          % (before, after, i0.iters.max(), i1.iters.max()))
