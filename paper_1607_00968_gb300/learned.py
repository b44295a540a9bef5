"""Learned preconditioning stage: network state, training data, training loop.

The network (six 3x3 convolutions, 32 hidden channels, ReLU between) maps the
residual left by one shifted-Laplacian V-cycle, r = v - A V(v), normalised by
its RMS rho, plus kappa = omega^2 m h^2, to a correction e ~ A^{-1} r in units
of h^2 rho; FGMRES then uses z = V(v) + h^2 rho N(r/rho, kappa) (see
include/helm.h, "Learned preconditioning stage").  Every forward, backward,
loss and optimiser step runs in libhelm's kernels (helm_conv3x3,
helm_conv3x3_wgrad, helm_conv3x3_flip, helm_learned_residual_loss,
helm_adam), and so does the training data (helm_vcycle,
helm_learned_residual_input, helm_learned_image_to_block); this module holds
the buffers and drives the loop.

Training data come from the solver itself on seeded random faulted/salt
models.  Loss: the residual left after the correction, ||r - h^2 A (h^2 rho
N)|| / ||r|| in the network's units (train_residual; the right-hand sides
follow the stationary iteration's residual chain, and every pair costs one
V-cycle, no solve).

Weights are saved as the flat blob of the ABI (bf16 weights + float biases)
plus a JSON header (layer table, training record).
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import time

import numpy as np

from . import helm, inputs


def _vp(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class Network:
    """Device-resident network: the ABI weight blob (bf16 weights, float
    biases; the biases in the blob are the master copies), FP32 master
    weights, gradients and Adam moments."""

    def __init__(self, seed: int = 0, device="cuda"):
        import torch
        self.torch = torch
        self.lib = helm.load()
        L = self.lib
        self.layers = []
        for l in range(L.helm_learned_layers()):
            cin, cout, relu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            wo, bo = ctypes.c_longlong(), ctypes.c_longlong()
            L.helm_learned_layer(l, ctypes.byref(cin), ctypes.byref(cout), ctypes.byref(relu),
                                 ctypes.byref(wo), ctypes.byref(bo))
            self.layers.append(dict(cin=cin.value, cout=cout.value, relu=relu.value,
                                    w_off=wo.value, b_off=bo.value))
        self.blob = torch.zeros(int(L.helm_learned_blob_bytes()), dtype=torch.uint8, device=device)
        g = np.random.Generator(np.random.PCG64(seed))
        self.w32, self.wbf, self.b, self.dw, self.db, self.mom = [], [], [], [], [], []
        for l, t in enumerate(self.layers):
            n = t["cout"] * 9 * t["cin"]
            used_in = 3 if l == 0 else t["cin"]
            used_out = 2 if l == len(self.layers) - 1 else t["cout"]
            w = np.zeros((t["cout"], 9, t["cin"]), dtype=np.float32)
            std = math.sqrt(2.0 / (9 * used_in))
            if l == len(self.layers) - 1:
                std *= 0.1                       # start close to the plain cycle
            w[:used_out, :, :used_in] = g.standard_normal((used_out, 9, used_in)) * std
            w32 = torch.as_tensor(w.reshape(-1)).to(device)
            wbf = self.blob[t["w_off"]:t["w_off"] + 2 * n].view(torch.bfloat16)
            wbf.copy_(w32.to(torch.bfloat16))
            b = self.blob[t["b_off"]:t["b_off"] + 4 * t["cout"]].view(torch.float32)
            self.w32.append(w32)
            self.wbf.append(wbf)
            self.b.append(b)
            self.dw.append(torch.zeros_like(w32))
            self.db.append(torch.zeros_like(b))
            self.mom.append([torch.zeros_like(w32), torch.zeros_like(w32),
                             torch.zeros_like(b), torch.zeros_like(b)])
        self.flip = [torch.empty(t["cin"] * 9 * t["cout"], dtype=torch.bfloat16, device=device)
                     for t in self.layers]
        self.step_count = 0
        self.record = {}

    # ------------------------------------------------------------------
    def _check(self, st, what):
        if st != 0:
            raise helm.HelmError(st, what + ": " + self.lib.helm_last_error(None).decode())

    def forward(self, x, B, H, W, keep=False):
        """x: bf16 [B, H, W, 16] -> float [B, H, W, 16] (channels 0, 1 used)."""
        torch = self.torch
        stream = _vp_stream(torch)
        acts = [x]
        cur = x
        for l, t in enumerate(self.layers):
            last = l == len(self.layers) - 1
            out = torch.empty((B, H, W, t["cout"]), device=x.device,
                              dtype=torch.float32 if last else torch.bfloat16)
            self._check(self.lib.helm_conv3x3(_vp(cur), B, H, W, t["cin"], _vp(self.wbf[l]),
                                              _vp(self.b[l]), t["cout"], t["relu"], None, _vp(out),
                                              1 if last else 0, stream), "conv3x3")
            acts.append(out)
            cur = out
        return (cur, acts) if keep else cur

    def backward(self, acts, grad, B, H, W):
        """grad: bf16 [B, H, W, 16], d loss / d output.  Accumulates dw, db."""
        torch = self.torch
        stream = _vp_stream(torch)
        g = grad
        for l in range(len(self.layers) - 1, -1, -1):
            t = self.layers[l]
            self._check(self.lib.helm_conv3x3_wgrad(_vp(acts[l]), _vp(g), B, H, W, t["cin"],
                                                    t["cout"], _vp(self.dw[l]), _vp(self.db[l]),
                                                    stream), "wgrad")
            if l == 0:
                break
            self._check(self.lib.helm_conv3x3_flip(_vp(self.wbf[l]), t["cin"], t["cout"],
                                                   _vp(self.flip[l]), t["cin"], stream), "flip")
            gin = torch.empty((B, H, W, t["cin"]), device=g.device, dtype=torch.bfloat16)
            # data gradient: conv with transposed, flipped weights, times the
            # ReLU derivative of the layer below (its output > 0)
            self._check(self.lib.helm_conv3x3(_vp(g), B, H, W, t["cout"], _vp(self.flip[l]), None,
                                              t["cin"], 0, _vp(acts[l]), _vp(gin), 0, stream),
                        "conv3x3 backward")
            g = gin

    def zero_grad(self):
        for a in self.dw + self.db:
            a.zero_()

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        stream = _vp_stream(self.torch)
        for l in range(len(self.layers)):
            m1, v1, m2, v2 = self.mom[l]
            self._check(self.lib.helm_adam(_vp(self.w32[l]), _vp(self.dw[l]), _vp(m1), _vp(v1),
                                           _vp(self.wbf[l]), self.w32[l].numel(), lr, b1, b2, eps,
                                           self.step_count, stream), "adam")
            self._check(self.lib.helm_adam(_vp(self.b[l]), _vp(self.db[l]), _vp(m2), _vp(v2), None,
                                           self.b[l].numel(), lr, b1, b2, eps, self.step_count,
                                           stream), "adam")

    # ------------------------------------------------------------------
    def save(self, path: str):
        """Flat blob (bytes of the ABI layout) + JSON header next to it."""
        with open(path, "wb") as f:
            f.write(self.blob.cpu().numpy().tobytes())
        head = dict(layers=self.layers, blob_bytes=int(self.blob.numel()), record=self.record,
                    format="libhelm learned-stage blob: bf16 weights [co][tap][ci], float biases")
        with open(path + ".json", "w") as f:
            json.dump(head, f, indent=1)

    @classmethod
    def load(cls, path: str, device="cuda"):
        net = cls(seed=0, device=device)
        raw = np.frombuffer(open(path, "rb").read(), dtype=np.uint8)
        if raw.size != net.blob.numel():
            raise ValueError("weight blob size %d does not match the layer table (%d)"
                             % (raw.size, net.blob.numel()))
        net.blob.copy_(net.torch.as_tensor(raw.copy()).to(device))
        for l in range(len(net.layers)):
            net.w32[l].copy_(net.wbf[l].float())
        hp = path + ".json"
        if os.path.exists(hp):
            net.record = json.load(open(hp)).get("record", {})
        return net


def _vp_stream(torch):
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ----------------------------------------------------------------------
# training data from the solver
# ----------------------------------------------------------------------

# ----------------------------------------------------------------------
# residual-loss training: the residual of the corrected iterate
# ----------------------------------------------------------------------

def residual_pairs(seed, freq, cells=(512, 256), h=12.5, nsrc=32, steps=16, shift=0.2, levels=3,
                   width=20):
    """(x bf16 [P, H, W, 16], r float [P, H, W, 2], coef float [P, H, W, 2]),
    P = nsrc * steps, from one seeded random model at one frequency.

    The right-hand sides follow the stationary iteration's residual chain,
    v_{k+1} = (v_k - A V(v_k)) / rho_k, started at unit point sources: half
    on the top node row (where the benchmark's sources sit), half at seeded
    random interior nodes.  Every step runs in libhelm kernels (V-cycle,
    residual, packing, the chain's next vector)."""
    import torch
    lib = helm.load()
    P = inputs.random_problem_2d(seed, cells, h, freq, nsrc, width=width, levels=levels)
    S = helm.Solver(P.m, P.gamma, P.h, P.omega, shift=shift, levels=levels, block=8, restart=10,
                    prec="c64", max_restarts=50)
    H, W = P.shape
    N = S.N
    g = np.random.Generator(np.random.PCG64(7919 + seed))
    top = inputs.line_positions(P.shape, nsrc - nsrc // 2, 0, width)
    inner = [(int(g.integers(2, H - width)), int(g.integers(width, W - width)))
             for _ in range(nsrc // 2)]
    b = torch.as_tensor(inputs.point_sources(P.shape, top + inner, h)).cuda()   # (s, N)
    v = b.T.contiguous()                                                         # (N, s) layout
    xs, rs, cs = [], [], []
    stream = _vp_stream(torch)
    for _ in range(steps):
        z1 = S.vcycle(v, "c64")
        x = torch.empty((nsrc, H, W, 16), dtype=torch.bfloat16, device="cuda")
        r = torch.empty((nsrc, H, W, 2), dtype=torch.float32, device="cuda")
        c = torch.empty((nsrc, H, W, 2), dtype=torch.float32, device="cuda")
        rho = torch.empty(nsrc, dtype=torch.float32, device="cuda")
        st = lib.helm_learned_residual_input(S.ctx, _vp(v), _vp(z1), nsrc, _vp(x), _vp(rho), _vp(r), _vp(c))
        if st != 0:
            raise helm.HelmError(st, lib.helm_last_error(S.ctx).decode())
        xs.append(x)
        rs.append(r)
        cs.append(c)
        v = torch.empty((N, nsrc), dtype=torch.complex128, device="cuda")
        st = lib.helm_learned_image_to_block(_vp(r), N, nsrc, _vp(v), stream)
        if st != 0:
            raise helm.HelmError(st, lib.helm_last_error(None).decode())
    S.close()
    return torch.cat(xs), torch.cat(rs), torch.cat(cs)


class ResidualLoss:
    """Scratch and the call of helm_learned_residual_loss for one batch shape."""

    def __init__(self, batch, H, W, device="cuda"):
        import torch
        self.B, self.H, self.W = batch, H, W
        self.q = torch.empty((batch, H, W, 2), dtype=torch.float32, device=device)
        self.sums = torch.empty(2 * batch, dtype=torch.float32, device=device)
        self.loss = torch.empty(1, dtype=torch.float32, device=device)
        self.grad = torch.empty((batch, H, W, 16), dtype=torch.bfloat16, device=device)
        self.lib = helm.load()
        self.torch = torch

    def __call__(self, pred, r, c):
        st = self.lib.helm_learned_residual_loss(_vp(pred), _vp(r), _vp(c), self.B, self.H, self.W, _vp(self.q),
                                                 _vp(self.sums), _vp(self.grad), _vp(self.loss),
                                                 _vp_stream(self.torch))
        if st != 0:
            raise helm.HelmError(st, self.lib.helm_last_error(None).decode())
        return self.grad


def evaluate_residual_loss(net: Network, x, r, c, batch=8):
    """Mean residual loss over a pool (1 = the correction removes nothing)."""
    P, H, W, _ = x.shape
    rl = ResidualLoss(batch, H, W, device=x.device)
    tot, n = 0.0, 0
    for i0 in range(0, P - batch + 1, batch):
        out = net.forward(x[i0:i0 + batch].contiguous(), batch, H, W)
        rl(out, r[i0:i0 + batch].contiguous(), c[i0:i0 + batch].contiguous())
        tot += float(rl.loss.item())
        n += 1
    return tot / max(n, 1)


def train_residual(net: Network, configs, iters_per_config=64, batch=8, lr=1e-3, buffer_configs=4,
                   seed=0, log_every=100, **pair_kw):
    """Online training on the residual loss: the pairs of each (seed, freq)
    configuration join a rolling buffer of the last `buffer_configs`
    configurations, and `iters_per_config` Adam steps on batches drawn from
    the buffer follow.  Returns the loss history."""
    import torch
    g = np.random.Generator(np.random.PCG64(seed))
    buf = []
    hist = []
    it = 0
    pairs = 0
    t0 = time.perf_counter()
    rl = None
    for (sd, f) in configs:
        buf.append(residual_pairs(sd, f, **pair_kw))
        pairs += buf[-1][0].shape[0]
        if len(buf) > buffer_configs:
            buf.pop(0)
        X = torch.cat([b[0] for b in buf])
        R = torch.cat([b[1] for b in buf])
        Cf = torch.cat([b[2] for b in buf])
        P, H, W, _ = X.shape
        if rl is None:
            rl = ResidualLoss(batch, H, W, device=X.device)
        for _ in range(iters_per_config):
            idx = torch.as_tensor(g.choice(P, size=batch, replace=False), device=X.device)
            xb, rb, cb = X[idx].contiguous(), R[idx].contiguous(), Cf[idx].contiguous()
            out, acts = net.forward(xb, batch, H, W, keep=True)
            grad = rl(out, rb, cb)
            net.zero_grad()
            net.backward(acts, grad, batch, H, W)
            net.adam(lr=lr)
            if it % log_every == 0:
                hist.append((it, float(rl.loss.item())))
            it += 1
        del X, R, Cf
    net.record.update(dict(loss="residual of the corrected iterate", iters=it, batch=batch, lr=lr,
                           pairs=int(pairs), configs=[list(c) for c in configs],
                           seconds=time.perf_counter() - t0, loss_history=hist))
    return hist


def main():
    """Train the stage on seeded models and save the blob:
    python -m paper_1607_00968_gb300.learned OUT_PATH [ITERS_PER_CONFIG]
    (the residual loss, online over 40 model/frequency configurations,
    about 20k pairs)."""
    import sys
    import torch
    out = sys.argv[1] if len(sys.argv) > 1 else "learned_salt2d.bin"
    torch.cuda.set_device(0)
    ipc = int(sys.argv[2]) if len(sys.argv) > 2 else 64
    configs = [(sd, f) for sd in range(101, 111) for f in (3.0, 4.5, 6.0, 7.5)]
    net = Network(seed=0)
    xv, rv, cv = residual_pairs(201, 5.0, nsrc=16, steps=8)
    before = evaluate_residual_loss(net, xv, rv, cv)
    train_residual(net, configs, iters_per_config=ipc)
    after = evaluate_residual_loss(net, xv, rv, cv)
    net.record.update(dict(val_loss_before=before, val_loss_after=after, val_seeds=[201],
                           val_freq_hz=5.0, cells=[512, 256], h=12.5))
    net.save(out)
    print(json.dumps(net.record))


if __name__ == "__main__":
    main()
