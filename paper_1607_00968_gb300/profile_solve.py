"""Run one multi-source Helmholtz solve of a named workload (for profilers).

    python -m paper_1607_00968_gb300.profile_solve --workload salt2d --freq 5 \
        --prec c64 --levels 3 --block 8 --restart 10 --nsrc 64

Sets the problem up, runs one warm-up solve on a few columns and one full
solve, and prints the cycle counts, the residuals and the per-kernel
profile of the full solve.  It is the small, self-contained case used for
Nsight Compute captures of single kernels.
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="salt2d", choices=["salt2d", "layered2d", "layered3d"])
    ap.add_argument("--freq", type=float, default=5.0)
    ap.add_argument("--prec", default="c64", choices=["c64", "c128"])
    ap.add_argument("--levels", type=int, default=3)
    ap.add_argument("--block", type=int, default=8)
    ap.add_argument("--restart", type=int, default=10)
    ap.add_argument("--shift", type=float, default=0.2)
    ap.add_argument("--nsrc", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cycle", default="V", choices=["V", "W", "K"])
    ap.add_argument("--krylov", default="fgmres", choices=["fgmres", "bicgstab"])
    args = ap.parse_args()

    import torch

    from paper_1607_00968_gb300 import helm, inputs
    if args.workload == "salt2d":
        P = inputs.salt2d_problem(seed=args.seed, freq_hz=args.freq, nsrc=args.nsrc)
    elif args.workload == "layered2d":
        P = inputs.layered2d_problem(seed=args.seed, nsrc=args.nsrc)
    else:
        P = inputs.layered3d_problem(seed=args.seed, freq_hz=args.freq)
    S = helm.Solver(P.m, P.gamma, P.h, P.omega, shift=args.shift, levels=args.levels,
                    block=args.block, restart=args.restart, prec=args.prec, max_restarts=200,
                    cycle=args.cycle, krylov=args.krylov)
    Q = torch.as_tensor(P.rhs()[: args.nsrc]).cuda()
    S.solve(Q, args.tol)          # warm-up on the full block (same launch shapes)
    S.profile(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    torch.cuda.profiler.start()   # an external profiler started with capture off records this solve
    U, info, st = S.solve(Q, args.tol)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    dt = time.perf_counter() - t0
    prof = {k: v for k, v in S.profile_read().items() if v["launches"]}
    print(json.dumps({"workload": P.name, "freq_hz": args.freq, "prec": args.prec,
                      "cycle": args.cycle, "krylov": args.krylov, "block": args.block,
                      "seconds": dt, "rhs_per_s": Q.shape[0] / dt,
                      "cycles": int(info.iters.max()), "max_relres": float(info.relres.max()),
                      "kernels": prof}))


if __name__ == "__main__":
    main()
