"""Fast marching and its sensitivity products for a set of sources on the
salt model (for profilers and timing).

    python -m paper_1607_00968_gb300.profile_eikonal --cells 512 256 --nsrc 64

Sets up the 2D faulted/salt velocity model (the Helmholtz salt workload's
model, or a smaller grid of the same generator), runs fast marching for
`nsrc` sources on the top row and one J v and one J^T w product, and prints
the wall times as JSON.
"""
from __future__ import annotations

import argparse
import json
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, nargs=2, default=[512, 256])
    ap.add_argument("--nsrc", type=int, default=64)
    ap.add_argument("--h", type=float, default=12.5)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()

    import numpy as np
    import torch

    from paper_1607_00968_gb300 import helm, inputs
    v = inputs.layered_velocity_2d(args.seed, tuple(args.cells), faults=3, salt=True)
    m = 1.0 / v ** 2
    shape = m.shape
    ns = args.nsrc
    sources = [(0, int(x)) for x in np.linspace(1, shape[1] - 2, ns).round()]
    ek = helm.Eikonal(shape, args.h, ns_max=ns)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()      # an external profiler started with capture off records from here
    t0 = time.perf_counter()
    ek.forward(m, sources, outputs=())
    t1 = time.perf_counter()
    vv = torch.ones(m.size, dtype=torch.float64, device="cuda")
    ek.jv(vv)
    t2 = time.perf_counter()
    ek.jtw(torch.ones((ns, m.size), dtype=torch.float64, device="cuda"))
    t3 = time.perf_counter()
    torch.cuda.profiler.stop()
    print(json.dumps({"cells": args.cells, "nodes": int(m.size), "sources": ns,
                      "forward_s": t1 - t0, "jv_ms": (t2 - t1) * 1e3, "jtw_ms": (t3 - t2) * 1e3,
                      "us_per_node": (t1 - t0) / m.size * 1e6}))
    ek.close()


if __name__ == "__main__":
    main()
