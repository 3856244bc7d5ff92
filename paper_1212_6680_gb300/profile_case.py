"""Run one small case of the solver path, for profiling under a kernel profiler.

    python -m paper_1212_6680_gb300.profile_case fpcg    --n 128 --prec fp32 --solves 2
    python -m paper_1212_6680_gb300.profile_case brick   --n 80 --prec fp32 --solves 1
    python -m paper_1212_6680_gb300.profile_case learned --n 128 --solves 1
    python -m paper_1212_6680_gb300.profile_case lobpcg  --n 48 --m 16
    python -m paper_1212_6680_gb300.profile_case batched --nsys 16

Every case runs through the C ABI on seeded synthetic inputs (the generators of `inputs`), after
one untimed warm-up call, and prints one line with the iteration counts.  The learned case uses
the seeded initial weights (no training), which is enough to exercise every kernel.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fpcg", "brick", "learned", "lobpcg", "batched"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--npost", type=int, default=0)
    ap.add_argument("--solves", type=int, default=1)
    ap.add_argument("--m", type=int, default=16)
    ap.add_argument("--nsys", type=int, default=16)
    ap.add_argument("--device-loop", dest="host_loop", action="store_false",
                    help="run krylov_solve's iterations as one CUDA graph (default: the host loop)")
    a = ap.parse_args()

    import torch

    from . import build

    build.build()
    from . import inputs
    from . import smg as S

    out = {"case": a.case}
    if a.case in ("fpcg", "brick", "learned"):
        # the n^3 cube, or the paper's 16n x n x n brick (long in x)
        nx, ny, nz = (16 * a.n, a.n, a.n) if a.case == "brick" else (a.n, a.n, a.n)
        b = torch.from_numpy(inputs.rhs(nx, ny, nz, seed=0).ravel().copy()).cuda()
        x = torch.zeros_like(b)
        h = S.smg_setup(nx, ny, nz, 1, a.npost)
        S.smg_set_precision(h, a.prec)
        # the host loop launches every kernel of an iteration itself, so a kernel profiler sees each
        # launch (the device-side loop runs them inside a conditional graph node)
        S.smg_set_option(h, S.SMG_OPT_GRAPH, 0 if a.host_loop else 1)
        if a.case == "learned":
            S.smg_set_learned(h, inputs.net_init_weights(seed=77))
        S.krylov_solve(h, "fpcg", b, x, 1e-8, 100)
        its = []
        for _ in range(a.solves):
            x.zero_()
            rc, it, res = S.krylov_solve(h, "fpcg", b, x, 1e-8, 100)
            its.append(it)
        S.smg_destroy(h)
        out["iters"] = its
    elif a.case == "lobpcg":
        n = a.n
        X0 = torch.from_numpy(np.ascontiguousarray(inputs.initial_block(n, n, n, a.m, seed=7)).ravel().copy()).cuda()
        X = torch.empty_like(X0)
        h = S.smg_setup(n, n, n, 1, a.npost)
        S.smg_set_precision(h, a.prec)
        its = []
        for _ in range(1 + a.solves):
            X.copy_(X0)
            rc, it, lam = S.lobpcg_solve(h, a.m, X, tol=1e-8, maxit=200)
            its.append(it)
        S.smg_destroy(h)
        out["iters"] = its[1:]
    else:
        dims = inputs.uneven_dims(a.nsys, 32, 96, seed=1000)
        bs = [torch.from_numpy(inputs.rhs(int(nx), int(ny), int(nz), seed=1000 + i).ravel().copy()).cuda()
              for i, (nx, ny, nz) in enumerate(dims)]
        xs = [torch.zeros_like(b) for b in bs]
        h = S.smg_batched_setup(dims)
        its = []
        for _ in range(1 + a.solves):
            for x in xs:
                x.zero_()
            rc, it, rel = S.smg_batched_solve(h, "fpcg", bs, xs)
            its.append(int(it.max()))
        S.smg_batched_destroy(h)
        out["iters"] = its[1:]
    torch.cuda.synchronize()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
