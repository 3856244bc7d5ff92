"""Training driver of the learned post-correction (argument marshalling over the C ABI; every
numerical step runs in the library's kernels).

Recipe: seeded systems with sides drawn uniformly from [lo, hi] per axis; for each, x* from an
FP64 flexible PCG solve with the balanced (1,1) cycle to a relative residual of 1e-13, then a
flexible PCG run with the FP32 (1,0) cycle whose iterations are recorded as (rho_k, e_k) pairs
(smg_collect_pairs); Adam over all pairs (smg_net_train) from seeded initial weights.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from . import smg as S


def collect_pairs(nsys: int, lo: int, hi: int, seed: int = 5000, max_pairs: int = 16, tol: float = 1e-8):
    """Returns (dims per pair, rho tensors, e tensors, stats) -- FP32 device tensors."""
    import torch

    dims = inputs.uneven_dims(nsys, lo, hi, seed=seed)
    dl, rl, el = [], [], []
    for i, (nx, ny, nz) in enumerate(dims):
        nx, ny, nz = int(nx), int(ny), int(nz)
        n = nx * ny * nz
        b = torch.from_numpy(inputs.rhs(nx, ny, nz, seed=seed + 10000 + i).ravel().copy()).cuda()
        xs = torch.zeros(n, dtype=torch.float64, device="cuda")
        h64 = S.smg_setup(nx, ny, nz, 1, 1)
        try:
            rc, _, res = S.krylov_solve(h64, "fpcg", b, xs, 1e-13, 300)
        finally:
            S.smg_destroy(h64)
        h = S.smg_setup(nx, ny, nz, 1, 0)
        try:
            S.smg_set_precision(h, "fp32")
            rho = torch.empty(max_pairs * n, dtype=torch.float32, device="cuda")
            e = torch.empty(max_pairs * n, dtype=torch.float32, device="cuda")
            k = S.smg_collect_pairs(h, b, xs, rho, e, max_pairs, tol=tol, maxit=100)
        finally:
            S.smg_destroy(h)
        for j in range(k):
            dl.append((nx, ny, nz))
            rl.append(rho[j * n:(j + 1) * n])
            el.append(e[j * n:(j + 1) * n])
    return dl, rl, el, {"systems": nsys, "pairs": len(rl), "unknowns": int(sum(np.prod(d) for d in dl))}


def train(nsys=200, lo=64, hi=128, epochs=4, lr=1e-3, seed=5000, init_seed=77, act="bf16"):
    """Collect pairs and train; returns (FP32 weights, info dict)."""
    t0 = time.perf_counter()
    dl, rl, el, info = collect_pairs(nsys, lo, hi, seed=seed)
    t1 = time.perf_counter()
    w0 = inputs.net_init_weights(seed=init_seed)
    w, hist = S.smg_net_train(dl, rl, el, w0, epochs=epochs, lr=lr, seed=seed, act=act)
    t2 = time.perf_counter()
    info.update({"collect_s": t1 - t0, "train_s": t2 - t1, "epochs": epochs, "lr": lr, "loss_per_epoch": hist.tolist(),
                 "sides": [lo, hi], "act": act})
    return w, info


def save_weights(path: str, w, info: dict) -> None:
    """Store FP32 weights and their training recipe (the info dict of `train`) in one .npz file."""
    import json

    np.savez(path, w=np.asarray(w, dtype=np.float32), info=np.array(json.dumps(info)))


def load_weights(path: str):
    """Returns (FP32 weights, recipe dict) stored by `save_weights`."""
    import json

    with np.load(path) as z:
        return z["w"].astype(np.float32), json.loads(str(z["info"]))
