"""Batched uneven systems: every system of a krylov_solve_batched call reaches
the tolerance on its own FP64 true residual (checked with the oracle's operator) in about the
oracle's FP64 iteration count, and the bounded grid barrier reports a timeout instead of
hanging when it waits for a CTA that does not exist."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1212_6680_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    assert torch.cuda.is_available()
    return m


@pytest.mark.parametrize("nsys,lo,hi", [(5, 8, 40), (12, 16, 48)])
def test_batched_uneven_systems_reach_tolerance(smg, orc, nsys, lo, hi):
    dims = inputs.uneven_dims(nsys, lo, hi, seed=2000 + nsys)
    bs, xs, bh = [], [], []
    for s, (nx, ny, nz) in enumerate(dims):
        b = inputs.rhs(int(nx), int(ny), int(nz), seed=3000 + s)
        bh.append(b)
        bs.append(torch.from_numpy(b.ravel().copy()).cuda())
        xs.append(torch.zeros(b.size, dtype=torch.float64, device="cuda"))
    rc, iters = smg.krylov_solve_batched(dims, bs, xs, npre=1, npost=0, prec="fp32", tol=1e-8, maxit=100)
    assert rc == smg.SMG_OK, smg.smg_last_error()
    for s, (nx, ny, nz) in enumerate(dims):
        b = bh[s]
        xh = xs[s].cpu().numpy().reshape(b.shape)
        true = np.linalg.norm(b - orc.apply_A(xh)) / np.linalg.norm(b)
        assert true <= 1e-8, (s, true)
        ref = orc.krylov(b, "fpcg", orc.SMG(int(nx), int(ny), int(nz), 1, 0), tol=1e-8, maxit=100)
        assert iters[s] <= ref["iters"] + 2, (s, iters[s], ref["iters"])


def test_batched_matches_single_system_path(smg):
    dims = np.array([[40, 33, 29], [17, 50, 22]])
    bs = [torch.from_numpy(inputs.rhs(*map(int, d), seed=11 + i).ravel().copy()).cuda() for i, d in enumerate(dims)]
    xb = [torch.zeros_like(b) for b in bs]
    rc, iters = smg.krylov_solve_batched(dims, bs, xb, tol=1e-10, maxit=100)
    assert rc == smg.SMG_OK
    for i, d in enumerate(dims):
        with smg.Handle(*map(int, d), 1, 0, precision="fp32") as h:
            x1 = torch.zeros_like(bs[i])
            rc1, it1, _ = smg.krylov_solve(h.h, "fpcg", bs[i], x1, tol=1e-10, maxit=100)
        assert abs(int(iters[i]) - it1) <= 1
        assert float(torch.linalg.norm(x1 - xb[i]) / torch.linalg.norm(x1)) <= 1e-7


def test_batched_rejects_bad_arguments(smg):
    b = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(smg.SMGError):
        smg.krylov_solve_batched([[200, 4, 4]], [b], [b])  # nx > 128
    with pytest.raises(smg.SMGError):
        smg.krylov_solve_batched([[4, 4, 4]], [b], [b], prec="fp64")


def test_grid_barrier_completes_and_times_out_cleanly(smg):
    assert smg.smg_barrier_selftest(0, 0.5) == smg.SMG_OK
    assert smg.smg_barrier_selftest(1, 0.2) == smg.SMG_ERR_TIMEOUT
    # the context is still usable afterwards
    assert smg.smg_barrier_selftest(0, 0.5) == smg.SMG_OK
    x = torch.ones(4, device="cuda")
    assert float(x.sum()) == 4.0
