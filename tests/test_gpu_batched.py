"""Batched uneven systems: every system of a krylov_solve_batched call reaches
the tolerance on its own FP64 true residual (checked with the oracle's operator) in about the
oracle's FP64 iteration count, and the bounded grid barrier reports a timeout instead of
hanging when it waits for a CTA that does not exist."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1212_6680_gb300 import inputs  # noqa: E402
from tests.parity import assert_close  # noqa: E402


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
        assert abs(int(iters[s]) - ref["iters"]) <= 1, (s, iters[s], ref["iters"])


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


def _systems(dims, seed0):
    bs, bh = [], []
    for s, (nx, ny, nz) in enumerate(dims):
        b = inputs.rhs(int(nx), int(ny), int(nz), seed=seed0 + s)
        bh.append(b)
        bs.append(torch.from_numpy(b.ravel().copy()).cuda())
    return bh, bs


@pytest.mark.parametrize("variant", ["pcg", "fpcg", "psd"])
def test_batched_handle_variants_match_oracle_counts(smg, orc, variant):
    """Each Krylov variant of Algorithm 1 through one handle: true residual <= tol and the
    oracle's FP64 iteration count within 1.  PCG eq. (1) uses the balanced (1,1) cycle, for which
    the paper shows it converges; PSD and FPCG use (1,0)."""
    npost = 1 if variant == "pcg" else 0
    dims = inputs.uneven_dims(6, 10, 36, seed=4000)
    bh, bs = _systems(dims, 5000)
    h = smg.smg_batched_setup(dims, npre=1, npost=npost)
    try:
        xs = [torch.zeros_like(b) for b in bs]
        rc, iters, rel = smg.smg_batched_solve(h, variant, bs, xs, tol=1e-8, maxit=100)
        assert rc == smg.SMG_OK, smg.smg_last_error()
        for s, (nx, ny, nz) in enumerate(dims):
            xh = xs[s].cpu().numpy().reshape(bh[s].shape)
            true = np.linalg.norm(bh[s] - orc.apply_A(xh)) / np.linalg.norm(bh[s])
            assert true <= 1e-8 and abs(true - rel[s]) <= 1e-3 * true + 1e-15, (s, true, rel[s])
            ref = orc.krylov(bh[s], variant, orc.SMG(int(nx), int(ny), int(nz), 1, npost), tol=1e-8, maxit=100)
            assert abs(int(iters[s]) - ref["iters"]) <= 1, (s, iters[s], ref["iters"])
    finally:
        smg.smg_batched_destroy(h)


def test_batched_handle_reuse_is_deterministic_and_profiles(smg):
    """Two solves through one captured graph give bit-identical results; x0 != 0 is honoured;
    the schedule report and the profile counters are consistent with the solve."""
    dims = inputs.uneven_dims(9, 20, 60, seed=4100)
    _, bs = _systems(dims, 5100)
    h = smg.smg_batched_setup(dims)
    try:
        info = smg.smg_batched_info(h)
        nsm = torch.cuda.get_device_properties(0).multi_processor_count
        assert info["threads"] in (256, 512) and info["order"] in (0, 1)
        assert info["blocks"] >= nsm and info["blocks"] % nsm == 0
        # the line tile: from the narrowest that holds the widest system's lines up to 4 rows per lane
        kmin = (int(max(d[0] for d in dims)) + 31) // 32
        assert kmin <= info["rows_per_lane"] <= 4
        smg.smg_batched_set_profile(h, 1)
        out = []
        for _ in range(2):
            xs = [torch.zeros_like(b) for b in bs]
            rc, iters, _ = smg.smg_batched_solve(h, "fpcg", bs, xs)
            assert rc == smg.SMG_OK
            out.append((iters.copy(), [x.clone() for x in xs]))
        assert (out[0][0] == out[1][0]).all()
        for a, b in zip(out[0][1], out[1][1]):
            assert torch.equal(a, b)
        n0, ms0, by0 = smg.smg_batched_profile_read(h, 0)
        n1, ms1, _ = smg.smg_batched_profile_read(h, 1)
        # one replay per iteration while any system iterates (restarts from the true residual add more)
        assert n0 == n1 and n0 >= 2 * int(out[0][0].max())
        assert ms0 > 0 and ms1 > 0 and by0 > 0
        # restart from the converged solution: every system is done at once
        xs = out[1][1]
        rc, iters, rel = smg.smg_batched_solve(h, "fpcg", bs, xs)
        assert rc == smg.SMG_OK and (iters == 0).all() and (rel <= 1e-8).all()
    finally:
        smg.smg_batched_destroy(h)


@pytest.mark.parametrize("npost", [0, 1])
def test_batched_apply_matches_oracle_cycle(smg, orc, npost):
    """One launch of the persistent V-cycle (smg_batched_apply) on seeded right-hand sides of
    uneven systems against the oracle's cycle of each system, element by element and plane by
    plane at the FP32 cycle's tolerance; two applications give identical results (section 3: the
    preconditioner is fixed and linear)."""
    dims = inputs.uneven_dims(10, 8, 70, seed=4200 + npost)
    rh = [inputs.rhs(int(nx), int(ny), int(nz), seed=4300 + s) for s, (nx, ny, nz) in enumerate(dims)]
    r = [torch.from_numpy(v.ravel().copy()).cuda() for v in rh]
    h = smg.smg_batched_setup(dims, npre=1, npost=npost)
    try:
        out = [torch.empty_like(v) for v in r]
        smg.smg_batched_apply(h, r, out)
        first = [o.clone() for o in out]
        smg.smg_batched_apply(h, r, out)
    finally:
        smg.smg_batched_destroy(h)
    for s, (nx, ny, nz) in enumerate(dims):
        assert torch.equal(first[s], out[s])
        ref = orc.SMG(int(nx), int(ny), int(nz), 1, npost).apply(rh[s])
        assert_close(out[s].cpu().numpy(), ref, 2e-5, (int(nx), int(ny), int(nz)), f"system {s} {tuple(dims[s])}")
