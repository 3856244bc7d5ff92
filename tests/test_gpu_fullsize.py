"""Parity at the benchmark's own sizes and launch configurations: the 128^3 cycle (FP64 against
the oracle to 1e-12, FP32 to 2e-5) and flexible PCG iteration counts against the oracle; LOBPCG's
16 smallest eigenvalues at 128^3 against the closed form; the 64 uneven systems of the batched
workload each to its tolerance by an independent residual, with sampled systems against the
oracle's iteration counts; and the learned correction at 256^3 on sampled points against the
oracle evaluated on the 7^3 crop around each point (clipped to the grid) -- exact because the
network's receptive field is 7^3 and, being positively homogeneous, its RMS-scaled output does
not depend on the scale the crop is normalised with."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1212_6680_gb300 import inputs  # noqa: E402
from tests import dense_ref as D  # noqa: E402
from tests.parity import assert_close  # noqa: E402


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    assert torch.cuda.is_available()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


N = 128


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_apply_128cube_matches_oracle(smg, orc, prec, tol):
    r = inputs.rhs(N, N, N, seed=0)
    ref = orc.SMG(N, N, N, 1, 0).apply(r)
    with smg.Handle(N, N, N, 1, 0, precision=prec) as h:
        s = torch.empty(r.size, dtype=torch.float64, device="cuda")
        smg.smg_apply(h.h, dev(r), s)
        got = s.cpu().numpy()
    assert_close(got, ref, tol, (N, N, N), f"{prec} cycle at 128^3")


def test_fpcg_128cube_matches_oracle_iterations(smg, orc):
    b = inputs.rhs(N, N, N, seed=0)
    ref = orc.krylov(b, "fpcg", orc.SMG(N, N, N, 1, 0), tol=1e-8, maxit=100)
    for prec in ("fp32", "bf16", "fp64"):
        with smg.Handle(N, N, N, 1, 0, precision=prec) as h:
            x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
            rc, it, res = smg.krylov_solve(h.h, "fpcg", dev(b), x, 1e-8, 100)
            xh = x.cpu().numpy().reshape(b.shape)
        assert rc == smg.SMG_OK
        true = np.linalg.norm(b - D.lap7(xh)) / np.linalg.norm(b)
        assert true <= 1e-8 and abs(true - res) <= 1e-3 * true, (prec, true, res)
        assert abs(it - ref["iters"]) <= 1, (prec, it, ref["iters"])


def test_lobpcg_128cube_16_eigenpairs_closed_form(smg):
    m = 16
    X0 = inputs.initial_block(N, N, N, m, seed=7)
    ev = [4 * np.sin(np.pi * np.arange(1, N + 1) / (2 * (N + 1))) ** 2] * 3
    ref = np.sort((ev[0][:, None, None] + ev[1][None, :, None] + ev[2][None, None, :]).ravel())[:m]
    with smg.Handle(N, N, N, 1, 0, precision="fp32") as h:
        X = dev(X0)
        rc, it, lam = smg.lobpcg_solve(h.h, m, X, tol=1e-8, maxit=200)
        Xh = X.cpu().numpy().reshape(m, -1)
    assert rc == smg.SMG_OK
    assert np.all(np.abs(lam - ref) <= 1e-10 * ref), np.max(np.abs(lam - ref) / ref)
    assert np.abs(Xh @ Xh.T - np.eye(m)).max() <= 1e-10
    # every Ritz vector is an eigenvector to the tolerance
    for j in range(m):
        v = Xh[j].reshape(N, N, N)
        assert np.linalg.norm(D.lap7(v) - lam[j] * v) <= 1e-8 * lam[j] * np.linalg.norm(v) * 1.0001


def test_batched_64_uneven_systems_full_config(smg, orc):
    dims = inputs.uneven_dims(64, 32, 96, seed=1000)
    bh = [inputs.rhs(int(nx), int(ny), int(nz), seed=1000 + i) for i, (nx, ny, nz) in enumerate(dims)]
    bs = [dev(b) for b in bh]
    xs = [torch.zeros_like(b) for b in bs]
    h = smg.smg_batched_setup(dims)
    try:
        rc, its, relres = smg.smg_batched_solve(h, "fpcg", bs, xs)
    finally:
        smg.smg_batched_destroy(h)
    assert rc == smg.SMG_OK
    for i, b in enumerate(bh):
        xh = xs[i].cpu().numpy().reshape(b.shape)
        true = np.linalg.norm(b - D.lap7(xh)) / np.linalg.norm(b)
        assert true <= 1e-8, (i, true)
    for i in (0, 31, 63):  # sampled systems against the oracle's FP64 iteration counts
        nx, ny, nz = map(int, dims[i])
        ref = orc.krylov(bh[i], "fpcg", orc.SMG(nx, ny, nz, 1, 0), tol=1e-8, maxit=100)
        assert abs(int(its[i]) - ref["iters"]) <= 1, (i, its[i], ref["iters"])


def test_batched_apply_64_uneven_systems_full_config(smg, orc):
    """The persistent V-cycle of the batched workload itself (the same 64 systems, sides drawn in
    {32..96}, FP32 cycle, (1,0)), one launch through smg_batched_apply, against the oracle's cycle
    of every system element by element and plane by plane."""
    dims = inputs.uneven_dims(64, 32, 96, seed=1000)
    rh = [inputs.rhs(int(nx), int(ny), int(nz), seed=1000 + i) for i, (nx, ny, nz) in enumerate(dims)]
    r = [dev(v) for v in rh]
    out = [torch.empty_like(v) for v in r]
    h = smg.smg_batched_setup(dims)
    try:
        smg.smg_batched_apply(h, r, out)
    finally:
        smg.smg_batched_destroy(h)
    for i, (nx, ny, nz) in enumerate(dims):
        ref = orc.SMG(int(nx), int(ny), int(nz), 1, 0).apply(rh[i])
        assert_close(out[i].cpu().numpy(), ref, 2e-5, (int(nx), int(ny), int(nz)), f"system {i} {tuple(dims[i])}")


def _crop(a, z, y, x, r=3):
    """The part of the (2r+1)^3 neighbourhood of (z, y, x) inside the grid, and the point's index in
    it.  Clipped, not zero-filled: the network pads every layer with zeros at the grid boundary,
    which the oracle reproduces at the crop's edges exactly where they are grid edges; elsewhere
    the crop edge is r = 3 away, beyond the receptive field."""
    nz, ny, nx = a.shape
    zs, ys, xs_ = max(z - r, 0), max(y - r, 0), max(x - r, 0)
    ze, ye, xe = min(z + r + 1, nz), min(y + r + 1, ny), min(x + r + 1, nx)
    return a[zs:ze, ys:ye, xs_:xe], (z - zs, y - ys, x - xs_)


@pytest.mark.parametrize("act,tol", [("fp32", 1e-5), ("bf16", 1e-2)])
def test_learned_correction_256cube_sampled_points(smg, orc, act, tol):
    n = 256
    w = inputs.net_init_weights(seed=141, last_scale=1.0)
    if act == "bf16":
        w = (smg.bf16_bits(w).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    rho = inputs.rhs(n, n, n, seed=142)
    d = torch.empty(rho.size, dtype=torch.float64, device="cuda")
    smg.smg_net_forward((n, n, n), act, w, dev(rho), d)
    delta = d.cpu().numpy().reshape(n, n, n)
    scale = np.sqrt(np.mean(delta ** 2))
    rng = np.random.default_rng(143)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, 128, 255)] + [tuple(rng.integers(0, n, 3)) for _ in range(24)]
    for (z, y, x) in pts:
        c, q = _crop(rho, z, y, x)
        ref = orc.net_forward(w, np.ascontiguousarray(c), act_bf16=(act == "bf16"))[q]
        assert abs(delta[z, y, x] - ref) <= tol * scale, ((z, y, x), delta[z, y, x], ref)
