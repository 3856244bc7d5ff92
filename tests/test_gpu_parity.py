"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances:
  * FP64 cycle: relative 1e-12 per V-cycle (both sides follow the same sequence of exact
    line solves; they differ only in summation order and in the line-solve algorithm
    (partition + cyclic reduction vs Thomas), whose rounding differences are amplified at
    most by the line systems' condition number, below ~1e4 here).
  * FP32 cycle: relative 2e-5 per V-cycle (unit roundoff 6e-8 times the same amplification);
    BF16 storage: relative 3e-2 (storage roundoff 4e-3 per level vector, a few levels deep).
  * Krylov solves: true relative residual <= tol, checked independently with the oracle's
    operator, and iteration counts within +-1 of the oracle's FP64 run.
"""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


SHAPES = [(32, 32, 32), (33, 17, 20), (7, 5, 3), (1, 1, 8), (8, 1, 1), (5, 6, 1), (64, 48, 40), (130, 9, 6),
          (257, 4, 5), (96, 96, 9), (2, 3, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("npre,npost", [(1, 1), (1, 0), (2, 1)])
def test_apply_fp64_matches_oracle(smg, orc, shape, npre, npost):
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=11)
    ref = orc.SMG(nx, ny, nz, npre, npost).apply(r)
    with smg.Handle(nx, ny, nz, npre, npost) as h:
        rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
        smg.smg_apply(h.h, rd, sd)
        torch.cuda.synchronize()
        s = sd.cpu().numpy()
        # applying twice gives identical results (fixed, linear preconditioner)
        smg.smg_apply(h.h, rd, sd)
        assert np.array_equal(sd.cpu().numpy(), s)
    assert_close(s, ref, 1e-12, shape, f"FP64 cycle {shape} ({npre},{npost})")


@pytest.mark.parametrize("shape", [(256, 256, 2), (256, 200, 3)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("cluster_max", [16, 1])
def test_coarsest_plane_cluster_with_global_arrays(smg, orc, shape, prec, tol, cluster_max):
    """A 256-wide FP64 coarsest plane: spread over a cluster, the 2D-cycle arrays do not all fit
    in the cluster's shared memory, and the finest ones live in the cluster's global slot."""
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=13)
    ref = orc.SMG(nx, ny, nz, 1, 1).apply(r)
    h = smg.smg_setup(nx, ny, nz, 1, 1)
    try:
        smg.smg_set_precision(h, prec)
        smg.smg_set_option(h, smg.SMG_OPT_CLUSTER_MAX, cluster_max)
        rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
        smg.smg_apply(h, rd, sd)
        torch.cuda.synchronize()
        s = sd.cpu().numpy()
    finally:
        smg.smg_destroy(h)
    assert_close(s, ref, tol, shape, f"{prec} cluster_max {cluster_max}")


@pytest.mark.parametrize("cluster_max32", [0, 1, 2, 16])
def test_fp32_plane_clusters(smg, orc, cluster_max32):
    """FP32 256-wide planes on one CTA or spread over clusters (0 = the size-dependent default),
    with the arrays that do not fit on chip in global memory."""
    nx, ny, nz = 256, 96, 6
    r = inputs.rhs(nx, ny, nz, seed=17)
    ref = orc.SMG(nx, ny, nz, 1, 0).apply(r)
    h = smg.smg_setup(nx, ny, nz, 1, 0)
    try:
        smg.smg_set_precision(h, "fp32")
        smg.smg_set_option(h, smg.SMG_OPT_CLUSTER_MAX32, cluster_max32)
        rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
        smg.smg_apply(h, rd, sd)
        torch.cuda.synchronize()
        s = sd.cpu().numpy()
    finally:
        smg.smg_destroy(h)
    assert_close(s, ref, 2e-5, (nx, ny, nz), f"FP32 cluster_max32 {cluster_max32}")


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("bf16", 3e-2)])
@pytest.mark.parametrize("shape", [(32, 32, 32), (33, 17, 20), (96, 96, 9)])
@pytest.mark.parametrize("npost", [1, 0])
def test_apply_mixed_precision_close_to_oracle(smg, orc, prec, tol, shape, npost):
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=12)
    ref = orc.SMG(nx, ny, nz, 1, npost).apply(r)
    with smg.Handle(nx, ny, nz, 1, npost, precision=prec) as h:
        sd = torch.empty(r.size, dtype=torch.float64, device="cuda")
        smg.smg_apply(h.h, dev(r), sd)
        s = sd.cpu().numpy()
    assert_close(s, ref, tol, shape, f"{prec} cycle {shape} (1,{npost})")


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("shape", [(128, 128, 16), (96, 80, 64), (33, 17, 20), (100, 3, 5), (5, 6, 1), (1, 1, 8),
                                   (256, 256, 8), (200, 96, 20), (160, 40, 12), (256, 130, 3)])
@pytest.mark.parametrize("npost", [1, 0])
def test_shortened_step_plane_cycle_is_bitwise_the_general_one(smg, orc, prec, shape, npost):
    """The FP32 plane kernel with fewer barrier-separated steps (SMG_OPT_LEAN = 1, the default for
    nx <= 256; clusters of 2-4 CTAs for 256-wide planes) does the same line solves in the same order
    as the general kernel: bit-identical cycles, and both within the precision's tolerance of the
    oracle."""
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=14)
    out = {}
    for lean in (1, 0):
        with smg.Handle(nx, ny, nz, 1, npost, precision=prec) as h:
            smg.smg_set_option(h.h, smg.SMG_OPT_LEAN, lean)
            sd = torch.empty(r.size, dtype=torch.float64, device="cuda")
            smg.smg_apply(h.h, dev(r), sd)
            out[lean] = sd.cpu().numpy()
    assert np.array_equal(out[0], out[1])
    assert_close(out[1], orc.SMG(nx, ny, nz, 1, npost).apply(r), 2e-5 if prec == "fp32" else 3e-2, shape, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(128, 128, 16), (256, 256, 2), (200, 96, 20), (96, 80, 64), (64, 64, 4)])
@pytest.mark.parametrize("threads", [512, 256])
def test_solo_coarse_levels_are_bitwise_the_spread_ones(smg, orc, prec, shape, threads):
    """Planes spread over a cluster with the coarse 2D levels held whole by the cluster's first CTA
    (SMG_OPT_SOLO = T: the levels of at most T lines) give bit-identical cycles to every level
    spread over the cluster: the same line solves in the same order, only their placement
    differs."""
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=15)
    out = {}
    for solo in (32, 8, 0):
        with smg.Handle(nx, ny, nz, 1, 1, precision=prec) as h:
            smg.smg_set_option(h.h, smg.SMG_OPT_THREADS, threads)
            smg.smg_set_option(h.h, smg.SMG_OPT_SOLO, solo)
            sd = torch.empty(r.size, dtype=torch.float64, device="cuda")
            smg.smg_apply(h.h, dev(r), sd)
            out[solo] = sd.cpu().numpy()
    assert np.array_equal(out[0], out[8]) and np.array_equal(out[0], out[32])
    assert_close(out[8], orc.SMG(nx, ny, nz, 1, 1).apply(r), 1e-12 if prec == "fp64" else 2e-5, shape, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("shape", [(32, 32, 32), (33, 17, 20), (7, 5, 3), (1, 1, 8), (5, 6, 1), (64, 48, 41),
                                   (24, 20, 127), (9, 7, 18), (16, 8, 10)])
@pytest.mark.parametrize("npost", [0, 1])
def test_column_restriction_is_bitwise_the_per_point_one(smg, orc, prec, shape, npost):
    """The residual + restriction walking four coarse planes per thread (each fine residual computed
    once, SMG_OPT_RESTRICT_COLUMN = 1, the default) gives the same cycle, bit for bit, as one coarse
    plane per thread, for one and for several right-hand sides, and both match the oracle."""
    nx, ny, nz = shape
    nb = 2
    R = np.stack([inputs.rhs(nx, ny, nz, seed=50 + j).ravel() for j in range(nb)])
    out = {}
    for col in (1, 0):
        with smg.Handle(nx, ny, nz, 1, npost, precision=prec) as h:
            smg.smg_set_option(h.h, smg.SMG_OPT_RESTRICT_COLUMN, col)
            Sd = torch.empty((nb, nx * ny * nz), dtype=torch.float64, device="cuda")
            smg.smg_apply_batched(h.h, nb, dev(R), Sd)
            out[col] = Sd.cpu().numpy()
    assert np.array_equal(out[0], out[1])
    tol = {"fp64": 1e-12, "fp32": 2e-5, "bf16": 3e-2}[prec]
    ref = orc.SMG(nx, ny, nz, 1, npost).apply(R[1].reshape(nz, ny, nx)).ravel()
    assert_close(out[1][1], ref, tol, shape, prec)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_column_restriction_large_launch_is_bitwise(smg, prec):
    """FP32 and BF16 storage walk columns only from 4M coarse points per launch (128 x 128 x 512:
    the finest restriction has 4M): bit-identical to one coarse plane per thread there too."""
    nx, ny, nz = 128, 128, 512
    r = inputs.rhs(nx, ny, nz, seed=51).ravel()
    out = {}
    for col in (1, 0):
        with smg.Handle(nx, ny, nz, 1, 0, precision=prec) as h:
            smg.smg_set_option(h.h, smg.SMG_OPT_RESTRICT_COLUMN, col)
            sd = torch.empty(r.size, dtype=torch.float64, device="cuda")
            smg.smg_apply(h.h, dev(r), sd)
            out[col] = sd.cpu().numpy()
    assert np.isfinite(out[1]).all() and np.abs(out[1]).max() > 0
    assert np.array_equal(out[0], out[1])


def test_apply_batched_matches_columns(smg, orc):
    nx, ny, nz, nb = 24, 20, 18, 3
    R = np.stack([inputs.rhs(nx, ny, nz, seed=20 + j).ravel() for j in range(nb)])
    T = orc.SMG(nx, ny, nz, 1, 0)
    with smg.Handle(nx, ny, nz, 1, 0) as h:
        Sd = torch.empty(nb * R.shape[1], dtype=torch.float64, device="cuda")
        smg.smg_apply_batched(h.h, nb, dev(R), Sd)
        S = Sd.cpu().numpy().reshape(nb, -1)
    for j in range(nb):
        assert_close(S[j], T.apply(R[j].reshape(nz, ny, nx)), 1e-12, (nx, ny, nz), f"column {j}")


def test_apply_A_matches_oracle(smg, orc):
    nx, ny, nz = 37, 21, 13
    u = inputs.rhs(nx, ny, nz, seed=3)
    with smg.Handle(nx, ny, nz) as h:
        o = torch.empty(u.size, dtype=torch.float64, device="cuda")
        smg.smg_apply_A(h.h, dev(u), o)
        assert_close(o.cpu().numpy(), orc.apply_A(u), 1e-15, None, "A u")


@pytest.mark.parametrize("variant", ["pcg", "fpcg", "psd"])
@pytest.mark.parametrize("npost", [1, 0])
def test_krylov_32cube_matches_oracle(smg, orc, variant, npost):
    n = 32
    b = inputs.rhs(n, n, n, seed=0)
    maxit = 100 if not (variant == "pcg" and npost == 0) else 25
    ref = orc.krylov(b, variant, orc.SMG(n, n, n, 1, npost), tol=1e-8, maxit=maxit)
    with smg.Handle(n, n, n, 1, npost) as h:
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        rc, it, relres = smg.krylov_solve(h.h, variant, dev(b), x, tol=1e-8, maxit=maxit)
        xh = x.cpu().numpy().reshape(b.shape)
    true = np.linalg.norm(b - orc.apply_A(xh)) / np.linalg.norm(b)
    assert abs(true - relres) <= 1e-3 * relres + 1e-15
    if ref["status"] == 0:
        assert rc == smg.SMG_OK
        assert true <= 1e-8
        assert abs(it - ref["iters"]) <= 1, (it, ref["iters"])
    else:  # eq. (1) with the nonsymmetric cycle stalls on both sides
        assert rc == smg.SMG_ERR_NOCONV and it == maxit
        assert true > 1e-8


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("variant", ["fpcg", "psd"])
def test_krylov_mixed_precision_reaches_tolerance(smg, orc, prec, variant):
    nx, ny, nz = 40, 33, 29
    b = inputs.rhs(nx, ny, nz, seed=1)
    ref = orc.krylov(b, variant, orc.SMG(nx, ny, nz, 1, 0), tol=1e-8, maxit=100)
    with smg.Handle(nx, ny, nz, 1, 0, precision=prec) as h:
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        rc, it, relres = smg.krylov_solve(h.h, variant, dev(b), x, tol=1e-8, maxit=100)
        xh = x.cpu().numpy().reshape(b.shape)
    assert rc == smg.SMG_OK
    assert np.linalg.norm(b - orc.apply_A(xh)) / np.linalg.norm(b) <= 1e-8
    # FP64 solution error of the mixed path vs the oracle's FP64 solve: both within tol of A^{-1} b
    assert_close(xh, ref["x"], 1e-5, (nx, ny, nz), "solution vs the oracle's FP64 solve")
    assert it <= ref["iters"] + (2 if prec == "fp32" else 6)


def test_krylov_host_pointers(smg, orc):
    nx, ny, nz = 20, 18, 16
    b = inputs.rhs(nx, ny, nz, seed=5).ravel().copy()
    x = np.zeros_like(b)
    with smg.Handle(nx, ny, nz, 1, 0, precision="fp32") as h:
        rc, it, relres = smg.krylov_solve(h.h, "fpcg", b, x, tol=1e-8, maxit=100)
    assert rc == smg.SMG_OK and relres <= 1e-8
    assert np.linalg.norm(b - orc.apply_A(x.reshape(nz, ny, nx)).ravel()) / np.linalg.norm(b) <= 1e-8


def test_krylov_maxit_zero_and_nan(smg):
    n = 8
    b = inputs.rhs(n, n, n, seed=2).ravel().copy()
    with smg.Handle(n, n, n) as h:
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        rc, it, relres = smg.krylov_solve(h.h, "fpcg", dev(b), x, maxit=0)
        assert rc == smg.SMG_ERR_NOCONV and it == 0 and abs(relres - 1.0) < 1e-12
        b[5] = np.nan
        rc, it, relres = smg.krylov_solve(h.h, "fpcg", dev(b), torch.zeros_like(x), maxit=10, check=False)
        assert rc == smg.SMG_ERR_NAN


def test_krylov_nonzero_initial_guess(smg, orc):
    n = 16
    b = inputs.rhs(n, n, n, seed=8)
    x0 = inputs.rhs(n, n, n, seed=9)
    with smg.Handle(n, n, n, 1, 1) as h:
        x = dev(x0)
        rc, it, relres = smg.krylov_solve(h.h, "pcg", dev(b), x, tol=1e-10, maxit=50)
        xh = x.cpu().numpy().reshape(b.shape)
    assert rc == smg.SMG_OK
    assert np.linalg.norm(b - orc.apply_A(xh)) / np.linalg.norm(b) <= 1e-10


def closed_form_smallest(nx, ny, nz, m):
    lx = 4 * np.sin(np.pi * np.arange(1, nx + 1) / (2 * (nx + 1))) ** 2
    ly = 4 * np.sin(np.pi * np.arange(1, ny + 1) / (2 * (ny + 1))) ** 2
    lz = 4 * np.sin(np.pi * np.arange(1, nz + 1) / (2 * (nz + 1))) ** 2
    return np.sort((lz[:, None, None] + ly[None, :, None] + lx[None, None, :]).ravel())[:m]


@pytest.mark.parametrize("shape,m,npost", [((16, 16, 16), 4, 0), ((12, 10, 14), 6, 1), ((20, 20, 20), 16, 0)])
def test_lobpcg_matches_closed_form(smg, shape, m, npost):
    nx, ny, nz = shape
    X0 = inputs.initial_block(nx, ny, nz, m, seed=7)
    with smg.Handle(nx, ny, nz, 1, npost) as h:
        X = dev(X0)
        rc, it, lam = smg.lobpcg_solve(h.h, m, X, tol=1e-8, maxit=200)
        Xh = X.cpu().numpy().reshape(m, -1)
    assert rc == smg.SMG_OK, smg.smg_last_error()
    ref = closed_form_smallest(nx, ny, nz, m)
    assert np.all(np.abs(lam - ref) <= 1e-10 * ref), (lam, ref)
    G = Xh @ Xh.T
    assert np.abs(G - np.eye(m)).max() <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_handles_with_different_layouts_coexist(smg, orc, prec):
    """A handle set up after another one, with the same x-line chunk but a smaller shared-memory
    layout, must not break the first handle's launches."""
    big, small = (96, 96, 24), (70, 6, 5)
    with smg.Handle(*big, 1, 1, precision=prec) as hb, smg.Handle(*small, 1, 1, precision=prec) as hs:
        for h, shape in ((hb, big), (hs, small), (hb, big)):
            u = inputs.rhs(*shape, seed=61)
            r = torch.from_numpy(u.ravel().copy()).cuda()
            s = torch.empty_like(r)
            smg.smg_apply(h.h, r, s)
            torch.cuda.synchronize()
            ref = orc.SMG(*shape, 1, 1).apply(u)
            assert_close(s.cpu().numpy(), ref, 1e-12 if prec == "fp64" else 2e-5, shape, f"{prec} {shape}")


def test_integer_pipe_conversions_match_hardware(smg):
    # the library's own FP32 <-> FP64 conversions against the hardware instructions, bit for bit:
    # random magnitudes over the whole float range, ties, carries into the exponent, overflow to
    # infinity, denormal results, zeros, infinities and NaN
    rng = np.random.default_rng(3)
    vals = [rng.standard_normal(200000) * np.exp(rng.uniform(-90, 90, 200000)),
            rng.uniform(-1, 1, 100000)]
    f = rng.standard_normal(50000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    vals += [f + ulp / 2, f - ulp / 2, f + ulp / 2 * (1 + 2.0 ** -40), f + ulp * 0.49999]  # ties and near-ties
    vals.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028235677973366e38, 3.4028235e38 * 1.0000001,
                          1.1754943508222875e-38, 1.17549e-38, 1e-40, -1e-45, 1.401298464324817e-45, 2.0 ** -126,
                          np.nextafter(2.0 ** 128, 0), 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1e300, -1e-300]))
    src = torch.from_numpy(np.concatenate(vals)).cuda()
    mism = torch.zeros(2, dtype=torch.int32, device="cuda")
    smg.smg_check_conversions(src, mism)
    assert mism.cpu().tolist() == [0, 0]


@pytest.mark.parametrize("variant,npost", [("fpcg", 0), ("psd", 0), ("pcg", 1), ("pcg", 0)])
def test_residual_history_matches_oracle(smg, orc, variant, npost):
    """The per-iteration relative residual ||r_k|| / ||b|| (figures 2 and 5) of the GPU solve with
    the FP64 cycle against the oracle's history on the same system: same length, and entry by
    entry within 1e-6 relative (the two sides differ by rounding only); with the nonsymmetric
    (1,0) cycle PCG by eq. (1) stalls on both sides (figure 5)."""
    n = 24
    b = inputs.rhs(n, n, n, seed=0)
    maxit = 30
    ref = orc.krylov(b, variant, orc.SMG(n, n, n, 1, npost), tol=1e-8, maxit=maxit)
    with smg.Handle(n, n, n, 1, npost) as h:
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        rc, it, relres = smg.krylov_solve(h.h, variant, dev(b), x, tol=1e-8, maxit=maxit, check=False)
        hist = smg.smg_krylov_history(h.h)
    assert len(hist) == it + 1 == len(ref["hist"]), (len(hist), it, len(ref["hist"]))
    assert abs(hist[0] - 1.0) <= 1e-14
    assert np.all(np.abs(hist - ref["hist"]) <= 1e-6 * ref["hist"]), np.max(np.abs(hist - ref["hist"]) / ref["hist"])
    if variant == "pcg" and npost == 0:
        assert rc == smg.SMG_ERR_NOCONV and hist[-1] > 1e-8
    else:
        assert rc == smg.SMG_OK and hist[-1] <= 1e-8
