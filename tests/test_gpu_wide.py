"""x-lines split over the warps of a team (plane_wide.cu): 513 <= nx <= 2048 in 512-row segments
(16 rows per lane), 257 <= nx <= 512 in 256-row segments (8 rows per lane), one warp each,
coupled exactly through a reduced system.
Checked element by element against the oracle's Thomas-algorithm line solves at the tolerances
of the other apply tests, and at the paper's brick 1280 x 80 x 80 (n = 80 of the 16n x n x n
family, section 3, figures 5-7): apply parity and the figure 5 residual histories."""
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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel().copy()).cuda()


# two, three and four segments; ragged last segments (600, 1100, 1290) and full ones (1024, 2048,
# with vector access); a single line per plane (ny = 1) and a single plane (nz = 1)
SHAPES = [(600, 20, 10), (1100, 12, 7), (1024, 16, 6), (2048, 8, 4), (1290, 9, 5), (777, 1, 6), (1536, 5, 1),
          (300, 7, 3), (512, 32, 12), (257, 9, 5), (480, 20, 6)]
TOL = {"fp64": 1e-12, "fp32": 2e-5, "bf16": 3e-2}


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("npre,npost", [(1, 0), (1, 1)])
def test_wide_lines_apply_matches_oracle(smg, orc, shape, prec, npre, npost):
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=17)
    ref = orc.SMG(nx, ny, nz, npre, npost).apply(r)
    h = smg.smg_setup(nx, ny, nz, npre, npost)
    try:
        smg.smg_set_precision(h, prec)
        rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
        smg.smg_apply(h, rd, sd)
        torch.cuda.synchronize()
        s = sd.cpu().numpy()
        smg.smg_apply(h, rd, sd)  # a fixed, linear preconditioner: the same result again
        assert np.array_equal(sd.cpu().numpy(), s)
    finally:
        smg.smg_destroy(h)
    assert_close(s, ref, TOL[prec], shape, f"{prec} wide lines {shape} ({npre},{npost})")


@pytest.mark.parametrize("shape", [(600, 20, 10), (1100, 12, 7), (2048, 8, 4), (1290, 9, 5), (777, 1, 6),
                                   (1536, 5, 1), (320, 20, 20), (512, 32, 12)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_wide_factor_tables_are_bitwise_the_on_the_fly_ones(smg, orc, shape, prec):
    """FP64 wide-line planes (the coarsest plane; every plane of the FP64 cycle) reading their
    line-solver data from tables formed once (SMG_OPT_WIDE_FACTORS = 1, the default) give the cycle
    bit for bit that forming the data inside the plane cycle gives."""
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=19)
    out = {}
    for wf in (1, 0):
        h = smg.smg_setup(nx, ny, nz, 1, 1)
        try:
            smg.smg_set_precision(h, prec)
            smg.smg_set_option(h, smg.SMG_OPT_WIDE_FACTORS, wf)
            rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
            smg.smg_apply(h, rd, sd)
            torch.cuda.synchronize()
            out[wf] = sd.cpu().numpy()
        finally:
            smg.smg_destroy(h)
    assert np.array_equal(out[0], out[1])
    assert_close(out[1], orc.SMG(nx, ny, nz, 1, 1).apply(r), TOL[prec], shape, prec)


@pytest.mark.parametrize("shape", [(600, 20, 10), (1100, 12, 7), (2048, 8, 4), (1290, 9, 5), (777, 1, 6),
                                   (1536, 5, 1), (1280, 40, 3), (320, 20, 20), (512, 32, 12)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_wide_planes_on_clusters_are_bitwise_one_cta(smg, orc, shape, prec):
    """Wide-line planes spread over thread-block clusters (each CTA relaxing the lines it owns,
    reading the others' through distributed shared memory) give the cycle of one CTA per plane bit
    for bit: every line is solved by the same code on the same data."""
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=23)
    out = {}
    for one in (False, True):
        h = smg.smg_setup(nx, ny, nz, 1, 1)
        try:
            smg.smg_set_precision(h, prec)
            if one:
                smg.smg_set_option(h, smg.SMG_OPT_CLUSTER_MAX, 1)
                smg.smg_set_option(h, smg.SMG_OPT_CLUSTER_MAX32, 1)
            rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
            smg.smg_apply(h, rd, sd)
            torch.cuda.synchronize()
            out[one] = sd.cpu().numpy()
        finally:
            smg.smg_destroy(h)
    assert np.array_equal(out[False], out[True])
    assert_close(out[False], orc.SMG(nx, ny, nz, 1, 1).apply(r), TOL[prec], shape, prec)


@pytest.mark.parametrize("shape", [(600, 20, 10), (1100, 12, 7), (2048, 8, 4), (1290, 9, 5), (777, 1, 6),
                                   (1536, 5, 1), (1280, 40, 3), (320, 20, 20), (512, 32, 12), (257, 9, 5)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("npre,npost", [(1, 0), (1, 1)])
def test_wide_shortened_step_order_is_bitwise_the_general_one(smg, orc, shape, prec, npre, npost):
    """The wide-line kernel's shortened step order (SMG_OPT_LEAN = 1, the default: each step that
    fills a 2D level's right-hand side also solves that level's even lines) performs the same line
    solves on the same data as the general order (SMG_OPT_LEAN = 0): the cycle is bit for bit the
    same, on one CTA or a cluster per plane."""
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=31)
    out = {}
    for lean in (1, 0):
        h = smg.smg_setup(nx, ny, nz, npre, npost)
        try:
            smg.smg_set_precision(h, prec)
            smg.smg_set_option(h, smg.SMG_OPT_LEAN, lean)
            rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
            smg.smg_apply(h, rd, sd)
            torch.cuda.synchronize()
            out[lean] = sd.cpu().numpy()
        finally:
            smg.smg_destroy(h)
    assert np.array_equal(out[0], out[1])
    assert_close(out[1], orc.SMG(nx, ny, nz, npre, npost).apply(r), TOL[prec], shape, prec)


@pytest.mark.parametrize("shape", [(320, 20, 20), (512, 32, 12), (300, 7, 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_two_warp_lines_and_one_warp_lines_both_match_oracle(smg, orc, shape, prec):
    """Lines of 257-512 rows: two warps of 8 rows per lane (the wide-line kernel, the default) and
    one warp of 16 (SMG_OPT_WIDE_MIN_ROWS = 513: the general plane cycle) solve the same line
    systems exactly; both cycles match the oracle at the precision's tolerance."""
    nx, ny, nz = shape
    r = inputs.rhs(nx, ny, nz, seed=29)
    ref = orc.SMG(nx, ny, nz, 1, 0).apply(r)
    for wmin in (257, 513):
        h = smg.smg_setup(nx, ny, nz, 1, 0)
        try:
            smg.smg_set_precision(h, prec)
            smg.smg_set_option(h, smg.SMG_OPT_WIDE_MIN_ROWS, wmin)
            rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
            smg.smg_apply(h, rd, sd)
            torch.cuda.synchronize()
            s = sd.cpu().numpy()
        finally:
            smg.smg_destroy(h)
        assert_close(s, ref, TOL[prec], shape, f"{prec} lines of {nx} rows, wide from {wmin}")


def test_wide_lines_batched_apply_matches_single(smg, orc):
    """Several right-hand sides per launch (LOBPCG's block preconditioner) on wide lines."""
    nx, ny, nz, m = 700, 6, 5, 3
    R = np.stack([inputs.rhs(nx, ny, nz, seed=30 + k).ravel() for k in range(m)])
    ref = np.stack([orc.SMG(nx, ny, nz, 1, 0).apply(R[k]) for k in range(m)])
    with smg.Handle(nx, ny, nz, 1, 0) as h:
        rd = dev(R)
        sd = torch.empty_like(rd)
        smg.smg_apply_batched(h.h, m, rd, sd)
        torch.cuda.synchronize()
        s = sd.cpu().numpy().reshape(m, -1)
    for k in range(m):
        assert_close(s[k], ref[k].ravel(), 1e-12, (nx, ny, nz), f"rhs {k}")


def test_setup_refuses_lines_past_2048(smg):
    with pytest.raises(Exception):
        smg.smg_setup(2049, 4, 4, 1, 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_brick_n80_apply_matches_oracle(smg, orc, prec):
    """The paper's brick at n = 80: 1280 x 80 x 80 = 8.2M unknowns, x-lines of 1280 rows."""
    nx, ny, nz = 1280, 80, 80
    r = inputs.rhs(nx, ny, nz, seed=5)
    ref = orc.SMG(nx, ny, nz, 1, 0).apply(r)
    h = smg.smg_setup(nx, ny, nz, 1, 0)
    try:
        smg.smg_set_precision(h, prec)
        rd, sd = dev(r), torch.empty(nz * ny * nx, dtype=torch.float64, device="cuda")
        smg.smg_apply(h, rd, sd)
        torch.cuda.synchronize()
        s = sd.cpu().numpy()
    finally:
        smg.smg_destroy(h)
    assert_close(s, ref, TOL[prec], (nx, ny, nz), f"{prec} brick n=80")


@pytest.mark.parametrize("variant", ["pcg", "fpcg", "psd"])
def test_brick_n80_residual_history_figure5(smg, orc, variant):
    """Figure 5's experiment on its own brick (1280 x 80 x 80, SMG (1,0)): the GPU solve with the
    FP64 cycle follows the oracle's residual history entry by entry; PCG by eq. (1) stalls (its
    last four of 16 iterations cut the residual less than 2x; the oracle stalls near 2.4e-4, the
    paper's hypre run near 3e-2), while flexible PCG (eq. (2)) and PSD reach 1e-8 in at most 16
    iterations."""
    nx, ny, nz = 1280, 80, 80
    b = inputs.rhs(nx, ny, nz, seed=0)
    maxit = 16 if variant == "pcg" else 40
    ref = orc.krylov(b, variant, orc.SMG(nx, ny, nz, 1, 0), tol=1e-8, maxit=maxit)
    with smg.Handle(nx, ny, nz, 1, 0) as h:
        x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
        rc, it, relres = smg.krylov_solve(h.h, variant, dev(b), x, tol=1e-8, maxit=maxit, check=False)
        hist = smg.smg_krylov_history(h.h)
    assert len(hist) == it + 1 == len(ref["hist"]), (len(hist), it, len(ref["hist"]))
    assert np.all(np.abs(hist - ref["hist"]) <= 1e-6 * ref["hist"]), np.max(np.abs(hist - ref["hist"]) / ref["hist"])
    if variant == "pcg":
        assert rc == smg.SMG_ERR_NOCONV and hist[-1] > 1e-5 and hist[-1] > 0.5 * hist[-5]
    else:
        assert rc == smg.SMG_OK and hist[-1] <= 1e-8 and relres <= 1e-8 and it <= 16
