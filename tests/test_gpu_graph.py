"""The device-side solve loop (SMG_OPT_GRAPH = 1, the default): krylov_solve's iterations run as one
CUDA graph whose conditional while node repeats the V-cycle and the four Krylov kernels until the
recurrence residual meets tol.  It launches the same kernels in the same order on the same data
as the host loop (SMG_OPT_GRAPH = 0), so the two give bit-identical iterates, iteration counts,
residual histories and launch counts."""
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


def solve(smg, shape, variant, prec, graph, maxit=40, npost=0, precond=1, x_new=False, fused=1, tol=1e-8):
    nx, ny, nz = shape
    b = torch.from_numpy(inputs.rhs(nx, ny, nz, seed=3).ravel().copy()).cuda()
    h = smg.smg_setup(nx, ny, nz, 1, npost)
    try:
        smg.smg_set_precision(h, prec)
        smg.smg_set_option(h, smg.SMG_OPT_GRAPH, graph)
        smg.smg_set_option(h, smg.SMG_OPT_PRECOND, precond)
        smg.smg_set_option(h, smg.SMG_OPT_FUSED_TAIL, fused)
        x = torch.zeros_like(b)
        out = []
        for rep in range(2):  # a second solve on the same handle (the graph is reused or rebuilt)
            if x_new and rep == 1:
                x = torch.zeros_like(b)
            x.zero_()
            l0 = smg.smg_launch_count(h)
            rc, it, rr = smg.krylov_solve(h, variant, b, x, tol, maxit, check=False)
            out.append((rc, it, rr, x.cpu().numpy().copy(), smg.smg_krylov_history(h), smg.smg_launch_count(h) - l0))
    finally:
        smg.smg_destroy(h)
    return out


def same(a, b):
    for (rc1, it1, rr1, x1, h1, l1), (rc2, it2, rr2, x2, h2, l2) in zip(a, b):
        assert (rc1, it1, l1) == (rc2, it2, l2)
        assert rr1 == rr2
        assert np.array_equal(x1, x2)
        assert np.array_equal(h1, h2)


@pytest.mark.parametrize("variant", ["pcg", "fpcg", "psd"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_device_loop_is_bitwise_the_host_loop(smg, variant, prec):
    g = solve(smg, (40, 36, 33), variant, prec, 1)
    h = solve(smg, (40, 36, 33), variant, prec, 0)
    same(g, h)
    assert g[0][1] > 3 and len(g[0][4]) == g[0][1] + 1


@pytest.mark.parametrize("maxit", [0, 1, 3])
def test_device_loop_stops_at_maxit(smg, maxit):
    g = solve(smg, (24, 24, 24), "fpcg", "fp32", 1, maxit=maxit)
    h = solve(smg, (24, 24, 24), "fpcg", "fp32", 0, maxit=maxit)
    same(g, h)
    assert g[0][1] == maxit and g[0][0] == smg.SMG_ERR_NOCONV


def test_device_loop_stalled_pcg_and_new_iterate_buffer(smg):
    """PCG by eq. (1) with the nonsymmetric (1,0) cycle stalls and ends at maxit; the second solve
    writes a different x buffer (the graph is rebuilt for it)."""
    g = solve(smg, (32, 32, 32), "pcg", "fp64", 1, maxit=25, x_new=True)
    h = solve(smg, (32, 32, 32), "pcg", "fp64", 0, maxit=25, x_new=True)
    same(g, h)


@pytest.mark.parametrize("precond", [0, 1])
def test_device_loop_wide_lines_and_no_preconditioner(smg, precond):
    g = solve(smg, (600, 10, 8), "fpcg", "fp32", 1, precond=precond, maxit=60)
    h = solve(smg, (600, 10, 8), "fpcg", "fp32", 0, precond=precond, maxit=60)
    same(g, h)


@pytest.mark.parametrize("variant", ["pcg", "fpcg", "psd"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("graph", [0, 1])
def test_fused_krylov_tail_is_bitwise_the_four_kernels(smg, variant, prec, graph):
    """SMG_OPT_FUSED_TAIL: the iteration's Krylov part as one cooperative kernel with grid-wide
    barriers gives the same bits as the four separate kernels (same grid, chunks and reductions)."""
    f = solve(smg, (40, 36, 32), variant, prec, graph, fused=1)
    u = solve(smg, (40, 36, 32), variant, prec, graph, fused=0)
    same(f, u)


def test_fused_krylov_tail_128cube(smg):
    f = solve(smg, (128, 128, 128), "fpcg", "fp32", 1, fused=1)
    u = solve(smg, (128, 128, 128), "fpcg", "fp32", 1, fused=0)
    same(f, u)
    assert f[0][0] == smg.SMG_OK


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_device_loop_tight_tolerance_with_true_residual_restarts(smg, prec):
    """At tol = 1e-13 the recurrence residual of a reduced-precision cycle can pass the test while
    the true residual does not; the host then continues from the true residual (beta = 0) and
    relaunches the device loop.  Whatever path a solve takes, both loops take the same one."""
    g = solve(smg, (48, 40, 36), "fpcg", prec, 1, maxit=80, tol=1e-13)
    h = solve(smg, (48, 40, 36), "fpcg", prec, 0, maxit=80, tol=1e-13)
    same(g, h)
