"""LOBPCG with one eigenpair on the paper's 4n x 2n x 2n bricks (figures 8-9): the smallest
eigenvalue against the closed form, the iteration count against the LOBPCG oracle, and the
relation the paper's figure 9 shows -- without post-smoothing ((1,0)) LOBPCG takes more iterations
than with the balanced (1,1) cycle."""
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


def closed_form_smallest(nx, ny, nz):
    return sum(4 * np.sin(np.pi / (2 * (k + 1))) ** 2 for k in (nx, ny, nz))


def gpu_lobpcg(smg, shape, npost, prec="fp32"):
    nx, ny, nz = shape
    X = torch.from_numpy(np.ascontiguousarray(inputs.initial_block(nx, ny, nz, 1, seed=7)).ravel().copy()).cuda()
    with smg.Handle(nx, ny, nz, 1, npost, precision=prec) as h:
        rc, it, lam = smg.lobpcg_solve(h.h, 1, X, tol=1e-8, maxit=200)
    assert rc == smg.SMG_OK, smg.smg_last_error()
    return it, float(lam[0])


@pytest.mark.parametrize("n", [6, 10])
def test_lobpcg_brick_matches_oracle(smg, orc, n):
    from oracle import lobpcg as olob

    shape = (4 * n, 2 * n, 2 * n)
    nx, ny, nz = shape
    X0 = inputs.initial_block(nx, ny, nz, 1, seed=7)
    for npost in (1, 0):
        ref = olob.lobpcg((nz, ny, nx), X0.T, orc.SMG(nx, ny, nz, 1, npost), tol=1e-8, maxit=200)
        assert ref["converged"]
        it, lam = gpu_lobpcg(smg, shape, npost, "fp64")
        assert abs(lam - ref["lam"][0]) <= 1e-10 * ref["lam"][0]
        assert abs(it - ref["iters"]) <= 2, (npost, it, ref["iters"])


@pytest.mark.parametrize("n", [20, 40])
def test_lobpcg_brick_closed_form_and_figure9(smg, n):
    shape = (4 * n, 2 * n, 2 * n)
    it11, lam11 = gpu_lobpcg(smg, shape, 1)
    it10, lam10 = gpu_lobpcg(smg, shape, 0)
    ref = closed_form_smallest(*shape)
    assert abs(lam11 - ref) <= 1e-10 * ref and abs(lam10 - ref) <= 1e-10 * ref
    assert it10 >= it11
