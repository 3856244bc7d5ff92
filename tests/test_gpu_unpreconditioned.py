"""Krylov without a preconditioner (T = I, SMG_OPT_PRECOND = 0): plain CG by eq. (1) and by eq. (2)
and steepest descent (PSD with T = I), the comparison of section 2 and figures 1-2.  Iteration
counts against the oracle's (smg=None), the identity of eq. (1) and eq. (2) for SPD T, and steepest
descent far behind."""
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


def solve(smg, shape, variant, maxit, prec="fp64"):
    nx, ny, nz = shape
    b = torch.from_numpy(inputs.rhs(nx, ny, nz, seed=0).ravel().copy()).cuda()
    x = torch.zeros_like(b)
    h = smg.smg_setup(nx, ny, nz, 1, 0)
    try:
        smg.smg_set_precision(h, prec)
        smg.smg_set_option(h, smg.SMG_OPT_PRECOND, 0)
        rc, it, rr = smg.krylov_solve(h, variant, b, x, 1e-8, maxit, check=False)
    finally:
        smg.smg_destroy(h)
    return rc, it, rr, x.cpu().numpy()


@pytest.mark.parametrize("shape", [(16, 16, 16), (24, 12, 20)])
def test_unpreconditioned_cg_matches_oracle(smg, orc, shape):
    nx, ny, nz = shape
    b = inputs.rhs(nx, ny, nz, seed=0)
    for v in ("pcg", "fpcg"):
        ref = orc.krylov(b, v, None, tol=1e-8, maxit=500)
        assert ref["status"] == 0
        rc, it, rr, x = solve(smg, shape, v, 500)
        assert rc == smg.SMG_OK and rr <= 1e-8
        assert abs(it - ref["iters"]) <= 1, (v, it, ref["iters"])
        # the iterates agree with the oracle's to the tolerance the solve reaches
        assert np.linalg.norm(x - ref["x"].ravel()) <= 1e-6 * np.linalg.norm(ref["x"])


def test_eq1_eq2_identical_and_steepest_descent_slow(smg):
    shape = (32, 32, 32)
    rc1, it1, _, _ = solve(smg, shape, "pcg", 1000)
    rc2, it2, _, _ = solve(smg, shape, "fpcg", 1000)
    assert rc1 == smg.SMG_OK and rc2 == smg.SMG_OK
    assert abs(it1 - it2) <= max(2, it1 // 50)     # T = I is SPD: eq. (1) = eq. (2) up to rounding
    rc3, it3, rr3, _ = solve(smg, shape, "psd", 4 * it1)
    assert rc3 == smg.SMG_ERR_NOCONV and rr3 > 1e-8  # steepest descent: not there in 4x CG's count


def test_precond_option_validated(smg):
    h = smg.smg_setup(8, 8, 8, 1, 0)
    try:
        with pytest.raises(Exception):
            smg.smg_set_option(h, smg.SMG_OPT_PRECOND, 2)
    finally:
        smg.smg_destroy(h)
