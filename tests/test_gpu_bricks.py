"""The paper's brick sweep (figures 4, 5 and 7: 16n x n x n bricks, long in x) on the GPU path.

For n = 10, 16, 20 every Krylov variant (PCG eq. (1), FPCG eq. (2), PSD) with the (1,1) and the
(1,0) FP64 cycle takes the oracle's iteration count (+-1, or both stop at maxit), and at every n,
up to the largest brick whose x-lines a warp solves (16n = 512), the counts keep the relations the
paper's figures show: eq. (1) = eq. (2) with the balanced cycle, PSD 0-3 more; without
post-smoothing FPCG and PSD close and eq. (1) far behind.  The FP32 cycle matches the FP64
count within one iteration.
"""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1212_6680_gb300 import inputs  # noqa: E402

MAXIT = 40


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    assert torch.cuda.is_available()
    return m


def gpu_counts(smg, n, prec="fp64"):
    nx, ny, nz = 16 * n, n, n
    b = torch.from_numpy(inputs.rhs(nx, ny, nz, seed=0).ravel().copy()).cuda()
    x = torch.zeros_like(b)
    out = {}
    for npost in (1, 0):
        h = smg.smg_setup(nx, ny, nz, 1, npost)
        try:
            smg.smg_set_precision(h, prec)
            for v in ("pcg", "fpcg", "psd"):
                x.zero_()
                rc, it, rr = smg.krylov_solve(h, v, b, x, 1e-8, MAXIT, check=False)
                assert rc in (smg.SMG_OK, smg.SMG_ERR_NOCONV)
                out[f"{v}1{npost}"] = it if rc == smg.SMG_OK else None
                if rc == smg.SMG_OK:
                    assert rr <= 1e-8
        finally:
            smg.smg_destroy(h)
    return out


def check_relations(c):
    assert c["pcg11"] is not None and c["pcg11"] == c["fpcg11"]
    assert 0 <= c["psd11"] - c["pcg11"] <= 3
    assert 0 <= c["psd10"] - c["fpcg10"] <= 2
    assert c["pcg10"] is None or c["pcg10"] > 2 * c["fpcg10"]


@pytest.mark.parametrize("n", [10, 16, 20])
def test_brick_counts_match_oracle(smg, orc, n):
    nx, ny, nz = 16 * n, n, n
    b = inputs.rhs(nx, ny, nz, seed=0)
    ref = {}
    for npost in (1, 0):
        T = orc.SMG(nx, ny, nz, 1, npost)
        for v in ("pcg", "fpcg", "psd"):
            o = orc.krylov(b, v, T, tol=1e-8, maxit=MAXIT)
            ref[f"{v}1{npost}"] = o["iters"] if o["status"] == 0 else None
    got = gpu_counts(smg, n)
    for k, r in ref.items():
        if r is None:
            assert got[k] is None, (k, got[k])
        else:
            assert got[k] is not None and abs(got[k] - r) <= 1, (k, got[k], r)
    check_relations(got)


def test_largest_brick_relations_and_fp32_cycle(smg):
    c64 = gpu_counts(smg, 32)
    check_relations(c64)
    c32 = gpu_counts(smg, 32, "fp32")
    assert c32["fpcg10"] is not None and abs(c32["fpcg10"] - c64["fpcg10"]) <= 1
    assert c32["pcg11"] is not None and abs(c32["pcg11"] - c64["pcg11"]) <= 1
