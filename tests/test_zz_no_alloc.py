"""smg_apply_A_dot_static: the allocation-free operator + inner product, checked on two calls in
a row against the oracle's operator (oracle.apply_A, element by element) and an FP64 NumPy inner
product, and against the library's regular entry point smg_apply_A on the same inputs.

It serves callers that cannot allocate device memory where they need the product (a host
framework that owns all device allocations, or a section where cudaMalloc must not run).  The
file sorts last so that a run stopping at the first failure has run every other test first.
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


@pytest.mark.parametrize("shape", [(37, 21, 13), (128, 128, 128), (1, 1, 5)])
def test_static_scratch_entry_point_matches_oracle_and_apply_A(smg, orc, shape):
    nx, ny, nz = shape
    with smg.Handle(nx, ny, nz) as h:
        for seed in (31, 32):  # two calls in a row share (and must reset) the static scratch
            uh = inputs.rhs(nx, ny, nz, seed=seed)
            u = torch.from_numpy(uh.ravel().copy()).cuda()
            ref = torch.empty_like(u)
            smg.smg_apply_A(h.h, u, ref)
            out = torch.full_like(u, float("nan"))
            dot = torch.zeros(1, dtype=torch.float64, device="cuda")
            smg.smg_apply_A_dot_static(nx, ny, nz, u, out, dot)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            Au = orc.apply_A(uh).ravel()
            # FP64 stencil on both sides, summation order aside: 1e-15 norm- and element-wise
            assert_close(got, Au, 1e-15, None, "A u vs the oracle")
            assert_close(got, ref.cpu().numpy(), 1e-15, None, "vs smg_apply_A")
            d_ref = float(np.dot(uh.ravel(), Au))
            assert abs(float(dot[0]) - d_ref) <= 1e-12 * abs(d_ref)


def test_static_scratch_entry_point_rejects_oversize(smg):
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(smg.SMGError) as e:
        smg.smg_apply_A_dot_static(512, 512, 129, u, u, u)  # 33,816,576 > 33,554,432 points
    assert e.value.code == smg.SMG_ERR_ARG
    assert "33,554,432" in str(e.value)
