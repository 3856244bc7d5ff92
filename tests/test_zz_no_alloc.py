"""smg_apply_A_dot_static: the allocation-free operator + inner product, checked against the
regular entry point smg_apply_A on the same inputs, on two calls in a row.

It serves callers that cannot allocate device memory where they need the product (a host
framework that owns all device allocations, or a section where cudaMalloc must not run).  The
file sorts last so that a run stopping at the first failure has run every other test first.
"""
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


@pytest.mark.parametrize("shape", [(37, 21, 13), (128, 128, 128), (1, 1, 5)])
def test_static_scratch_entry_point_matches_apply_A(smg, shape):
    nx, ny, nz = shape
    with smg.Handle(nx, ny, nz) as h:
        for seed in (31, 32):  # two calls in a row share (and must reset) the static scratch
            u = torch.from_numpy(inputs.rhs(nx, ny, nz, seed=seed).ravel().copy()).cuda()
            ref = torch.empty_like(u)
            smg.smg_apply_A(h.h, u, ref)
            out = torch.full_like(u, float("nan"))
            dot = torch.zeros(1, dtype=torch.float64, device="cuda")
            smg.smg_apply_A_dot_static(nx, ny, nz, u, out, dot)
            torch.cuda.synchronize()
            # same FP64 stencil on both sides: relative 1e-15 (the tests' FP64 operator tolerance)
            err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
            assert err <= 1e-15, err
            d_ref = float(torch.dot(u, ref))
            assert abs(float(dot[0]) - d_ref) <= 1e-12 * abs(d_ref)


def test_static_scratch_entry_point_rejects_oversize(smg):
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(smg.SMGError) as e:
        smg.smg_apply_A_dot_static(512, 512, 129, u, u, u)  # 33,816,576 > 33,554,432 points
    assert e.value.code == smg.SMG_ERR_ARG
    assert "33,554,432" in str(e.value)
