"""The C oracle built with OpenMP gives bitwise the same results on one thread and on many: the
planes of one colour, the lines of one colour and the points of a transfer are independent, and
every output is computed in a fixed order (so the timed multi-core CPU baseline is the same
computation as the single-thread one)."""
import os

import numpy as np
import pytest

from paper_1212_6680_gb300 import inputs


@pytest.mark.parametrize("shape,npost", [((24, 20, 18), 1), ((33, 17, 40), 0), ((16, 16, 3), 1)])
def test_threads_do_not_change_results(orc, shape, npost):
    nx, ny, nz = shape
    b = inputs.rhs(nx, ny, nz, seed=5)
    out = []
    for nt in (1, max(2, os.cpu_count() or 2)):
        orc.set_threads(nt)
        T = orc.SMG(nx, ny, nz, 1, npost)
        s = T.apply(b)
        res = orc.krylov(b, "fpcg", T, tol=1e-10, maxit=60)
        out.append((s, res["x"], res["iters"], orc.apply_A(b)))
    orc.set_threads(1)
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]
    assert np.array_equal(out[0][3], out[1][3])
