"""Parity of the SMG set-up (section 3's semicoarsening hierarchy) between the library's host
set-up code, which every GPU solve uses, and the oracle's independent construction: per z-level
the z-couplings M, K and interpolation weights, and per plane and 2D level the y-couplings S, T
and weights.  Host only (smg_setup_coefs touches no device)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    return m


SHAPES = [(8, 8, 8), (5, 7, 9), (12, 13, 32), (9, 33, 17), (3, 1, 6), (4, 6, 1), (6, 2, 2)]


@pytest.mark.parametrize("shape", SHAPES)
def test_setup_coefficients_match_oracle(smg, orc, shape):
    nx, ny, nz = shape
    T = orc.SMG(nx, ny, nz, 1, 1)
    L = T.num_levels()
    P = T.plane_num_levels()
    for l in range(L):
        M, K, wm, wp = T.level_coefs(l)
        for z in range(T.level_nz(l)):
            for m in range(P):
                zc, lines = smg.smg_setup_coefs(nx, ny, nz, l, z, m)
                ref_z = np.concatenate([M[z], K[z], [wm[z], wp[z]]])
                assert np.allclose(zc, ref_z, rtol=1e-13, atol=1e-15), (l, z, zc, ref_z)
                S, Tm, swm, swp = T.plane_coefs(l, z, m)
                assert lines.shape[0] == S.shape[0] == T.plane_level_ny(m)
                ref_l = np.concatenate([S, Tm, swm[:, None], swp[:, None]], axis=1)
                assert np.allclose(lines, ref_l, rtol=1e-13, atol=1e-15), (l, z, m)


def test_setup_coefficients_reject_bad_indices(smg):
    with pytest.raises(Exception):
        smg.smg_setup_coefs(8, 8, 8, 9, 0, 0)
    with pytest.raises(Exception):
        smg.smg_setup_coefs(8, 8, 8, 0, 8, 0)
    with pytest.raises(Exception):
        smg.smg_setup_coefs(0, 8, 8, 0, 0, 0)


@pytest.mark.parametrize("shape", [(1 << 20, 8, 8), (8, 1 << 20, 8), (8, 8, 1 << 30), (8, 8, -3)])
def test_setup_coefficients_refuse_grids_smg_setup_refuses(smg, shape):
    """Sizes outside smg_setup's limits are refused before the host hierarchy is built (an
    nz of 2^30 would otherwise ask for tens of GB of host memory), and nothing is written."""
    import ctypes

    nx, ny, nz = shape
    zc = np.full(8, 7.0)
    lines = np.full((8, 8), 7.0)
    dp_ = ctypes.POINTER(ctypes.c_double)
    rc = smg._lib.smg_setup_coefs(nx, ny, nz, 0, 0, 0, zc.ctypes.data_as(dp_), lines.ctypes.data_as(dp_), None, None)
    assert rc == smg.SMG_ERR_ARG
    assert np.all(zc == 7.0) and np.all(lines == 7.0)
    with pytest.raises(Exception):
        smg.smg_setup_coefs(8, 8, 8, 0, 0, 5)  # m past the number of 2D levels
