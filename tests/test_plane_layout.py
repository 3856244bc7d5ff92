"""Host logic of the plane relaxation's memory plan (smg_plane_layout, no device): for one CTA per
plane and for clusters of 2..16 CTAs, in FP32 and FP64 arithmetic, over plane sizes up to the
library's limits, the shared-memory plan stays within the 227 KB a CTA may use, its regions
(coefficient table, line-solver factor sets, the 2D-cycle arrays kept on chip) do not overlap,
and the arrays left in the global slot do not overlap and fit in it."""
import pytest

BUDGET = 227 * 1024


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    return m


def a4(v):
    return (v + 3) & ~3


def disjoint(intervals):
    iv = sorted(i for i in intervals if i[1] > i[0])
    return all(iv[k][1] <= iv[k + 1][0] for k in range(len(iv) - 1))


@pytest.mark.parametrize("elem", [4, 8])
@pytest.mark.parametrize("R", [1, 2, 4, 16])
@pytest.mark.parametrize("nx,ny", [(1, 1), (32, 32), (128, 128), (96, 57), (256, 256), (512, 64), (160, 512),
                                   (512, 512), (33, 3)])
def test_plane_layout_fits_and_does_not_overlap(smg, nx, ny, elem, R):
    L = smg.smg_plane_layout(nx, ny, elem, R)
    P, ny_m = L["P"], L["ny_m"]
    assert len(ny_m) == P and ny_m[0] == ny and ny_m[-1] == 1
    if L["smem_bytes"] == 0:
        assert R > 1  # a cluster layout that does not fit is reported as unusable, never planned over budget
        return
    assert L["smem_bytes"] <= BUDGET
    cap = L["smem_bytes"] // elem
    coef = (0, L["sum_ny"] * L["coef_per_line"])
    fs = (L["off_fs"], L["off_fs"] + 2 * L["MF"] * L["set_elems"])
    assert fs[0] >= coef[1]
    on_chip, in_global = [coef, fs], []
    for m in range(P):
        loc = ny_m[m] if R == 1 else 2 * (((ny_m[m] + 1) // 2 + R - 1) // R)
        for mask, off in ((L["u_mask"], L["off_u"][m]), (L["g_mask"], L["off_g"][m])):
            if (mask >> m) & 1:
                iv = (off, off + a4(nx * loc))
                assert iv[0] >= fs[1] and iv[1] <= cap, (m, iv, cap)
                on_chip.append(iv)
            else:
                iv = (off, off + a4(nx * ny_m[m]))
                assert iv[1] <= L["ws_elems"], (m, iv, L["ws_elems"])
                in_global.append(iv)
    assert disjoint(on_chip) and disjoint(in_global)
    assert L["MF"] >= 1 and nx <= 32 * L["K"]


def test_plane_layout_rejects_bad_arguments(smg):
    for args in ((0, 8, 4, 1), (8, 513, 4, 1), (8, 8, 2, 1), (8, 8, 4, 3)):
        with pytest.raises(Exception):
            smg.smg_plane_layout(*args)
