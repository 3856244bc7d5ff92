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


def check_kind_layout(L, nx, elem, R, budget):
    """The checks of test_plane_layout_fits_and_does_not_overlap for a layout whose levels from
    solo_from on keep every line on each CTA's plan."""
    P, ny_m = L["P"], L["ny_m"]
    assert L["smem_bytes"] <= budget
    cap = L["smem_bytes"] // elem
    coef = (0, L["sum_ny"] * L["coef_per_line"])
    fs = (L["off_fs"], L["off_fs"] + 2 * L["MF"] * L["set_elems"])
    assert fs[0] >= coef[1]
    on_chip, in_global = [coef, fs], []
    for m in range(P):
        spread = R > 1 and m < L["solo_from"]
        loc = 2 * (((ny_m[m] + 1) // 2 + R - 1) // R) if spread else ny_m[m]
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


@pytest.mark.parametrize("elem", [4, 8])
@pytest.mark.parametrize("R", [1, 2, 4, 16])
@pytest.mark.parametrize("solo", [0, 8, 32])
@pytest.mark.parametrize("nx,ny", [(1, 1), (32, 32), (128, 128), (96, 57), (256, 256), (160, 512), (200, 96),
                                   (33, 3)])
def test_shortened_step_layout_fits_and_does_not_overlap(smg, nx, ny, elem, R, solo):
    """Kind 1 (the shortened-step cycle): every 2D level's factor sets on chip, and on a cluster the
    levels of at most `solo` lines held whole by the first CTA only where the spread plan's on-chip
    arrays all stay on chip."""
    L = smg.smg_plane_layout_kind(nx, ny, elem, R, 1, solo)
    P = L["P"]
    if L["smem_bytes"] == 0 or L["smem_bytes"] > BUDGET - 1024 or L["MF"] != P:
        # the coefficient table and the factor sets alone exceed the budget: the library does not
        # run the shortened-step cycle on this plane (it takes the general one)
        assert 2 * P * L["set_elems"] * elem + L["sum_ny"] * L["coef_per_line"] * elem > BUDGET - 1024 - 4096
        return
    if R == 1 or solo == 0:
        assert L["solo_from"] == P
    else:
        sf = L["solo_from"]
        assert sf == P or (1 <= sf <= P - 2 and L["ny_m"][sf] <= solo)
        if sf < P:  # the spread plan keeps no array on chip that this one moves off
            base = smg.smg_plane_layout_kind(nx, ny, elem, R, 1, 0)
            assert (L["u_mask"] & base["u_mask"]) == base["u_mask"]
            assert (L["g_mask"] & base["g_mask"]) == base["g_mask"]
    check_kind_layout(L, nx, elem, R, BUDGET)


@pytest.mark.parametrize("elem", [4, 8])
@pytest.mark.parametrize("R", [1, 2, 8, 16])
@pytest.mark.parametrize("nx,ny", [(513, 1), (600, 20), (1280, 80), (2048, 512), (777, 33), (1536, 5), (257, 3),
                                   (320, 20), (512, 32), (480, 240), (300, 512)])
def test_wide_line_layout_fits_and_does_not_overlap(smg, nx, ny, elem, R):
    """Kind 2 (lines of 257-2048 rows in segments of 8 or 16 rows per lane): no factor sets on
    chip, 2 KB left for the kernel's own shared arrays."""
    L = smg.smg_plane_layout_kind(nx, ny, elem, R, 2)
    assert L["MF"] == 0 and L["K"] == (16 if nx > 512 else 8) and L["solo_from"] == L["P"]
    if L["smem_bytes"] == 0:
        assert R > 1
        return
    check_kind_layout(L, nx, elem, R, BUDGET - 2048)


def test_plane_layout_kind_rejects_bad_arguments(smg):
    for args in ((300, 8, 4, 1, 1, 8), (256, 8, 4, 1, 2, 8), (2049, 8, 4, 1, 2, 8), (8, 8, 4, 1, 3, 8),
                 (8, 8, 4, 3, 1, 8), (8, 8, 4, 2, 1, -1)):
        with pytest.raises(Exception):
            smg.smg_plane_layout_kind(*args)
    # kind 0 is smg_plane_layout's plan
    a, b = smg.smg_plane_layout(96, 57, 4, 2), smg.smg_plane_layout_kind(96, 57, 4, 2, 0)
    assert all(a[k] == b[k] for k in a)


def test_plane_layout_rejects_bad_arguments(smg):
    for args in ((0, 8, 4, 1), (8, 513, 4, 1), (8, 8, 2, 1), (8, 8, 4, 3)):
        with pytest.raises(Exception):
            smg.smg_plane_layout(*args)
