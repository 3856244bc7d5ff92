"""Host logic of the wide-line tables' sharing (smg_plane_classes, no device): the planes of a
z-level fall into classes of bit-identical 2D hierarchies, one line-solver table per class.
Checked against the set-up's own coefficients (smg_setup_coefs) plane by plane and 2D level by
2D level: planes of one class agree in every coefficient, planes of different classes differ in
one, the classes are numbered in order of first appearance; for the paper's bricks (7-point
Laplacian, section 3) every level has at most three classes, so the tables shrink from one per
plane to one per class."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    return m


def levels(n):
    L = 1
    while n > 1:
        n //= 2
        L += 1
    return L


def hierarchy_of(smg, nx, ny, nz, l, z):
    """Every 2D level's coefficient lines of plane z of level l, concatenated."""
    out = []
    for m in range(levels(ny)):
        _, lines = smg.smg_setup_coefs(nx, ny, nz, l, z, m)
        out.append(lines)
    return np.concatenate(out)


@pytest.mark.parametrize("shape", [(320, 20, 20), (600, 20, 10), (1290, 9, 5), (777, 1, 6), (300, 7, 3), (257, 9, 33)])
def test_plane_classes_follow_the_coefficients(smg, shape):
    nx, ny, nz = shape
    for l in range(levels(nz)):
        count, cls = smg.smg_plane_classes(nx, ny, nz, l)
        nzl = len(cls)
        assert nzl >= 1 and cls[0] == 0 and count == cls.max() + 1
        # numbered in order of first appearance
        seen = []
        for c in cls:
            if c not in seen:
                seen.append(c)
        assert seen == list(range(count))
        hs = [hierarchy_of(smg, nx, ny, nz, l, z) for z in range(nzl)]
        for a in range(nzl):
            for b in range(a + 1, nzl):
                same = np.array_equal(hs[a], hs[b])
                assert same == (cls[a] == cls[b]), (shape, l, a, b)


@pytest.mark.parametrize("n", [20, 32, 48, 80])
def test_brick_levels_have_few_plane_classes(smg, n):
    nx, ny, nz = 16 * n, n, n
    for l in range(levels(nz)):
        count, cls = smg.smg_plane_classes(nx, ny, nz, l)
        assert 1 <= count <= 3, (n, l, count)
    # the finest level's planes all carry the same plane operator
    assert smg.smg_plane_classes(nx, ny, nz, 0)[0] == 1


def test_plane_classes_refuses_bad_arguments(smg):
    with pytest.raises(smg.SMGError):
        smg.smg_plane_classes(320, 20, 20, levels(20))
    with pytest.raises(smg.SMGError):
        smg.smg_plane_classes(320, 20, 20, -1)
    with pytest.raises(smg.SMGError):
        smg.smg_plane_classes(0, 20, 20, 0)
