"""smg_gram: FP64-accurate Gram products on the tensor cores (BF16 digit splitting, exact FP32
sums per 64 rows) against the exactly rounded products of the same FP64 inputs (Dekker's
error-free products summed by math.fsum), element by element: |G_ij - u_i.v_j| <= 1e-14
||u_i|| ||v_j||.  Shapes span several 64-row stages and CTAs, ragged tails, k up to 64, a
symmetric product (V = U), a zero column and columns of very different magnitudes."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    assert torch.cuda.is_available()
    return m


def _split(a):
    c = 134217729.0 * a
    hi = c - (c - a)
    return hi, a - hi


def exact_gram(U, V):
    """Correctly rounded u_i . v_j: every product as an exact (p, e) pair, summed by fsum."""
    k1, k2 = U.shape[1], V.shape[1]
    G = np.empty((k1, k2))
    Vh, Vl = _split(V)
    for i in range(k1):
        a = U[:, i:i + 1]
        ah, al = _split(a)
        P = a * V
        E = ((ah * Vh - P) + ah * Vl + al * Vh) + al * Vl
        for j in range(k2):
            G[i, j] = math.fsum(np.concatenate([P[:, j], E[:, j]]))
    return G


def run(smg, U, V, sym=False):
    n, k1 = U.shape
    k2 = V.shape[1]
    Ud = torch.from_numpy(np.asfortranarray(U).T.copy()).cuda()  # column j contiguous
    Vd = Ud if sym else torch.from_numpy(np.asfortranarray(V).T.copy()).cuda()
    G = torch.empty(k1 * k2, dtype=torch.float64, device="cuda")
    smg.smg_gram(n, k1, Ud, k2, Vd, G)
    return G.cpu().numpy().reshape(k1, k2)


@pytest.mark.parametrize("n,k1,k2,sym", [(20000, 48, 48, False), (20000, 48, 48, True), (70001, 16, 33, False),
                                         (3000, 64, 64, False), (65, 5, 7, False), (1, 3, 2, False),
                                         (131072 + 17, 24, 40, False)])
def test_gram_matches_exact_products(smg, n, k1, k2, sym):
    rng = np.random.default_rng(n + 7 * k1 + k2)
    U = rng.standard_normal((n, k1)) / math.sqrt(n)
    V = U if sym else rng.standard_normal((n, k2)) * rng.uniform(0.1, 10.0, k2)
    got = run(smg, U, V, sym)
    ref = exact_gram(U, V)
    scale = np.outer(np.linalg.norm(U, axis=0), np.linalg.norm(V, axis=0))
    err = np.abs(got - ref) / scale
    assert err.max() <= 1e-14, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_gram_zero_column_and_wide_magnitudes(smg):
    rng = np.random.default_rng(5)
    n = 9000
    U = rng.standard_normal((n, 6))
    U[:, 1] = 0.0
    U[:, 2] *= 1e-200
    U[:, 3] *= 1e100
    U[::7, 4] = 0.0
    U[:, 5] = np.sin(np.arange(n) * 0.01)  # smooth, like an eigenvector
    V = rng.standard_normal((n, 4)) * np.array([1.0, 1e-150, 1e150, 3.0])
    got = run(smg, U, V)
    ref = exact_gram(U, V)
    scale = np.outer(np.linalg.norm(U, axis=0), np.linalg.norm(V, axis=0))
    assert np.all(got[1] == 0.0)
    ok = scale > 0
    assert np.all(np.abs(got - ref)[ok] <= 1e-14 * scale[ok])


def test_gram_rejects_bad_shapes(smg):
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(smg.SMGError):
        smg.smg_gram(8, 65, x, 1, x, x)
    with pytest.raises(smg.SMGError):
        smg.smg_gram(0, 1, x, 1, x, x)
