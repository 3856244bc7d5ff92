"""Pins of the LOBPCG oracle (oracle/lobpcg.py): its cyclic Jacobi against numpy's symmetric
eigensolver, its eigenpairs against a dense eigensolver on a small grid and against the
closed-form Dirichlet eigenvalues, orthonormality of X, and the SMG preconditioner reducing the
iteration count (the purpose of §4)."""
import numpy as np
import pytest

from paper_1212_6680_gb300 import inputs
from tests import dense_ref as D


@pytest.fixture(scope="module")
def lob(orc):
    from oracle import lobpcg

    return lobpcg


def closed_form(nx, ny, nz, m):
    lam = []
    for kx in range(1, nx + 1):
        for ky in range(1, ny + 1):
            for kz in range(1, nz + 1):
                lam.append(sum(4 * np.sin(np.pi * k / (2 * (n + 1))) ** 2 for k, n in ((kx, nx), (ky, ny), (kz, nz))))
    return np.sort(lam)[:m]


@pytest.mark.parametrize("n,seed", [(5, 1), (12, 2), (30, 3)])
def test_jacobi_matches_numpy_eigh(lob, n, seed):
    B = np.random.default_rng(seed).standard_normal((n, n))
    S = B + B.T
    lam, V = lob.jacobi_eigh(S)
    assert np.allclose(lam, np.linalg.eigvalsh(S), rtol=0, atol=1e-12 * np.abs(S).max())
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
    assert np.allclose(S @ V, V * lam, atol=1e-11 * np.abs(S).max())


@pytest.mark.parametrize("npost", [1, 0])
def test_lobpcg_equals_dense_eigh_on_small_grid(orc, lob, npost):
    nx, ny, nz, m = 6, 5, 4, 4
    A = D.laplacian3d(nx, ny, nz)
    ref = np.linalg.eigvalsh(A)[:m]
    X0 = inputs.initial_block(nx, ny, nz, m, seed=7).T
    out = lob.lobpcg((nz, ny, nx), X0, orc.SMG(nx, ny, nz, 1, npost), tol=1e-9, maxit=100)
    assert out["converged"]
    assert np.allclose(out["lam"], ref, rtol=1e-10, atol=0)
    X = out["X"]
    assert np.abs(X.T @ X - np.eye(m)).max() <= 1e-10


def test_lobpcg_matches_closed_form_and_preconditioner_helps(orc, lob):
    nx = ny = nz = 12
    m = 6
    X0 = inputs.initial_block(nx, ny, nz, m, seed=7).T
    ref = closed_form(nx, ny, nz, m)
    pre = lob.lobpcg((nz, ny, nx), X0, orc.SMG(nx, ny, nz, 1, 0), tol=1e-8, maxit=200)
    assert pre["converged"]
    assert np.all(np.abs(pre["lam"] - ref) <= 1e-10 * ref)
    plain = lob.lobpcg((nz, ny, nx), X0, None, tol=1e-8, maxit=200)
    assert pre["iters"] < plain["iters"]
