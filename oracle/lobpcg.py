"""Plain numpy LOBPCG oracle (test infrastructure only) for the SMG-preconditioned eigensolver
of §4 of arXiv:1212.6680, which only cites LOBPCG (Knyazev 2001).  The reading: standard LOBPCG
with the block [X W P], Rayleigh-Ritz on the trial subspace, soft locking of converged columns,
convergence ||A x_i - lambda_i x_i|| <= tol lambda_i ||x_i||.

Dense steps are written out: Cholesky-QR orthonormalisation (numpy's Cholesky as the library
step), and the small symmetric eigenproblem by cyclic Jacobi rotations (Golub & Van Loan,
algorithm "cyclic Jacobi") on the Cholesky-reduced matrix.  Vectors are columns of (N, k) arrays
in the grid's (z, y, x) order.
"""
from __future__ import annotations

import numpy as np

from . import apply_A


def jacobi_eigh(S: np.ndarray, sweeps: int = 60, tol: float = 1e-15):
    """Eigenvalues (ascending) and orthonormal eigenvectors of a symmetric matrix by cyclic
    Jacobi rotations."""
    A = np.array(S, dtype=np.float64)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(sweeps):
        off = np.sqrt(np.sum(np.tril(A, -1) ** 2))
        if off <= tol * max(np.linalg.norm(A), 1e-300):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                # rotation angle that zeroes A[p, q]: tan(2 theta) = 2 apq / (aqq - app)
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + np.sqrt(1.0 + tau * tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                Ap, Aq = A[:, p].copy(), A[:, q].copy()
                A[:, p] = c * Ap - s * Aq
                A[:, q] = s * Ap + c * Aq
                Ap, Aq = A[p, :].copy(), A[q, :].copy()
                A[p, :] = c * Ap - s * Aq
                A[q, :] = s * Ap + c * Aq
                Vp, Vq = V[:, p].copy(), V[:, q].copy()
                V[:, p] = c * Vp - s * Vq
                V[:, q] = s * Vp + c * Vq
    lam = np.diag(A).copy()
    order = np.argsort(lam)
    return lam[order], V[:, order]


def cholesky_qr(Y: np.ndarray) -> np.ndarray | None:
    """Y L^{-T} with Y^T Y = L L^T; None when the Gram matrix is not numerically positive."""
    G = Y.T @ Y
    G = 0.5 * (G + G.T)
    try:
        L = np.linalg.cholesky(G)
    except np.linalg.LinAlgError:
        return None
    return np.linalg.solve(L, Y.T).T


def svqb(Y: np.ndarray, eps: float = 1e-14) -> np.ndarray:
    """Orthonormal basis of span(Y) by the eigen-decomposition of its scaled Gram matrix,
    dropping directions below eps (fallback when Cholesky-QR fails)."""
    d = np.sqrt(np.maximum(np.einsum("ij,ij->j", Y, Y), 1e-300))
    Ys = Y / d
    lam, V = jacobi_eigh(Ys.T @ Ys)
    keep = lam > eps * lam.max()
    return Ys @ (V[:, keep] / np.sqrt(lam[keep]))


def orthonormalize(Y: np.ndarray) -> np.ndarray:
    Q = cholesky_qr(Y)
    if Q is None or not np.all(np.isfinite(Q)):
        Q = svqb(Y)
    return Q


def rayleigh_ritz(S: np.ndarray, AS: np.ndarray, k: int):
    """The k smallest Ritz pairs of A on span(S): (S^T A S) c = theta (S^T S) c by Cholesky
    reduction and cyclic Jacobi.  Returns (theta, C)."""
    G = S.T @ S
    H = S.T @ AS
    G, H = 0.5 * (G + G.T), 0.5 * (H + H.T)
    L = np.linalg.cholesky(G)
    Li = np.linalg.inv(L)
    lam, V = jacobi_eigh(Li @ H @ Li.T)
    C = Li.T @ V
    return lam[:k], C[:, :k]


def lobpcg(shape, X0: np.ndarray, T=None, tol: float = 1e-8, maxit: int = 200):
    """m smallest eigenpairs of the model operator on a (nz, ny, nx) grid.

    X0: (N, m) initial block; T: an oracle.SMG (its apply is the preconditioner) or None.
    Returns dict(lam, X, iters, converged)."""
    nz, ny, nx = shape
    N = nx * ny * nz
    m = X0.shape[1]

    def A(Y):
        return np.stack([apply_A(Y[:, j].reshape(shape)).ravel() for j in range(Y.shape[1])], axis=1)

    def prec(Y):
        if T is None:
            return Y.copy()
        return np.stack([T.apply(Y[:, j].reshape(shape)).ravel() for j in range(Y.shape[1])], axis=1)

    X = orthonormalize(np.array(X0, dtype=np.float64).reshape(N, m))
    lam, C = rayleigh_ritz(X, A(X), m)
    X = X @ C
    AX = A(X)
    P = AP = None
    it = 0
    converged = np.zeros(m, dtype=bool)
    for it in range(maxit + 1):
        R = AX - X * lam
        rn = np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(X, axis=0))
        converged = rn <= tol
        if converged.all() or it == maxit:
            break
        act = ~converged  # soft locking: converged columns contribute no new directions
        W = prec(R[:, act])
        W -= X @ (X.T @ W)
        W = orthonormalize(W)
        blocks, ablocks = [X, W], [AX, A(W)]
        if P is not None:
            Pa = P[:, act] if P.shape[1] == m else P
            APa = AP[:, act] if AP.shape[1] == m else AP
            # P orthogonal to X and W, then orthonormal (A P follows by the same linear map)
            Q = np.hstack([X, W])
            coef = Q.T @ Pa
            Pa = Pa - Q @ coef
            APa = APa - np.hstack([AX, ablocks[1]]) @ coef
            G = Pa.T @ Pa
            G = 0.5 * (G + G.T)
            try:
                L = np.linalg.cholesky(G)
                Li = np.linalg.inv(L)
                blocks.append(Pa @ Li.T)
                ablocks.append(APa @ Li.T)
            except np.linalg.LinAlgError:
                pass
        S = np.hstack(blocks)
        AS = np.hstack(ablocks)
        lam, C = rayleigh_ritz(S, AS, m)
        Xn = S @ C
        AXn = AS @ C
        # the new search directions: the W and P parts of the Ritz vectors
        P = S[:, m:] @ C[m:, :]
        AP = AS[:, m:] @ C[m:, :]
        X, AX = Xn, AXn
    return {"lam": lam, "X": X, "iters": it, "converged": bool(converged.all())}
