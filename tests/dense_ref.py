"""Dense-matrix restatement of the model problem and of the SMG cycle, for tiny grids.

Test-only brute force used to pin the C oracle.  It is written in a different form from the
oracle: every operator is an explicit dense matrix built from Kronecker products, the
interpolation weights are read off the dense operator's rows (the stencil collapsed
in-plane at an interior row), Galerkin products are dense matmuls, and a V-cycle is the
linear map T = (I - E) A^{-1} assembled from its error-propagation matrix E.
"""
from __future__ import annotations

import numpy as np


def lap1d(n: int) -> np.ndarray:
    return 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def laplacian3d(nx: int, ny: int, nz: int) -> np.ndarray:
    """7-point negative Laplacian, index (z*ny + y)*nx + x, as a sum of Kronecker products."""
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    return (np.kron(np.kron(Iz, Iy), lap1d(nx)) + np.kron(np.kron(Iz, lap1d(ny)), Ix)
            + np.kron(np.kron(lap1d(nz), Iy), Ix))


def collapse_weights_from_dense(Xc: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Interpolation weights of fine (even) points from a 1D coupling matrix Xc."""
    n = Xc.shape[0]
    wm, wp = np.zeros(n), np.zeros(n)
    for i in range(0, n, 2):
        if i - 1 >= 0:
            wm[i] = -Xc[i, i - 1] / Xc[i, i]
        if i + 1 < n:
            wp[i] = -Xc[i, i + 1] / Xc[i, i]
    return wm, wp


def prolongation_1d(n: int, wm: np.ndarray, wp: np.ndarray) -> np.ndarray:
    """n x n//2 interpolation: odd fine points injected, even ones weighted from neighbours."""
    nc = n // 2
    P = np.zeros((n, nc))
    for i in range(n):
        if i % 2 == 1:
            P[i, (i - 1) // 2] = 1.0
        else:
            if i - 1 >= 0:
                P[i, i // 2 - 1] = wm[i]
            if i + 1 < n and i // 2 < nc:
                P[i, i // 2] = wp[i]
    return P


def collapsed_z_coupling(A: np.ndarray, nx: int, ny: int, nz: int) -> np.ndarray:
    """nz x nz matrix of plane-to-plane couplings summed over the full interior 5-point stencil.

    Reads the row of an interior (x, y) point (needs nx, ny >= 3) in every plane and sums its
    entries in each neighbouring plane: the in-plane collapse of the stencil."""
    assert nx >= 3 and ny >= 3
    x0, y0 = nx // 2, ny // 2
    K = np.zeros((nz, nz))
    np_ = nx * ny
    for z in range(nz):
        row = A[z * np_ + y0 * nx + x0]
        for zz in range(max(0, z - 1), min(nz, z + 2)):
            blk = row[zz * np_:(zz + 1) * np_].reshape(ny, nx)
            K[z, zz] = blk[y0 - 1:y0 + 2, x0 - 1:x0 + 2].sum()
    return K


def collapsed_y_coupling(B: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """ny x ny matrix of line-to-line couplings of a 2D operator summed over an interior row."""
    assert nx >= 3
    x0 = nx // 2
    T = np.zeros((ny, ny))
    for y in range(ny):
        row = B[y * nx + x0]
        for yy in range(max(0, y - 1), min(ny, y + 2)):
            T[y, yy] = row[yy * nx + x0 - 1: yy * nx + x0 + 2].sum()
    return T


def block_relax_error(A: np.ndarray, blocks: list[np.ndarray], solves: list[np.ndarray]) -> np.ndarray:
    """Error propagation of one sweep of block relaxation u += E_b C_b E_b^T (f - A u), in order."""
    n = A.shape[0]
    E = np.eye(n)
    for idx, C in zip(blocks, solves):
        Eb = np.zeros((n, len(idx)))
        Eb[idx, np.arange(len(idx))] = 1.0
        E = (np.eye(n) - Eb @ C @ Eb.T @ A) @ E
    return E


def plane_cycle_matrix(B: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """The 2D cycle C ~ B^{-1}: y-semicoarsening, exact x-line solves, (1,1) line relaxation."""
    if ny == 1:
        return np.linalg.inv(B)
    if nx >= 3:
        Ty = collapsed_y_coupling(B, nx, ny)
    else:  # too narrow for an interior row: collapse the interior stencil analytically
        raise ValueError("plane too narrow for the dense collapse")
    wm, wp = collapse_weights_from_dense(Ty)
    P = np.kron(prolongation_1d(ny, wm, wp), np.eye(nx))
    Bc = P.T @ B @ P
    Cc = plane_cycle_matrix(Bc, nx, ny // 2)
    lines = [np.arange(y * nx, (y + 1) * nx) for y in range(ny)]
    even = [lines[y] for y in range(0, ny, 2)]
    odd = [lines[y] for y in range(1, ny, 2)]
    inv = lambda idx: np.linalg.inv(B[np.ix_(idx, idx)])
    pre = block_relax_error(B, even + odd, [inv(i) for i in even + odd])
    post = block_relax_error(B, odd + even, [inv(i) for i in odd + even])
    cgc = np.eye(B.shape[0]) - P @ Cc @ P.T @ B
    E = post @ cgc @ pre
    return (np.eye(B.shape[0]) - E) @ np.linalg.inv(B)


def smg_matrix(A: np.ndarray, nx: int, ny: int, nz: int, npre: int, npost: int,
               coarse_iters: int = 1) -> np.ndarray:
    """The 3D SMG cycle T ~ A^{-1} as a dense matrix (z-semicoarsening, plane relaxation)."""
    np_ = nx * ny
    planes = [np.arange(z * np_, (z + 1) * np_) for z in range(nz)]
    Cz = [plane_cycle_matrix(A[np.ix_(p, p)], nx, ny) for p in planes]
    if nz == 1:
        E = np.linalg.matrix_power(np.eye(np_) - Cz[0] @ A, coarse_iters)
        return (np.eye(np_) - E) @ np.linalg.inv(A)
    Kz = collapsed_z_coupling(A, nx, ny, nz)
    wm, wp = collapse_weights_from_dense(Kz)
    P = np.kron(prolongation_1d(nz, wm, wp), np.eye(np_))
    Ac = P.T @ A @ P
    Tc = smg_matrix(Ac, nx, ny, nz // 2, npre, npost, coarse_iters)
    red = list(range(0, nz, 2))
    black = list(range(1, nz, 2))
    pre_one = block_relax_error(A, [planes[z] for z in red + black], [Cz[z] for z in red + black])
    post_one = block_relax_error(A, [planes[z] for z in black + red], [Cz[z] for z in black + red])
    pre = np.linalg.matrix_power(pre_one, npre)
    post = np.linalg.matrix_power(post_one, npost)
    cgc = np.eye(A.shape[0]) - P @ Tc @ P.T @ A
    E = post @ cgc @ pre
    return (np.eye(A.shape[0]) - E) @ np.linalg.inv(A)


def assemble_columns(apply, n: int, shape) -> np.ndarray:
    """Dense matrix of a linear map given as a function on arrays of `shape`, column by column."""
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = np.asarray(apply(e.reshape(shape))).ravel()
    return M


def lap7(u: np.ndarray) -> np.ndarray:
    """7-point Dirichlet Laplacian of a (nz, ny, nx) array by numpy slicing (an independent
    restatement of the model operator for residual checks)."""
    out = 6.0 * u
    out[1:] -= u[:-1]
    out[:-1] -= u[1:]
    out[:, 1:] -= u[:, :-1]
    out[:, :-1] -= u[:, 1:]
    out[:, :, 1:] -= u[:, :, :-1]
    out[:, :, :-1] -= u[:, :, 1:]
    return out
