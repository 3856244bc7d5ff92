"""Comparison helpers of the GPU parity tests.

Every comparison checks two things: the norm-wise relative error ||a - b||_2 / ||b||_2, and the
element-wise one, max_i |a_i - b_i| / max_i |b_i| -- the second is what catches a single wrong
element or a wrong plane that a norm over millions of points would hide.  For grid vectors of
the reduced-precision cycles the element-wise check is made plane by plane (each z-plane against
its own largest value), so that a wrong plane cannot hide behind the others' scale.
"""
from __future__ import annotations

import numpy as np


def rel(a, b) -> float:
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b) -> float:
    a, b = np.ravel(a), np.ravel(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if b.size else 0.0


def plane_maxrel(a, b, shape) -> float:
    """Largest over z-planes of max|a_z - b_z| / max|b_z| (shape = (nx, ny, nz) or (nz, ny, nx)
    given as the grid's (nx, ny, nz))."""
    nx, ny, nz = shape
    a = np.reshape(a, (nz, ny * nx))
    b = np.reshape(b, (nz, ny * nx))
    den = np.maximum(np.max(np.abs(b), axis=1), 1e-300)
    return float(np.max(np.max(np.abs(a - b), axis=1) / den))


def assert_close(got, ref, tol: float, shape=None, what: str = "", elem_tol: float | None = None) -> None:
    """Norm-wise and element-wise (plane-wise when `shape` is given) relative errors <= tol
    (element-wise against elem_tol when it is given)."""
    et = tol if elem_tol is None else elem_tol
    r = rel(got, ref)
    assert r <= tol, f"{what}: norm-wise relative error {r:.3e} > {tol:.1e}"
    m = maxrel(got, ref)
    assert m <= et, f"{what}: element-wise relative error {m:.3e} > {et:.1e}"
    if shape is not None:
        p = plane_maxrel(got, ref, shape)
        assert p <= et, f"{what}: plane-wise relative error {p:.3e} > {et:.1e}"
