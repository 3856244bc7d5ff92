"""Plain FP64 CPU oracle for the SMG-preconditioned PCG / flexible PCG / PSD solvers and
LOBPCG of arXiv:1212.6680.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product library never loads it,
and it shares no code with the CUDA path.

The numerical core is ``smg_oracle.c`` (plain loops, FP64); this module compiles it with gcc
into ``_liboracle.so`` next to the sources and exposes numpy-friendly wrappers.  LOBPCG
(``lobpcg.py``) is written in numpy on top of these wrappers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

VARIANTS = {"pcg": 0, "fpcg": 1, "psd": 2}


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags: the same source builds on x86 and Arm)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "smg_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
             "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        vp = ctypes.c_void_p
        L.orc_apply_A.argtypes = [ctypes.c_int] * 3 + [dp, dp]
        L.orc_thomas.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
        L.orc_smg_setup.argtypes = [ctypes.c_int] * 6
        L.orc_smg_setup.restype = vp
        L.orc_smg_free.argtypes = [vp]
        L.orc_smg_apply.argtypes = [vp, dp, dp]
        L.orc_smg_num_levels.argtypes = [vp]
        L.orc_smg_level_nz.argtypes = [vp, ctypes.c_int]
        L.orc_smg_level_coefs.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp]
        L.orc_smg_plane_num_levels.argtypes = [vp]
        L.orc_smg_plane_level_ny.argtypes = [vp, ctypes.c_int]
        L.orc_smg_plane_coefs.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.orc_plane_cycle.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_krylov.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                 ctypes.c_double, ctypes.c_int, ip, dp, dp, dp, dp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def apply_A(u: np.ndarray) -> np.ndarray:
    """7-point negative Laplacian of a (nz, ny, nx) array, homogeneous Dirichlet."""
    u = _f64(u)
    nz, ny, nx = u.shape
    out = np.empty_like(u)
    lib().orc_apply_A(nx, ny, nz, _p(u), _p(out))
    return out


def thomas(a, b, c, d):
    a, b, c, d = map(_f64, (a, b, c, d))
    x = np.empty_like(d)
    lib().orc_thomas(len(d), _p(a), _p(b), _p(c), _p(d), _p(x))
    return x


def plane_cycle(c: float, d: float, g: np.ndarray) -> np.ndarray:
    g = _f64(g)
    ny, nx = g.shape
    v = np.empty_like(g)
    lib().orc_plane_cycle(nx, ny, c, d, _p(g), _p(v))
    return v


class SMG:
    """The SMG preconditioner T of one nx x ny x nz brick (arrays are (nz, ny, nx))."""

    def __init__(self, nx, ny, nz, npre=1, npost=1, coarse_iters=1):
        self.shape = (nz, ny, nx)
        self.npre, self.npost = npre, npost
        self._h = lib().orc_smg_setup(nx, ny, nz, npre, npost, coarse_iters)
        if not self._h:
            raise ValueError("orc_smg_setup rejected its arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_smg_free(h)
            self._h = None

    def apply(self, r: np.ndarray) -> np.ndarray:
        r = _f64(r).reshape(self.shape)
        s = np.empty_like(r)
        lib().orc_smg_apply(self._h, _p(r), _p(s))
        return s

    def num_levels(self):
        return lib().orc_smg_num_levels(self._h)

    def level_nz(self, l):
        return lib().orc_smg_level_nz(self._h, l)

    def level_coefs(self, l):
        n = self.level_nz(l)
        M, K = np.zeros((n, 3)), np.zeros((n, 3))
        wm, wp = np.zeros(n), np.zeros(n)
        lib().orc_smg_level_coefs(self._h, l, _p(M), _p(K), _p(wm), _p(wp))
        return M, K, wm, wp

    def plane_num_levels(self):
        return lib().orc_smg_plane_num_levels(self._h)

    def plane_level_ny(self, m):
        return lib().orc_smg_plane_level_ny(self._h, m)

    def plane_coefs(self, l, z, m):
        n = self.plane_level_ny(m)
        S, T = np.zeros((n, 3)), np.zeros((n, 3))
        wm, wp = np.zeros(n), np.zeros(n)
        lib().orc_smg_plane_coefs(self._h, l, z, m, _p(S), _p(T), _p(wm), _p(wp))
        return S, T, wm, wp


def krylov(b: np.ndarray, variant: str, smg: SMG | None = None, tol=1e-8, maxit=100,
           x0: np.ndarray | None = None, keep_vectors=False):
    """Algorithm 1 (PCG eq. (1), flexible PCG eq. (2), or PSD); smg=None means T = I.

    Returns dict(x, status, iters, relres, hist[, xs, rs])."""
    b = _f64(b)
    nz, ny, nx = b.shape
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    hist = np.full(maxit + 1, np.nan)
    n = b.size
    xs = np.zeros((maxit + 1, n)) if keep_vectors else None
    rs = np.zeros((maxit + 1, n)) if keep_vectors else None
    null = ctypes.POINTER(ctypes.c_double)()
    st = lib().orc_krylov(smg._h if smg is not None else None, nx, ny, nz, VARIANTS[variant],
                          _p(b), _p(x), tol, maxit, ctypes.byref(it), ctypes.byref(rr), _p(hist),
                          _p(xs) if keep_vectors else null, _p(rs) if keep_vectors else null)
    out = dict(x=x, status=st, iters=it.value, relres=rr.value, hist=hist[: it.value + 1])
    if keep_vectors:
        out["xs"] = xs[: it.value + 1].reshape(-1, nz, ny, nx)
        out["rs"] = rs[: it.value + 1].reshape(-1, nz, ny, nx)
    return out
