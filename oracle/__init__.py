"""Plain FP64 CPU oracle for the SMG-preconditioned PCG / flexible PCG / PSD solvers and
LOBPCG of arXiv:1212.6680.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product library never loads it,
and it shares no code with the CUDA path.

The numerical core is ``smg_oracle.c`` (plain loops, FP64) with ``net_oracle.c`` (the learned
post-correction: 3x3x3 convolutions, their adjoints and weight gradients, the energy-norm loss);
this module compiles both with gcc into ``_liboracle.so`` next to the sources and exposes
numpy-friendly wrappers.  LOBPCG
(``lobpcg.py``) is written in numpy on top of these wrappers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smg_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "net_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

VARIANTS = {"pcg": 0, "fpcg": 1, "psd": 2}
NET_C = 16
NET_WEIGHTS = 16 * 27 + 16 * 16 * 27 + 16 * 27  # layers [16][1][27], [16][16][27], [1][16][27]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags: the same source builds on x86 and Arm)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        [os.path.getmtime(f) for f in _SRCS] + [os.path.getmtime(os.path.join(_HERE, "smg_oracle.h"))]
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
             "-o", tmp] + _SRCS + ["-lm"]
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
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_smg_num_levels.argtypes = [vp]
        L.orc_smg_level_nz.argtypes = [vp, ctypes.c_int]
        L.orc_smg_level_coefs.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp]
        L.orc_smg_plane_num_levels.argtypes = [vp]
        L.orc_smg_plane_level_ny.argtypes = [vp, ctypes.c_int]
        L.orc_smg_plane_coefs.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.orc_plane_cycle.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_krylov.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                 ctypes.c_double, ctypes.c_int, ip, dp, dp, dp, dp]
        i3 = [ctypes.c_int] * 3
        L.orc_conv3d.argtypes = i3 + [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_conv3d_adj.argtypes = i3 + [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_conv3d_wgrad.argtypes = i3 + [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_net_forward.argtypes = i3 + [dp, dp, dp]
        L.orc_net_loss_grad.argtypes = i3 + [dp, dp, dp, dp]
        L.orc_net_loss_grad.restype = ctypes.c_double
        L.orc_net_forward_ex.argtypes = i3 + [dp, dp, dp, ctypes.c_int]
        L.orc_net_loss_grad_ex.argtypes = i3 + [dp, dp, dp, dp, ctypes.c_int]
        L.orc_net_loss_grad_ex.restype = ctypes.c_double
        L.orc_round_bf16.argtypes = [ctypes.c_double]
        L.orc_round_bf16.restype = ctypes.c_double
        L.orc_learned_correct.argtypes = i3 + [dp, dp, dp]
        L.orc_smg_set_learned.argtypes = [vp, dp]
        L.orc_smg_learned_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
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

    def set_learned(self, w):
        """Attach the learned post-correction (7776 weights) or detach it (None)."""
        if w is None:
            lib().orc_smg_set_learned(self._h, None)
        else:
            w = _f64(w).ravel()
            assert w.size == NET_WEIGHTS
            lib().orc_smg_set_learned(self._h, _p(w))

    def learned_stats(self):
        c, a = ctypes.c_longlong(), ctypes.c_longlong()
        lib().orc_smg_learned_stats(self._h, ctypes.byref(c), ctypes.byref(a))
        return c.value, a.value

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


# ---- learned post-correction (net_oracle.c) ------------------------------------------------------

def split_weights(w):
    """The flat 7776-weight array as its three layers, shapes (16,1,27), (16,16,27), (1,16,27)."""
    w = np.asarray(w).ravel()
    a, b = NET_C * 27, NET_C * 27 + NET_C * NET_C * 27
    return w[:a].reshape(NET_C, 1, 27), w[a:b].reshape(NET_C, NET_C, 27), w[b:].reshape(1, NET_C, 27)


def conv3d(w: np.ndarray, x: np.ndarray) -> np.ndarray:
    """w: (cout, cin, 27); x: (cin, nz, ny, nx) -> (cout, nz, ny, nx)."""
    w, x = _f64(w), _f64(x)
    cout, cin = w.shape[:2]
    _, nz, ny, nx = x.shape
    out = np.empty((cout, nz, ny, nx))
    lib().orc_conv3d(nx, ny, nz, cin, cout, _p(w), _p(x), _p(out))
    return out


def conv3d_adj(w: np.ndarray, g: np.ndarray) -> np.ndarray:
    w, g = _f64(w), _f64(g)
    cout, cin = w.shape[:2]
    _, nz, ny, nx = g.shape
    out = np.empty((cin, nz, ny, nx))
    lib().orc_conv3d_adj(nx, ny, nz, cin, cout, _p(w), _p(g), _p(out))
    return out


def conv3d_wgrad(x: np.ndarray, g: np.ndarray) -> np.ndarray:
    x, g = _f64(x), _f64(g)
    cin, nz, ny, nx = x.shape
    cout = g.shape[0]
    out = np.empty((cout, cin, 27))
    lib().orc_conv3d_wgrad(nx, ny, nz, cin, cout, _p(x), _p(g), _p(out))
    return out


def net_forward(w, rho: np.ndarray, act_bf16: bool = False) -> np.ndarray:
    """delta = rms(rho) Net(rho / rms(rho)) for a (nz, ny, nx) residual (hidden activations
    rounded to BF16 when act_bf16)."""
    w, rho = _f64(w).ravel(), _f64(rho)
    nz, ny, nx = rho.shape
    out = np.empty_like(rho)
    lib().orc_net_forward_ex(nx, ny, nz, _p(w), _p(rho), _p(out), int(act_bf16))
    return out


def net_loss_grad(w, rho: np.ndarray, e: np.ndarray, want_grad=True, act_bf16: bool = False):
    """(loss, gradient (7776,) or None) of L = (e - delta)^T A (e - delta) / e^T A e."""
    w, rho, e = _f64(w).ravel(), _f64(rho), _f64(e)
    nz, ny, nx = rho.shape
    g = np.empty(NET_WEIGHTS) if want_grad else None
    loss = lib().orc_net_loss_grad_ex(nx, ny, nz, _p(w), _p(rho), _p(e), _p(g) if want_grad else None,
                                      int(act_bf16))
    return loss, g


def round_bf16(v: float) -> float:
    return lib().orc_round_bf16(float(v))


def learned_correct(w, r: np.ndarray, s0: np.ndarray):
    """(s, accepted): s0 + delta(r - A s0) if the judge accepts it, else s0."""
    w, r = _f64(w).ravel(), _f64(r)
    s = _f64(s0).copy()
    nz, ny, nx = r.shape
    acc = lib().orc_learned_correct(nx, ny, nz, _p(w), _p(r), _p(s))
    return s, bool(acc)


def set_threads(n: int) -> int:
    """Threads the C oracle's loops may use (1 = sequential); results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))
