"""Thin ctypes binding of libsmg's C ABI (include/smg.h), with the same names.

Argument marshalling only: every step of the method runs in libsmg's CUDA kernels.  Vectors
are passed as raw pointers: a torch CUDA tensor (its data_ptr), a numpy array (host memory,
accepted where the C ABI accepts host pointers), or an int address.  Streams are torch
streams or raw cudaStream_t handles.  Importing this module loads libsmg.so and fails loudly
when it is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmg.so")

SMG_OK, SMG_ERR_ARG, SMG_ERR_CUDA, SMG_ERR_NOCONV, SMG_ERR_BREAKDOWN, SMG_ERR_TIMEOUT, SMG_ERR_NAN = 0, -1, -2, -3, -4, -5, -6
SMG_ERR_HOST = -7
SMG_PCG, SMG_FPCG, SMG_PSD = 0, 1, 2
SMG_FP64, SMG_FP32, SMG_BF16 = 0, 1, 2
SMG_OPT_COARSE_ITERS, SMG_OPT_THREADS, SMG_OPT_PROFILE, SMG_OPT_CLUSTER_MAX, SMG_OPT_CLUSTER_MAX32 = 0, 1, 2, 3, 4
SMG_OPT_PRECOND = 5
SMG_OPT_LEAN = 6
SMG_OPT_GRAM_TC = 7
SMG_OPT_GRAPH = 8
SMG_OPT_FUSED_TAIL = 9
SMG_OPT_SOLO = 10
SMG_OPT_RESTRICT_COLUMN = 11
SMG_OPT_WIDE_FACTORS = 12
SMG_OPT_WIDE_MIN_ROWS = 13

VARIANTS = {"pcg": SMG_PCG, "fpcg": SMG_FPCG, "psd": SMG_PSD}
PRECISIONS = {"fp64": SMG_FP64, "fp32": SMG_FP32, "bf16": SMG_BF16}

# every symbol include/smg.h declares
EXPORTS = ("smg_setup", "smg_set_precision", "smg_set_option", "smg_apply", "smg_apply_batched",
           "smg_apply_A", "krylov_solve", "lobpcg_solve", "smg_destroy", "smg_last_error",
           "smg_profile_read", "smg_launch_count", "smg_check_conversions", "smg_apply_A_dot_static",
           "krylov_solve_batched", "smg_barrier_selftest", "smg_batched_setup", "smg_batched_solve",
           "smg_batched_destroy", "smg_batched_apply", "smg_batched_info", "smg_batched_set_profile", "smg_batched_profile_read",
           "smg_set_learned", "smg_learned_stats", "smg_collect_pairs", "smg_net_forward", "smg_net_loss_grad",
           "smg_net_train", "smg_net_set_tensor_cores", "smg_net_tc_status", "smg_setup_coefs",
           "smg_plane_layout", "smg_plane_layout_kind", "smg_gram", "smg_krylov_history", "smg_plane_classes")
NET_WEIGHTS = 7776


class SMGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libsmg error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsmg.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double
    L.smg_setup.argtypes = [i, i, i, i, i, ctypes.POINTER(vp)]
    L.smg_set_precision.argtypes = [vp, i]
    L.smg_set_option.argtypes = [vp, i, i]
    L.smg_apply.argtypes = [vp, vp, vp, vp]
    L.smg_apply_batched.argtypes = [vp, i, vp, vp, vp]
    L.smg_apply_A.argtypes = [vp, vp, vp, vp]
    L.krylov_solve.argtypes = [vp, i, vp, vp, d, i, ip, dp, vp]
    L.lobpcg_solve.argtypes = [vp, i, vp, dp, d, i, ip, vp]
    L.smg_destroy.argtypes = [vp]
    L.smg_setup_coefs.argtypes = [i, i, i, i, i, i, dp, dp, ip, ip]
    L.smg_plane_classes.argtypes = [i, i, i, i, ip]
    L.smg_plane_layout.argtypes = [i, i, i, i, ctypes.POINTER(ctypes.c_longlong)]
    L.smg_plane_layout_kind.argtypes = [i, i, i, i, i, i, ctypes.POINTER(ctypes.c_longlong)]
    L.smg_last_error.restype = ctypes.c_char_p
    L.smg_profile_read.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong), dp, dp]
    L.smg_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.smg_check_conversions.argtypes = [ctypes.c_longlong, vp, vp, vp]
    L.smg_apply_A_dot_static.argtypes = [i, i, i, vp, vp, vp, vp]
    L.krylov_solve_batched.argtypes = [i, vp, i, i, i, vp, vp, d, i, vp, vp]
    L.smg_barrier_selftest.argtypes = [i, d, ip, vp]
    ll = ctypes.POINTER(ctypes.c_longlong)
    L.smg_batched_setup.argtypes = [i, vp, i, i, i, ctypes.POINTER(vp), vp]
    L.smg_batched_solve.argtypes = [vp, i, vp, vp, d, i, vp, vp, vp]
    L.smg_batched_destroy.argtypes = [vp]
    L.smg_batched_apply.argtypes = [vp, vp, vp, vp]
    L.smg_batched_info.argtypes = [vp, ip, ip, ip, ll, ll, ip]
    L.smg_batched_set_profile.argtypes = [vp, i]
    L.smg_batched_profile_read.argtypes = [vp, i, ll, dp, dp]
    L.smg_set_learned.argtypes = [vp, vp, i]
    L.smg_learned_stats.argtypes = [vp, ll, ll]
    L.smg_collect_pairs.argtypes = [vp, vp, vp, d, i, vp, vp, i, ip, vp]
    L.smg_net_forward.argtypes = [i, i, i, i, vp, vp, vp, vp]
    L.smg_net_loss_grad.argtypes = [i, i, i, i, vp, vp, vp, dp, vp, vp]
    L.smg_net_train.argtypes = [i, vp, vp, vp, i, d, ctypes.c_ulonglong, i, vp, vp, vp]
    L.smg_net_set_tensor_cores.argtypes = [i]
    L.smg_net_tc_status.argtypes = [ip]
    L.smg_gram.argtypes = [ctypes.c_longlong, i, vp, i, vp, vp, vp]
    L.smg_krylov_history.argtypes = [vp, dp, i, ip]
    for name in EXPORTS:
        getattr(L, name).restype = getattr(L, name).restype if name == "smg_last_error" else ctypes.c_int
    return L


_lib = _load()


def lib():
    return _lib


def smg_last_error() -> str:
    return _lib.smg_last_error().decode()


def _check(rc: int, allow=()):
    if rc != SMG_OK and rc not in allow:
        raise SMGError(rc, smg_last_error())
    return rc


def _ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _stream(s) -> int:
    if s is None:
        try:
            import torch

            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return 0
    if isinstance(s, int):
        return s
    return s.cuda_stream


def smg_setup(nx: int, ny: int, nz: int, npre: int = 1, npost: int = 1) -> int:
    h = ctypes.c_void_p()
    _check(_lib.smg_setup(nx, ny, nz, npre, npost, ctypes.byref(h)))
    return h.value


def smg_set_precision(h: int, prec) -> None:
    _check(_lib.smg_set_precision(h, PRECISIONS.get(prec, prec)))


def smg_set_option(h: int, option: int, value: int) -> None:
    _check(_lib.smg_set_option(h, option, value))


def smg_apply(h: int, r, s, stream=None) -> None:
    _check(_lib.smg_apply(h, _ptr(r), _ptr(s), _stream(stream)))


def smg_apply_batched(h: int, nb: int, R, S, stream=None) -> None:
    _check(_lib.smg_apply_batched(h, nb, _ptr(R), _ptr(S), _stream(stream)))


def smg_apply_A(h: int, u, out, stream=None) -> None:
    _check(_lib.smg_apply_A(h, _ptr(u), _ptr(out), _stream(stream)))


def krylov_solve(h: int, variant, b, x, tol: float = 1e-8, maxit: int = 100, stream=None, check=True):
    """Returns (status, iters, relres); raises on errors other than SMG_ERR_NOCONV when check."""
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = _lib.krylov_solve(h, VARIANTS.get(variant, variant), _ptr(b), _ptr(x), tol, maxit, ctypes.byref(it),
                           ctypes.byref(rr), _stream(stream))
    if check:
        _check(rc, allow=(SMG_ERR_NOCONV,))
    return rc, it.value, rr.value


def lobpcg_solve(h: int, m: int, X, tol: float = 1e-8, maxit: int = 100, stream=None, check=True):
    """Returns (status, iters, lambdas as a numpy array)."""
    lam = np.zeros(m)
    it = ctypes.c_int(0)
    rc = _lib.lobpcg_solve(h, m, _ptr(X), lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), tol, maxit,
                           ctypes.byref(it), _stream(stream))
    if check:
        _check(rc, allow=(SMG_ERR_NOCONV,))
    return rc, it.value, lam


def smg_profile_read(h: int, which: int):
    n = ctypes.c_longlong(0)
    ms = ctypes.c_double(0.0)
    by = ctypes.c_double(0.0)
    _check(_lib.smg_profile_read(h, which, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
    return n.value, ms.value, by.value


def smg_launch_count(h: int) -> int:
    n = ctypes.c_longlong(0)
    _check(_lib.smg_launch_count(h, ctypes.byref(n)))
    return n.value


def smg_check_conversions(src, mismatches, stream=None) -> None:
    """src: device doubles; mismatches: device int32[2]."""
    _check(_lib.smg_check_conversions(src.numel(), _ptr(src), _ptr(mismatches), _stream(stream)))


def smg_setup_coefs(nx: int, ny: int, nz: int, l: int, z: int, m: int):
    """Host-side set-up coefficients of z-level l, plane z, 2D level m: (zc (8,), lines (ny_m, 8))."""
    zc = np.zeros(8)
    lines = np.zeros((ny, 8))
    nzl, nym = ctypes.c_int(0), ctypes.c_int(0)
    dp_ = ctypes.POINTER(ctypes.c_double)
    _check(_lib.smg_setup_coefs(nx, ny, nz, l, z, m, zc.ctypes.data_as(dp_), lines.ctypes.data_as(dp_),
                                ctypes.byref(nzl), ctypes.byref(nym)))
    return zc, lines[: nym.value].copy()


def smg_plane_classes(nx: int, ny: int, nz: int, l: int):
    """Classes of the planes of z-level l with equal 2D hierarchies (host only): (count, cls)."""
    cls = np.full(max(nz, 1), -1, dtype=np.int32)  # level l holds at most nz planes
    rc = _lib.smg_plane_classes(nx, ny, nz, l, cls.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    _check(min(rc, 0))
    nzl = nz
    for _ in range(l):
        nzl //= 2
    return rc, cls[:nzl].copy()


def smg_plane_layout(nx: int, ny: int, elem_bytes: int, R: int = 1) -> dict:
    """The planned shared-memory / global layout of one plane's 2D-cycle arrays (host only)."""
    out = (ctypes.c_longlong * 64)()
    _check(_lib.smg_plane_layout(nx, ny, elem_bytes, R, out))
    v = list(out)
    P = v[0]
    return {"P": P, "K": v[1], "MF": v[2], "smem_bytes": v[3], "ws_elems": v[4], "off_fs": v[5],
            "u_mask": v[6], "g_mask": v[7], "sum_ny": v[8], "coef_per_line": v[9], "set_elems": v[10],
            "off_u": v[16:16 + P], "off_g": v[32:32 + P], "ny_m": v[48:48 + P]}


def smg_plane_layout_kind(nx: int, ny: int, elem_bytes: int, R: int, kind: int, solo: int = 8) -> dict:
    """The layout of one plane-cycle kernel (0 general, 1 shortened-step, 2 wide lines), host only."""
    out = (ctypes.c_longlong * 64)()
    _check(_lib.smg_plane_layout_kind(nx, ny, elem_bytes, R, kind, solo, out))
    v = list(out)
    P = v[0]
    return {"P": P, "K": v[1], "MF": v[2], "smem_bytes": v[3], "ws_elems": v[4], "off_fs": v[5],
            "u_mask": v[6], "g_mask": v[7], "sum_ny": v[8], "coef_per_line": v[9], "set_elems": v[10],
            "solo_from": v[11], "off_u": v[16:16 + P], "off_g": v[32:32 + P], "ny_m": v[48:48 + P]}


def smg_apply_A_dot_static(nx: int, ny: int, nz: int, u, out, dot, stream=None) -> None:
    """out = A u and dot[0] = (u, A u) with no device allocation (static scratch)."""
    _check(_lib.smg_apply_A_dot_static(nx, ny, nz, _ptr(u), _ptr(out), _ptr(dot), _stream(stream)))


def krylov_solve_batched(dims, b_list, x_list, npre=1, npost=0, prec="fp32", tol=1e-8, maxit=100, stream=None,
                         check=True):
    """dims: (nsys, 3) ints (nx, ny, nz); b_list, x_list: per-system device tensors.
    Returns (status, iters as a numpy array)."""
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
    nsys = dims.shape[0]
    bp = (ctypes.c_void_p * nsys)(*[_ptr(t) for t in b_list])
    xp = (ctypes.c_void_p * nsys)(*[_ptr(t) for t in x_list])
    it = np.zeros(nsys, dtype=np.int32)
    rc = _lib.krylov_solve_batched(nsys, dims.ctypes.data, npre, npost, PRECISIONS.get(prec, prec),
                                   ctypes.cast(bp, ctypes.c_void_p), ctypes.cast(xp, ctypes.c_void_p), tol, maxit,
                                   it.ctypes.data, _stream(stream))
    if check:
        _check(rc, allow=(SMG_ERR_NOCONV,))
    return rc, it


def smg_batched_setup(dims, npre=1, npost=0, prec="fp32", stream=None) -> int:
    """dims: (nsys, 3) ints (nx, ny, nz).  Returns the batched handle."""
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
    h = ctypes.c_void_p()
    _check(_lib.smg_batched_setup(dims.shape[0], dims.ctypes.data, npre, npost, PRECISIONS.get(prec, prec),
                                  ctypes.byref(h), _stream(stream)))
    return h.value


def smg_batched_solve(h, variant, b_list, x_list, tol=1e-8, maxit=100, stream=None, check=True):
    """b_list, x_list: per-system device tensors.  Returns (status, iters, relres) (numpy arrays)."""
    nsys = len(b_list)
    bp = (ctypes.c_void_p * nsys)(*[_ptr(t) for t in b_list])
    xp = (ctypes.c_void_p * nsys)(*[_ptr(t) for t in x_list])
    it = np.zeros(nsys, dtype=np.int32)
    rel = np.zeros(nsys, dtype=np.float64)
    rc = _lib.smg_batched_solve(ctypes.c_void_p(h), VARIANTS.get(variant, variant), ctypes.cast(bp, ctypes.c_void_p),
                                ctypes.cast(xp, ctypes.c_void_p), ctypes.c_double(tol), maxit, it.ctypes.data,
                                rel.ctypes.data, _stream(stream))
    if check:
        _check(rc, allow=(SMG_ERR_NOCONV,))
    return rc, it, rel


def smg_batched_apply(h, r_list, s_list, stream=None) -> None:
    """One persistent V-cycle launch: s_list[i] = T_i r_list[i] (per-system device tensors)."""
    nsys = len(r_list)
    rp = (ctypes.c_void_p * nsys)(*[_ptr(t) for t in r_list])
    sp = (ctypes.c_void_p * nsys)(*[_ptr(t) for t in s_list])
    _check(_lib.smg_batched_apply(ctypes.c_void_p(h), ctypes.cast(rp, ctypes.c_void_p), ctypes.cast(sp, ctypes.c_void_p),
                                  _stream(stream)))


def smg_batched_destroy(h) -> None:
    _check(_lib.smg_batched_destroy(ctypes.c_void_p(h)))


def smg_batched_info(h) -> dict:
    t, o, b, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    n, la = ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib.smg_batched_info(ctypes.c_void_p(h), ctypes.byref(t), ctypes.byref(o), ctypes.byref(b),
                                 ctypes.byref(n), ctypes.byref(la), ctypes.byref(k)))
    return {"threads": t.value, "order": o.value, "blocks": b.value, "tasks": n.value, "launches": la.value,
            "rows_per_lane": k.value}


def smg_batched_set_profile(h, on: int) -> None:
    _check(_lib.smg_batched_set_profile(ctypes.c_void_p(h), on))


def smg_batched_profile_read(h, which: int):
    n, ms, by = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.smg_batched_profile_read(ctypes.c_void_p(h), which, ctypes.byref(n), ctypes.byref(ms),
                                         ctypes.byref(by)))
    return n.value, ms.value, by.value


def bf16_bits(w) -> np.ndarray:
    """FP32 values as BF16 bit patterns (round to nearest, ties to even) -- the weight format of
    smg_set_learned."""
    u = np.ascontiguousarray(np.asarray(w, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def smg_set_learned(h, w, enable=True) -> None:
    """w: SMG_NET_WEIGHTS values (FP32/FP64, rounded to BF16 here) or BF16 bit patterns (uint16)."""
    if not enable:
        _check(_lib.smg_set_learned(h, None, 0))
        return
    w = np.asarray(w)
    bits = w if w.dtype == np.uint16 else bf16_bits(w)
    bits = np.ascontiguousarray(bits.ravel())
    assert bits.size == NET_WEIGHTS
    _check(_lib.smg_set_learned(h, bits.ctypes.data, 1))


def smg_learned_stats(h):
    c, a = ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib.smg_learned_stats(h, ctypes.byref(c), ctypes.byref(a)))
    return c.value, a.value


def smg_collect_pairs(h, b, xstar, rho_out, e_out, max_pairs, tol=1e-8, maxit=100, stream=None) -> int:
    n = ctypes.c_int(0)
    _check(_lib.smg_collect_pairs(h, _ptr(b), _ptr(xstar), tol, maxit, _ptr(rho_out), _ptr(e_out), max_pairs,
                                  ctypes.byref(n), _stream(stream)))
    return n.value


def _w32(w):
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float32).ravel())
    assert w.size == NET_WEIGHTS
    return w


def smg_net_forward(dims, act, w, rho, delta, stream=None) -> None:
    nx, ny, nz = map(int, dims)
    w = _w32(w)
    _check(_lib.smg_net_forward(nx, ny, nz, PRECISIONS.get(act, act), w.ctypes.data, _ptr(rho), _ptr(delta),
                                _stream(stream)))


def smg_net_loss_grad(dims, act, w, rho, e, stream=None):
    nx, ny, nz = map(int, dims)
    w = _w32(w)
    loss = ctypes.c_double()
    g = np.zeros(NET_WEIGHTS, dtype=np.float32)
    _check(_lib.smg_net_loss_grad(nx, ny, nz, PRECISIONS.get(act, act), w.ctypes.data, _ptr(rho), _ptr(e),
                                  ctypes.byref(loss), g.ctypes.data, _stream(stream)))
    return loss.value, g


def smg_net_train(dims_list, rho_list, e_list, w, epochs=3, lr=1e-3, seed=0, act="bf16", stream=None):
    """Returns (trained FP32 weights, per-epoch mean loss)."""
    npairs = len(rho_list)
    dims = np.ascontiguousarray(np.asarray(dims_list, dtype=np.int32).reshape(-1, 3))
    assert dims.shape[0] == npairs == len(e_list)
    rp = (ctypes.c_void_p * npairs)(*[_ptr(t) for t in rho_list])
    ep = (ctypes.c_void_p * npairs)(*[_ptr(t) for t in e_list])
    w = _w32(w).copy()
    hist = np.zeros(epochs, dtype=np.float64)
    _check(_lib.smg_net_train(npairs, dims.ctypes.data, ctypes.cast(rp, ctypes.c_void_p), ctypes.cast(ep, ctypes.c_void_p),
                              epochs, lr, seed, PRECISIONS.get(act, act), w.ctypes.data, hist.ctypes.data,
                              _stream(stream)))
    return w, hist


def smg_net_set_tensor_cores(on: bool) -> None:
    _check(_lib.smg_net_set_tensor_cores(1 if on else 0))


def smg_net_tc_status() -> int:
    e = ctypes.c_int(0)
    _check(_lib.smg_net_tc_status(ctypes.byref(e)))
    return e.value


def smg_barrier_selftest(extra_blocks: int, limit_seconds: float = 0.5, stream=None) -> int:
    st = ctypes.c_int(-99)
    _check(_lib.smg_barrier_selftest(extra_blocks, limit_seconds, ctypes.byref(st), _stream(stream)))
    return st.value


def smg_krylov_history(h: int) -> np.ndarray:
    """||r_k|| / ||b||, k = 0 .. iters, of the handle's last krylov_solve."""
    cnt = ctypes.c_int(0)
    _check(_lib.smg_krylov_history(ctypes.c_void_p(h), None, 0, ctypes.byref(cnt)))
    out = np.zeros(cnt.value, dtype=np.float64)
    if cnt.value:
        _check(_lib.smg_krylov_history(ctypes.c_void_p(h), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       cnt.value, ctypes.byref(cnt)))
    return out


def smg_gram(n: int, k1: int, U, k2: int, V, G, stream=None) -> None:
    """G (device, k1 x k2 row-major) = U^T V with U, V column-major device blocks (n rows)."""
    _check(_lib.smg_gram(n, k1, _ptr(U), k2, _ptr(V), _ptr(G), _stream(stream)))


def smg_destroy(h: int) -> None:
    _check(_lib.smg_destroy(h))


class Handle:
    """Owns one smg_handle (context manager); attribute access only marshals arguments."""

    def __init__(self, nx, ny, nz, npre=1, npost=1, precision="fp64"):
        self.h = smg_setup(nx, ny, nz, npre, npost)
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        if precision != "fp64":
            smg_set_precision(self.h, precision)

    def close(self):
        if self.h:
            smg_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
