"""Pins of the learned post-correction oracle (oracle/net_oracle.c) against what does not depend
on it: scipy's correlation (the single-channel case of the convolution), adjoint and linearity
identities, central finite differences of the loss, closed forms for special weights (zero
weights, a ReLU pair that passes the residual through), the dense-matrix form of the cycle with a
Jacobi post-step, and the judge's two outcomes.

The network is not in arXiv:1212.6680; its reading (1 -> 16 -> 16 -> 1 channels, 3x3x3, zero
padding, no bias, ReLU between layers, RMS scaling, energy-norm loss, accept-if-the-residual-
shrinks judge) is stated in net_oracle.c."""
import numpy as np
import pytest

from paper_1212_6680_gb300 import inputs
from tests import dense_ref as D

ndimage = pytest.importorskip("scipy.ndimage")


def rng(seed):
    return np.random.default_rng(seed)


def tap(dx, dy, dz):
    return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)


def passthrough_weights(orc, omega):
    """Net(x) = omega * (relu(x) - relu(-x)) = omega * x with centre taps only."""
    w1, w2, w3 = (np.zeros(s) for s in ((16, 1, 27), (16, 16, 27), (1, 16, 27)))
    c = tap(0, 0, 0)
    w1[0, 0, c], w1[1, 0, c] = 1.0, -1.0
    w2[0, 0, c], w2[1, 1, c] = 1.0, 1.0
    w3[0, 0, c], w3[0, 1, c] = omega, -omega
    w = np.concatenate([w1.ravel(), w2.ravel(), w3.ravel()])
    assert w.size == orc.NET_WEIGHTS
    return w


def test_conv_single_channel_is_scipy_correlate(orc):
    x = rng(1).standard_normal((1, 5, 6, 7))
    k = rng(2).standard_normal((1, 1, 27))
    out = orc.conv3d(k, x)
    ref = ndimage.correlate(x[0], k[0, 0].reshape(3, 3, 3), mode="constant", cval=0.0)
    assert np.allclose(out[0], ref, rtol=0, atol=1e-13)


def test_conv_multichannel_is_sum_of_correlations(orc):
    x = rng(3).standard_normal((3, 4, 5, 6))
    w = rng(4).standard_normal((2, 3, 27))
    out = orc.conv3d(w, x)
    for co in range(2):
        ref = sum(ndimage.correlate(x[ci], w[co, ci].reshape(3, 3, 3), mode="constant", cval=0.0) for ci in range(3))
        assert np.allclose(out[co], ref, rtol=0, atol=1e-12)


def test_conv_adjoint_identity(orc):
    x = rng(5).standard_normal((4, 3, 5, 7))
    g = rng(6).standard_normal((2, 3, 5, 7))
    w = rng(7).standard_normal((2, 4, 27))
    lhs = np.vdot(orc.conv3d(w, x), g)
    rhs = np.vdot(x, orc.conv3d_adj(w, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_conv_weight_gradient_identity(orc):
    # <conv(w, x), g> is linear in w, so it equals <w, dL/dw>
    x = rng(8).standard_normal((3, 4, 4, 5))
    g = rng(9).standard_normal((2, 4, 4, 5))
    w = rng(10).standard_normal((2, 3, 27))
    lhs = np.vdot(orc.conv3d(w, x), g)
    rhs = np.vdot(w, orc.conv3d_wgrad(x, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_loss_gradient_matches_central_differences(orc):
    nx, ny, nz = 5, 4, 3
    w = rng(11).standard_normal(orc.NET_WEIGHTS) * 0.3
    rho = rng(12).standard_normal((nz, ny, nx))
    e = rng(13).standard_normal((nz, ny, nx))
    loss, g = orc.net_loss_grad(w, rho, e)
    idx = np.concatenate([rng(14).choice(432, 12, replace=False),
                          432 + rng(15).choice(6912, 30, replace=False),
                          432 + 6912 + rng(16).choice(432, 12, replace=False)])
    h = 1e-6
    scale = np.abs(g).max()
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (orc.net_loss_grad(wp, rho, e, False)[0] - orc.net_loss_grad(wm, rho, e, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * scale, (i, fd, g[i])


def test_zero_weights_zero_correction_unit_loss(orc):
    rho = rng(17).standard_normal((3, 4, 5))
    w = np.zeros(orc.NET_WEIGHTS)
    assert np.array_equal(orc.net_forward(w, rho), np.zeros_like(rho))
    loss, g = orc.net_loss_grad(w, rho, rng(18).standard_normal(rho.shape))
    assert loss == 1.0
    # zero weights make every pre-activation 0: the ReLUs pass no gradient back and the last
    # layer's inputs are 0, so the whole gradient vanishes
    assert np.array_equal(g, np.zeros_like(g))


@pytest.mark.parametrize("c", [1e-3, 2.5, 1e4])
def test_correction_is_scale_equivariant(orc, c):
    w = rng(19).standard_normal(orc.NET_WEIGHTS) * 0.3
    rho = rng(20).standard_normal((4, 5, 6))
    d1 = orc.net_forward(w, rho)
    d2 = orc.net_forward(w, c * rho)
    assert np.allclose(d2, c * d1, rtol=1e-12, atol=0)


def test_passthrough_weights_give_omega_times_residual(orc):
    rho = rng(21).standard_normal((4, 5, 6))
    w = passthrough_weights(orc, 0.37)
    assert np.allclose(orc.net_forward(w, rho), 0.37 * rho, rtol=1e-14, atol=0)


def test_learned_cycle_with_jacobi_weights_is_dense_post_step(orc):
    """With Net(x) = x/6 (a Jacobi step for the diagonal 6 of A) the judge always accepts, since
    the eigenvalues of A/6 lie in (0, 2), and the preconditioner is the linear map
    T10 + (I - A T10)/6, written here from the dense matrices."""
    nx, ny, nz = 5, 4, 6
    A = D.laplacian3d(nx, ny, nz)
    T10 = D.smg_matrix(A, nx, ny, nz, 1, 0)
    M = T10 + (np.eye(A.shape[0]) - A @ T10) / 6.0
    h = orc.SMG(nx, ny, nz, 1, 0)
    h.set_learned(passthrough_weights(orc, 1.0 / 6.0))
    for seed in (0, 1, 2):
        r = inputs.rhs(nx, ny, nz, seed=seed)
        s = h.apply(r)
        ref = (M @ r.ravel()).reshape(r.shape)
        assert np.linalg.norm(s - ref) <= 1e-12 * np.linalg.norm(ref)
    assert h.learned_stats() == (3, 3)


@pytest.mark.parametrize("omega", [1.0, -1.0 / 6.0])
def test_judge_rejects_a_correction_that_grows_the_residual(orc, omega):
    """omega = 1: (I - A) has eigenvalues down to -11, omega = -1/6: (I + A/6) > I; for a random
    residual both grow its norm, and the correction is dropped."""
    nx, ny, nz = 6, 5, 4
    r = inputs.rhs(nx, ny, nz, seed=3)
    s0 = orc.SMG(nx, ny, nz, 1, 0).apply(r)
    w = passthrough_weights(orc, omega)
    rho = r - orc.apply_A(s0)
    assert np.linalg.norm(rho - omega * orc.apply_A(rho)) >= np.linalg.norm(rho)
    s, acc = orc.learned_correct(w, r, s0)
    assert not acc and np.array_equal(s, s0)


def test_fpcg_with_zero_network_is_plain_fpcg_10(orc):
    nx, ny, nz = 12, 10, 14
    b = inputs.rhs(nx, ny, nz, seed=4)
    plain = orc.krylov(b, "fpcg", orc.SMG(nx, ny, nz, 1, 0), tol=1e-8)
    h = orc.SMG(nx, ny, nz, 1, 0)
    h.set_learned(np.zeros(orc.NET_WEIGHTS))
    learned = orc.krylov(b, "fpcg", h, tol=1e-8)
    assert learned["iters"] == plain["iters"]
    assert np.array_equal(learned["x"], plain["x"])
    calls, acc = h.learned_stats()
    assert calls == plain["iters"] and acc == 0


def test_fpcg_with_jacobi_post_step_converges_no_slower(orc):
    """A Jacobi post-step restores part of the dropped post-smoothing: flexible PCG with it
    reaches 1e-8 in no more iterations than with the bare (1,0) cycle."""
    nx, ny, nz = 16, 16, 16
    b = inputs.rhs(nx, ny, nz, seed=5)
    plain = orc.krylov(b, "fpcg", orc.SMG(nx, ny, nz, 1, 0), tol=1e-8)
    h = orc.SMG(nx, ny, nz, 1, 0)
    h.set_learned(passthrough_weights(orc, 1.0 / 6.0))
    learned = orc.krylov(b, "fpcg", h, tol=1e-8)
    assert learned["status"] == 0 and learned["relres"] <= 1e-8
    assert learned["iters"] <= plain["iters"]


@pytest.mark.parametrize("v,r", [(1.0 + 2.0**-8, 1.0),                 # tie -> even (1.0)
                                 (1.0 + 3 * 2.0**-9, 1.0 + 2.0**-7),   # nearest
                                 (1.0 + 2.0**-7 + 2.0**-8, 1.0 + 2.0**-6),  # tie -> even
                                 (-1.0 - 3 * 2.0**-9, -1.0 - 2.0**-7),
                                 (0.15625, 0.15625),                    # representable: unchanged
                                 (3.0e38, None)])
def test_round_bf16_known_values(orc, v, r):
    if r is None:  # large finite value: stays finite, relative error below 2^-8
        out = orc.round_bf16(v)
        assert np.isfinite(out) and abs(out - v) <= 2.0**-8 * v
        return
    assert orc.round_bf16(v) == r


def _bf16(x):
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _restated_grad(orc, w, rho, e, rnd):
    """The loss gradient written with scipy correlations (an independent restatement of the
    backward pass), hidden activations passed through `rnd`."""
    def conv(wl, x):
        return np.stack([sum(ndimage.correlate(x[ci], wl[co, ci].reshape(3, 3, 3), mode="constant")
                             for ci in range(wl.shape[1])) for co in range(wl.shape[0])])

    def conv_t(wl, g):
        return np.stack([sum(ndimage.correlate(g[co], wl[co, ci].reshape(3, 3, 3)[::-1, ::-1, ::-1], mode="constant")
                             for co in range(wl.shape[0])) for ci in range(wl.shape[1])])

    def wgrad(x, g):
        nz, ny, nx = x.shape[1:]
        xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
        out = np.zeros((g.shape[0], x.shape[0], 27))
        for t in range(27):
            dz, dy, dx = t // 9, (t // 3) % 3, t % 3
            out[:, :, t] = np.einsum("opqr,ipqr->oi", g, xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx])
        return out

    w1, w2, w3 = orc.split_weights(w)
    rms = np.sqrt((rho ** 2).mean())
    x0 = rho / rms
    a1 = rnd(np.maximum(conv(w1, x0[None]), 0))
    a2 = rnd(np.maximum(conv(w2, a1), 0))
    d = e - rms * conv(w3, a2)[0]
    gy = -2 * rms / np.vdot(e, D_apply(e)) * D_apply(d)
    gh2 = conv_t(w3, gy[None]) * (a2 > 0)
    gh1 = conv_t(w2, gh2) * (a1 > 0)
    return np.concatenate([wgrad(x0[None], gh1).ravel(), wgrad(a1, gh2).ravel(), wgrad(a2, gy[None]).ravel()])


def D_apply(u):
    """7-point Dirichlet Laplacian with numpy slicing (independent of the oracle's stencil)."""
    out = 6.0 * u
    out[1:] -= u[:-1]
    out[:-1] -= u[1:]
    out[:, 1:] -= u[:, :-1]
    out[:, :-1] -= u[:, 1:]
    out[:, :, 1:] -= u[:, :, :-1]
    out[:, :, :-1] -= u[:, :, 1:]
    return out


@pytest.mark.parametrize("act_bf16", [False, True])
def test_loss_gradient_matches_scipy_restatement(orc, act_bf16):
    nx, ny, nz = 9, 7, 6
    w = _bf16(inputs.net_init_weights(seed=111, last_scale=1.0))
    rho = inputs.rhs(nx, ny, nz, seed=112)
    e = inputs.rhs(nx, ny, nz, seed=113)
    _, g = orc.net_loss_grad(w, rho, e, act_bf16=act_bf16)
    ref = _restated_grad(orc, w, rho, e, _bf16 if act_bf16 else (lambda v: v))
    for lo, hi in ((0, 432), (432, 7344), (7344, 7776)):
        assert np.linalg.norm(g[lo:hi] - ref[lo:hi]) <= 1e-10 * np.linalg.norm(ref[lo:hi])
    # rounding the activations moves the gradient by a measurable amount (why the BF16 GPU path
    # is held to the BF16-activation oracle)
    if act_bf16:
        _, g64 = orc.net_loss_grad(w, rho, e)
        assert np.linalg.norm(g - g64) > 1e-4 * np.linalg.norm(g64)


def test_crop_around_a_point_reproduces_the_full_grid(orc):
    """The correction at a point depends only on the residual within distance 3 (three 3x3x3
    layers), and its RMS scaling cancels (positive homogeneity), so the oracle on the neighbourhood
    clipped to the grid gives the full-grid value -- the basis of the sampled full-size GPU check."""
    n = 14
    w = inputs.net_init_weights(seed=141, last_scale=1.0)
    rho = inputs.rhs(n, n, n, seed=142)
    full = orc.net_forward(w, rho)
    for (z, y, x) in [(0, 0, 0), (5, 6, 7), (13, 13, 13), (3, 0, 9), (13, 2, 6)]:
        zs, ys, xs = max(z - 3, 0), max(y - 3, 0), max(x - 3, 0)
        c = np.ascontiguousarray(rho[zs:z + 4, ys:y + 4, xs:x + 4])
        v = orc.net_forward(w, c)[z - zs, y - ys, x - xs]
        assert abs(v - full[z, y, x]) <= 1e-12 * max(abs(full[z, y, x]), 1.0)
