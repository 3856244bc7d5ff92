"""The learned post-correction on the GPU against the FP64 oracle (oracle/net_oracle.c):
forward pass and loss gradient with FP32 activations (relative 1e-5 against the FP64 oracle)
and with BF16 weights and activations (against the oracle with the same BF16 rounding of its
hidden activations: 3e-4 forward, 1e-3 gradient; against the plain FP64 oracle: 5e-2, since
rounding the activations alone moves the gradient by about 2% even in exact arithmetic), the
correction inside smg_apply and flexible PCG with fixed weights (the same weights handed to the
oracle), the training pairs' defining relation, and training lowering the loss.  Weights are
seeded draws or hand-set special cases, never GPU results."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1212_6680_gb300 import inputs  # noqa: E402
from tests.parity import assert_close  # noqa: E402


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    assert torch.cuda.is_available()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def bf16_round(smg, w):
    """The FP32 values of the BF16 weights the GPU uses (exact, as bit patterns)."""
    return (smg.bf16_bits(w).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def passthrough(omega):
    w1, w2, w3 = np.zeros((16, 1, 27)), np.zeros((16, 16, 27)), np.zeros((1, 16, 27))
    w1[0, 0, 13], w1[1, 0, 13] = 1.0, -1.0
    w2[0, 0, 13], w2[1, 1, 13] = 1.0, 1.0
    w3[0, 0, 13], w3[0, 1, 13] = omega, -omega
    return np.concatenate([w1.ravel(), w2.ravel(), w3.ravel()])


SHAPES = [(37, 21, 13), (64, 9, 5), (1, 1, 1), (3, 1, 7), (33, 4, 4)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("act", ["fp32", "bf16"])
def test_forward_matches_oracle(smg, orc, shape, act):
    nx, ny, nz = shape
    w = inputs.net_init_weights(seed=101, last_scale=1.0)
    if act == "bf16":
        w = bf16_round(smg, w)
    rho = inputs.rhs(nx, ny, nz, seed=102)
    d = torch.empty(rho.size, dtype=torch.float64, device="cuda")
    smg.smg_net_forward(shape, act, w, dev(rho), d)
    d = d.cpu().numpy()
    if act == "fp32":
        assert_close(d, orc.net_forward(w, rho), 1e-5, None, "FP32 forward")
    else:
        # FP32 summation order flips a few BF16 roundings of hidden activations by one ulp: an
        # output element moves by at most about one BF16 ulp (2^-8) of the output's scale
        assert_close(d, orc.net_forward(w, rho, act_bf16=True), 3e-4, None, "BF16 forward", elem_tol=3e-3)
        assert_close(d, orc.net_forward(w, rho), 1e-2, None, "BF16 forward vs the FP64 network")


@pytest.mark.parametrize("shape", [(20, 13, 9), (40, 6, 5)])
@pytest.mark.parametrize("act", ["fp32", "bf16"])
def test_loss_gradient_matches_oracle(smg, orc, shape, act):
    nx, ny, nz = shape
    w = inputs.net_init_weights(seed=111, last_scale=1.0)
    if act == "bf16":
        w = bf16_round(smg, w)
    rho = inputs.rhs(nx, ny, nz, seed=112)
    e = inputs.rhs(nx, ny, nz, seed=113)
    loss, g = smg.smg_net_loss_grad(shape, act, w, dev(rho), dev(e))
    # against the plain FP64 network, rounding the hidden activations to BF16 alone moves single
    # weight gradients by up to ~5% (the element-wise bound there is 1e-1); the oracle with the
    # same BF16 rounding points is the tight check
    refs = [(False, 1e-5, 1e-5)] if act == "fp32" else [(True, 1e-3, 1e-3), (False, 5e-2, 1e-1)]
    for act_bf16, tol, etol in refs:
        loss_ref, g_ref = orc.net_loss_grad(w, rho, e, act_bf16=act_bf16)
        assert abs(loss - loss_ref) <= tol * abs(loss_ref)
        for lo, hi in ((0, 432), (432, 7344), (7344, 7776)):  # each layer on its own scale
            assert_close(g[lo:hi], g_ref[lo:hi], tol, None, f"gradient [{lo}:{hi}] act_bf16={act_bf16}", elem_tol=etol)


@pytest.mark.parametrize("which", ["jacobi", "random"])
def test_apply_with_learned_correction_matches_oracle(smg, orc, which):
    nx, ny, nz = 24, 20, 16
    w = passthrough(1.0 / 6.0) if which == "jacobi" else inputs.net_init_weights(seed=121, last_scale=0.3)
    w = bf16_round(smg, w)
    r = inputs.rhs(nx, ny, nz, seed=122)
    T = orc.SMG(nx, ny, nz, 1, 0)
    T.set_learned(w)
    ref = T.apply(r)
    with smg.Handle(nx, ny, nz, 1, 0) as h:
        smg.smg_set_learned(h.h, w)
        s = torch.empty(r.size, dtype=torch.float64, device="cuda")
        smg.smg_apply(h.h, dev(r), s)
        calls, acc = smg.smg_learned_stats(h.h)
    assert (calls, acc) == (1, T.learned_stats()[1])
    # BF16 activations: the correction carries their rounding; the cycle itself is FP64
    assert_close(s.cpu().numpy(), ref, 2e-3, (nx, ny, nz), "cycle with the learned correction", elem_tol=1e-2)


def test_fpcg_learned_jacobi_matches_oracle_iterations(smg, orc):
    nx, ny, nz = 32, 32, 32
    w = bf16_round(smg, passthrough(1.0 / 6.0))
    b = inputs.rhs(nx, ny, nz, seed=0)
    T = orc.SMG(nx, ny, nz, 1, 0)
    T.set_learned(w)
    ref = orc.krylov(b, "fpcg", T, tol=1e-8)
    for prec in ("fp64", "fp32"):
        with smg.Handle(nx, ny, nz, 1, 0, precision=prec) as h:
            smg.smg_set_learned(h.h, w)
            x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
            rc, it, res = smg.krylov_solve(h.h, "fpcg", dev(b), x, 1e-8, 100)
            calls, acc = smg.smg_learned_stats(h.h)
        assert rc == smg.SMG_OK and res <= 1e-8
        assert abs(it - ref["iters"]) <= 1, (prec, it, ref["iters"])
        # the Jacobi correction shrinks the residual (exactly so in FP64; BF16 activations perturb it)
        assert calls == it and acc >= it // 2


def test_zero_network_leaves_fpcg_unchanged(smg):
    nx, ny, nz = 30, 26, 22
    b = dev(inputs.rhs(nx, ny, nz, seed=1))
    out = []
    for learned in (False, True):
        with smg.Handle(nx, ny, nz, 1, 0, precision="fp32") as h:
            if learned:
                smg.smg_set_learned(h.h, np.zeros(smg.NET_WEIGHTS))
            x = torch.zeros_like(b)
            rc, it, _ = smg.krylov_solve(h.h, "fpcg", b, x, 1e-8, 100)
            if learned:
                assert smg.smg_learned_stats(h.h) == (it, 0)
        out.append((it, x))
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])


def test_collected_pairs_satisfy_their_definition(smg, orc):
    """A e_k = b - A x_k - A s_k and rho_k = r_k - A s_k: with x* solving A x = b to 1e-13,
    A e_k equals rho_k up to the FP32 rounding of the pair; pair 0 has x_0 = 0, r_0 = b, so
    rho_0 = b - A T b, checked against the oracle's cycle."""
    nx, ny, nz = 28, 24, 20
    b = inputs.rhs(nx, ny, nz, seed=2)
    n = b.size
    with smg.Handle(nx, ny, nz, 1, 1) as h64:
        xs = torch.zeros(n, dtype=torch.float64, device="cuda")
        rc, _, res = smg.krylov_solve(h64.h, "fpcg", dev(b), xs, 1e-13, 200)
        assert rc == smg.SMG_OK
    with smg.Handle(nx, ny, nz, 1, 0, precision="fp32") as h:
        rho = torch.zeros(12 * n, dtype=torch.float32, device="cuda")
        e = torch.zeros(12 * n, dtype=torch.float32, device="cuda")
        npairs = smg.smg_collect_pairs(h.h, dev(b), xs, rho, e, 12, tol=1e-8, maxit=100)
    assert 5 <= npairs <= 12
    rho = rho.cpu().numpy().astype(np.float64).reshape(12, nz, ny, nx)
    e = e.cpu().numpy().astype(np.float64).reshape(12, nz, ny, nx)
    for k in range(npairs):
        Ae = orc.apply_A(e[k])
        assert_close(Ae, rho[k], 3e-4, (nx, ny, nz), f"A e_{k} vs rho_{k}", elem_tol=3e-3)
    rho0 = b - orc.apply_A(orc.SMG(nx, ny, nz, 1, 0).apply(b))
    assert_close(rho[0], rho0, 1e-4, (nx, ny, nz), "rho_0", elem_tol=1e-3)


def test_training_lowers_the_loss(smg):
    """Adam over pairs from a few small solves: the mean loss of the last epoch is below the
    first, and the result is finite."""
    dims = inputs.uneven_dims(4, 20, 36, seed=3000)
    rl, el, dl = [], [], []
    for i, (nx, ny, nz) in enumerate(dims):
        nx, ny, nz = int(nx), int(ny), int(nz)
        n = nx * ny * nz
        b = dev(inputs.rhs(nx, ny, nz, seed=3100 + i))
        with smg.Handle(nx, ny, nz, 1, 1) as h64:
            xs = torch.zeros(n, dtype=torch.float64, device="cuda")
            smg.krylov_solve(h64.h, "fpcg", b, xs, 1e-13, 200)
        with smg.Handle(nx, ny, nz, 1, 0, precision="fp32") as h:
            rho = torch.zeros(16 * n, dtype=torch.float32, device="cuda")
            e = torch.zeros(16 * n, dtype=torch.float32, device="cuda")
            k = smg.smg_collect_pairs(h.h, b, xs, rho, e, 16)
        for j in range(k):
            rl.append(rho[j * n:(j + 1) * n])
            el.append(e[j * n:(j + 1) * n])
            dl.append((nx, ny, nz))
    w0 = inputs.net_init_weights(seed=77)
    w, hist = smg.smg_net_train(dl, rl, el, w0, epochs=4, lr=2e-3, seed=5)
    assert np.isfinite(w).all() and np.isfinite(hist).all()
    assert hist[-1] < hist[0], hist


def test_learned_argument_errors(smg):
    with smg.Handle(8, 8, 8, 1, 0) as h:
        with pytest.raises(smg.SMGError):
            smg._check(smg.lib().smg_set_learned(h.h, None, 1))
        with pytest.raises(smg.SMGError):
            smg._check(smg.lib().smg_set_learned(h.h, None, 2))
    with pytest.raises(smg.SMGError):
        smg.smg_net_forward((0, 4, 4), "bf16", np.zeros(smg.NET_WEIGHTS), 0, 0)
    with pytest.raises(smg.SMGError):
        smg.smg_net_forward((4, 4, 4), "fp64", np.zeros(smg.NET_WEIGHTS), 0, 0)


@pytest.mark.parametrize("shape", [(37, 21, 13), (64, 9, 5), (3, 1, 7), (130, 14, 20), (32, 6, 6)])
def test_tensor_core_layer_matches_cuda_cores_and_oracle(smg, orc, shape):
    """The tcgen05 16 -> 16 layer (default) against the CUDA-core kernel on the same BF16 inputs
    and weights (they differ only in FP32 summation order, so in rare BF16 roundings of the hidden
    activation) and against the BF16-activation oracle."""
    nx, ny, nz = shape
    w = bf16_round(smg, inputs.net_init_weights(seed=131, last_scale=1.0))
    rho = dev(inputs.rhs(nx, ny, nz, seed=132))
    out = {}
    try:
        for tc in (True, False):
            smg.smg_net_set_tensor_cores(tc)
            d = torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda")
            smg.smg_net_forward(shape, "bf16", w, rho, d)
            out[tc] = d.cpu().numpy()
    finally:
        smg.smg_net_set_tensor_cores(True)
    assert smg.smg_net_tc_status() == 0
    assert_close(out[True], out[False], 3e-4, None, "tensor cores vs CUDA cores", elem_tol=3e-3)
    ref = orc.net_forward(w, rho.cpu().numpy().reshape(nz, ny, nx), act_bf16=True)
    assert_close(out[True], ref, 3e-4, None, "tensor cores vs the oracle", elem_tol=3e-3)


def test_trained_network_cuts_iterations_on_a_held_out_system(smg):
    """What the trained network gains over the method without it: trained on the GPU (own forward
    and backward kernels, Adam) on pairs from 16 seeded solves with sides in {32..56}, it must
    reach 1e-8 on a held-out 64^3 system (right-hand side seed not used in training) in fewer
    flexible PCG iterations than the bare (1,0) cycle, with every judged correction kept or
    dropped as the judge decides and the true residual at tolerance."""
    from paper_1212_6680_gb300 import learned

    w, info = learned.train(nsys=16, lo=32, hi=56, epochs=6, lr=2e-3, seed=7000)
    assert info["loss_per_epoch"][-1] < info["loss_per_epoch"][0] < 1.0
    n = 64
    b = dev(inputs.rhs(n, n, n, seed=424242))
    its = {}
    for use in (False, True):
        with smg.Handle(n, n, n, 1, 0, precision="fp32") as h:
            if use:
                smg.smg_set_learned(h.h, w)
            x = torch.zeros_like(b)
            rc, it, res = smg.krylov_solve(h.h, "fpcg", b, x, 1e-8, 100)
            assert rc == smg.SMG_OK and res <= 1e-8
            its[use] = it
            if use:
                calls, acc = smg.smg_learned_stats(h.h)
                assert calls == it and acc >= 1
    assert its[True] < its[False], its
