"""GPU parity of the learned warm start (shell_mlp_*, shell_node_features, shell_warm_targets)
against the FP64 oracle in oracle/mlp.py, and what the trained network gains over the plain
zero-guess Newton.

Tolerances. The kernels store the normalised input, the weights used in products, the hidden
activations and the back-propagated dZ in BF16 and accumulate in FP32. Against an oracle that
rounds the same quantities to BF16 (bf16=True) the remaining differences are FP32 accumulation
(about sqrt(K) 2^-24 relative) and rare BF16 rounding flips of values that FP32 and FP64 place on
opposite sides of a tie: normwise relative <= 1e-3. Against the plain FP64 oracle the BF16
storage itself (2^-9 relative per rounding, a few roundings deep) bounds the difference:
normwise relative <= 5e-2. Features and targets are FP64 arithmetic rounded once to FP32:
relative <= 2^-22.
"""
import numpy as np
import pytest

import oracle.mlp as om
from paper_2312_14839_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _norm(seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(0, 0.3, 28), rng.uniform(0.5, 2.0, 28), rng.normal(0, 0.3, 12), rng.uniform(0.5, 2.0, 12))


def _net(max_rows, seed, norm):
    from paper_2312_14839_gb300 import bhem
    net = bhem.Mlp(max_rows)
    p = S.mlp_init_params(seed, last_scale=1.0)
    net.set_params(p)
    net.set_normalization(*[np.asarray(x, dtype=np.float32) for x in norm])
    # the kernels see the FP32 normalisation; give the oracle the same values
    return net, p.astype(np.float64), tuple(np.asarray(x, dtype=np.float32).astype(np.float64) for x in norm)


SHELLS = {
    "sheet9x7": lambda: S.flat_sheet(9, 7),
    "annulus8x3-periodic": lambda: S.annulus(8, 3),
    "sheet1x1": lambda: S.flat_sheet(1, 1),
}


@pytest.mark.parametrize("case", list(SHELLS))
def test_node_features_parity(case):
    from paper_2312_14839_gb300 import bhem
    g, rest = SHELLS[case]()
    rng = np.random.default_rng(10)
    q = S.noisy(rest, 1e-2, 11).reshape(-1)
    v = rng.normal(0, 0.1, g.n_dof)
    want = om.node_features(g, rest, q, v)
    with bhem.Shell(g, S.SHEET_MATERIAL, rest.reshape(-1)) as sh:
        X = host(bhem.node_features(sh, dev(q), dev(v)))
    np.testing.assert_allclose(X, want, rtol=2.0 ** -22, atol=1e-30)


def test_warm_targets_parity():
    from paper_2312_14839_gb300 import bhem
    rng = np.random.default_rng(12)
    n = 12 * 1001
    q, v = rng.normal(size=n), rng.normal(size=n)
    q1 = q + 1e-3 * v + 1e-6 * rng.normal(size=n)
    T = host(bhem.warm_targets(dev(q1), dev(q), dev(v), 1e-3))
    want = om.warm_targets(q1, q, v, 1e-3).reshape(-1)
    # the FP64 difference is cancellation-limited: compare within one FP32 rounding of each term
    np.testing.assert_allclose(T, want, rtol=2.0 ** -22, atol=4 * 2.0 ** -52 * np.abs(q1).max())


@pytest.mark.parametrize("rows", [1, 63, 300, 4097])
def test_forward_parity(rows):
    norm = _norm(20)
    net, p, normf = _net(4097, 21, norm)
    X = np.random.default_rng(22).normal(0, 1.5, (rows, 28))
    Y = host(net.forward(dev(X, torch.float32)))
    Xf = X.astype(np.float32).astype(np.float64)
    want16 = om.predict(p, Xf, normf, bf16=True)
    want64 = om.predict(p, Xf, normf, bf16=False)
    assert rel(Y, want16) <= 1e-3, rel(Y, want16)
    assert rel(Y, want64) <= 5e-2, rel(Y, want64)
    net.close()


@pytest.mark.parametrize("rows,use_idx", [(3000, False), (777, True)])
def test_gradient_parity(rows, use_idx):
    norm = _norm(30)
    data_rows = 5000
    net, p, normf = _net(max(rows, 64), 31, norm)
    rng = np.random.default_rng(32)
    X = rng.normal(0, 1.5, (data_rows, 28)).astype(np.float32)
    T = rng.normal(0, 1.0, (data_rows, 12)).astype(np.float32)
    idx = rng.integers(0, data_rows, rows).astype(np.int32) if use_idx else np.arange(rows, dtype=np.int32)
    loss = net.gradients(dev(X, torch.float32), dev(T, torch.float32),
                         idx=dev(idx, torch.int32) if use_idx else None, rows=rows)
    G = net.get_grads().astype(np.float64)
    Xs, Ts = X[idx].astype(np.float64), T[idx].astype(np.float64)
    loss16, g16 = om.loss_and_grads(p, Xs, Ts, normf, bf16=True)
    loss64, g64 = om.loss_and_grads(p, Xs, Ts, normf, bf16=False)
    assert loss == pytest.approx(loss16, rel=1e-4)
    assert loss == pytest.approx(loss64, rel=5e-2)
    off = 0
    for fi, fo in om.LAYERS:
        for name, size in (("W", fi * fo), ("b", fo)):
            sl = slice(off, off + size)
            assert rel(G[sl], g16[sl]) <= 1e-3, (fi, fo, name, rel(G[sl], g16[sl]))
            assert rel(G[sl], g64[sl]) <= 5e-2, (fi, fo, name, rel(G[sl], g64[sl]))
            off += size
    net.close()


def test_adam_parity():
    norm = _norm(40)
    net, p, _ = _net(512, 41, norm)
    rng = np.random.default_rng(42)
    X = dev(rng.normal(size=(512, 28)), torch.float32)
    T = dev(rng.normal(size=(512, 12)), torch.float32)
    idx = dev(np.arange(512), torch.int32)
    params = net.get_params().astype(np.float64)
    m = np.zeros_like(params)
    v = np.zeros_like(params)
    lr = 2e-3
    for step in range(1, 4):
        net.train_step(X, T, idx, lr)
        g = net.get_grads().astype(np.float64)
        params, m, v = om.adam(params, g, m, v, step, lr)
        # The kernel keeps m and v in FP32: a gradient that changes sign between steps cancels in
        # m = b1 m + (1 - b1) g and loses up to ~7 bits, so each update (size <= a few lr) may differ
        # from the FP64 recursion by ~1e-5 lr; the parameters themselves by one FP32 ulp.
        np.testing.assert_allclose(net.get_params(), params, rtol=2.0 ** -22, atol=2e-5 * lr * step)
    net.close()


def test_training_reduces_loss():
    """A smooth synthetic regression: 400 Adam steps cut the loss at least tenfold."""
    from paper_2312_14839_gb300 import bhem
    rng = np.random.default_rng(50)
    n = 20000
    X = rng.normal(size=(n, 28)).astype(np.float32)
    A = rng.normal(size=(28, 12)) / np.sqrt(28)
    T = (np.tanh(X @ A) + 0.1 * (X[:, :12] ** 2)).astype(np.float32)
    net = bhem.Mlp(2048)
    net.set_params(S.mlp_init_params(51))
    Xd, Td = dev(X, torch.float32), dev(T, torch.float32)
    net.set_normalization(*[np.asarray(a, np.float32) for a in (*net.column_stats(Xd), *net.column_stats(Td))])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(52)
    first = net.gradients(Xd, Td, rows=2048)
    for it in range(400):
        idx = torch.randint(0, n, (2048,), generator=gen, device="cuda", dtype=torch.int32)
        net.train_step(Xd, Td, idx, 1e-3)
    last = net.gradients(Xd, Td, rows=2048)
    assert last < 0.1 * first, (first, last)
    net.close()


def test_index_out_of_range_is_an_error():
    from paper_2312_14839_gb300 import bhem
    net, _, _ = _net(64, 60, _norm(60))
    X = dev(np.zeros((100, 28)), torch.float32)
    T = dev(np.zeros((100, 12)), torch.float32)
    bad = dev(np.array([0, 5, 100, 3]), torch.int32)
    with pytest.raises(bhem.ShellError):
        net.gradients(X, T, idx=bad)
    good = dev(np.array([0, 5, 99, 3]), torch.int32)
    assert np.isfinite(net.gradients(X, T, idx=good))
    net.close()


def test_warm_start_parity():
    from paper_2312_14839_gb300 import bhem
    g, rest = S.flat_sheet(11, 6)
    q = S.noisy(rest, 1e-2, 70).reshape(-1)
    v = np.random.default_rng(71).normal(0, 0.1, g.n_dof)
    norm = (np.zeros(28), np.full(28, 0.05), np.zeros(12), np.full(12, 1e-4))
    net, p, normf = _net(g.n_nodes, 72, norm)
    dt = 1e-3
    with bhem.Shell(g, S.SHEET_MATERIAL, rest.reshape(-1)) as sh:
        w = host(net.warm_start(sh, dev(q), dev(v), dt))
        wi = host(bhem.inertial_warm_start(sh, dev(q), dev(v), dt))
    inertial = q + dt * v
    # one rounding of q + dt v (fused or not), measured against the operands' size
    np.testing.assert_allclose(wi, inertial, rtol=0, atol=2.0 ** -51 * float(np.abs(q).max() + dt * np.abs(v).max()))
    X = om.node_features(g, rest, q, v).astype(np.float32).astype(np.float64)
    pred = om.predict(p, X, normf, bf16=True).reshape(-1)
    assert rel(w - inertial, pred) <= 1e-3
    net.close()


def test_learned_warm_start_gains():
    """Train on trajectories of the plain solver (16x16 sheets, corner twists), then roll out an
    unseen trajectory: the learned start needs fewer Newton iterations than the zero guess, every
    step still meets the 1e-8 residual measured from the zero guess, and the states agree with the
    zero-guess rollout to the solver tolerance."""
    from paper_2312_14839_gb300 import learned as L
    scene = L.Scene(n=16)
    data = L.generate(scene, n_traj=12, steps=60, seed=80)
    net = L.make_network(65536, 81)
    L.set_normalization(net, data)
    untrained = L.validation_loss(net, data, rows=65536)
    L.train(net, data, iters=1500, batch_rows=4096, seed=82)
    trained = L.validation_loss(net, data, rows=65536)
    rates = S.corner_twist_rates(83, 1)[0]
    zero = L.rollout(scene, rates, 40, "zero", keep_states=True)
    lrn = L.rollout(scene, rates, 40, "learned", net, keep_states=True)
    g, _, rest = scene.sheet()
    disp = max(float((s - dev(rest.reshape(-1))).abs().max()) for s in zero["states"])
    diff = max(float((a - b).abs().max()) for a, b in zip(lrn["states"], zero["states"]))
    info = dict(untrained=untrained, trained=trained, zero_newton=zero["mean_newton"],
                learned_newton=lrn["mean_newton"], zero_res=zero["max_res_ratio"], learned_res=lrn["max_res_ratio"],
                fallbacks=lrn["fallbacks"], diff=diff, disp=disp)
    assert trained < 0.5 * untrained, info
    assert lrn["max_res_ratio"] <= 1e-8 and zero["max_res_ratio"] <= 1e-8, info
    assert lrn["mean_newton"] < zero["mean_newton"], info
    assert diff <= 1e-4 * disp, info
    net.close()


@pytest.mark.parametrize("grid", [(11, 6), (64, 64)])
def test_fused_warm_start_matches_gemm_path(grid):
    """shell_mlp_warm_start (one fused launch) against the unfused path: node features ->
    shell_mlp_forward (tensor-core GEMM kernels) -> q + dt v + y. Both issue the same tcgen05 MMAs
    over the same K chunks in the same order and finish with the same epilogue arithmetic, so the
    network outputs agree to the rounding of the final FP64 sum."""
    from paper_2312_14839_gb300 import bhem
    g, rest = S.flat_sheet(*grid)
    q = S.noisy(rest, 1e-2, 90).reshape(-1)
    v = np.random.default_rng(91).normal(0, 0.1, g.n_dof)
    net, _, _ = _net(g.n_nodes, 92, (np.zeros(28), np.full(28, 0.05), np.zeros(12), np.full(12, 1e-4)))
    dt = 1e-3
    with bhem.Shell(g, S.SHEET_MATERIAL, rest.reshape(-1)) as sh:
        qd, vd = dev(q), dev(v)
        w = host(net.warm_start(sh, qd, vd, dt))
        Y = host(net.forward(bhem.node_features(sh, qd, vd))).reshape(-1)
    y_fused = w - (q + dt * v)
    scale = np.abs(Y).max()
    assert np.abs(y_fused - Y).max() <= 1e-9 * scale + 8 * 2.0 ** -52 * np.abs(q).max()
    net.close()


def test_tensor_core_wait_timeout_is_reported_and_the_network_recovers():
    """Every mbarrier wait of the network's tcgen05 kernels (the GEMM's TMA stages and MMA
    completion, the fused warm start's weight copies and layers) is bounded. With a budget of 0
    polls each wait expires at once: the kernel drains its own copies and commits, frees its tensor
    memory, skips its output and raises an error bit that the next synchronising call returns as
    SHELL_ERR_TIMEOUT. With the default budget restored the same network computes the same loss and
    gradients as before, and its warm start equals one computed before the expired waits."""
    from paper_2312_14839_gb300 import bhem
    net, _, _ = _net(2000, 41, _norm(40))
    rng = np.random.default_rng(42)
    X = dev(rng.normal(0, 1.5, (2000, 28)), torch.float32)
    T = dev(rng.normal(0, 1.0, (2000, 12)), torch.float32)
    loss0 = net.gradients(X, T)
    G0 = net.get_grads().astype(np.float64)
    g, rest = S.flat_sheet(11, 6)
    q = dev(S.noisy(rest, 1e-2, 43).reshape(-1))
    v = dev(np.random.default_rng(44).normal(0, 0.1, g.n_dof))
    with bhem.Shell(g, S.SHEET_MATERIAL, rest.reshape(-1)) as sh:
        w0 = host(net.warm_start(sh, q, v, 1e-3))
        net.set_wait_budget(0)
        with pytest.raises(bhem.ShellError) as ei:
            net.gradients(X, T)
        assert ei.value.status == 9
        net.warm_start(sh, q, v, 1e-3)
        torch.cuda.synchronize()
        net.set_wait_budget(-1)
        with pytest.raises(bhem.ShellError) as ei:   # raised by the warm start's expired waits
            net.gradients(X, T)
        assert ei.value.status == 9
        loss1 = net.gradients(X, T)
        w1 = host(net.warm_start(sh, q, v, 1e-3))
    assert loss1 == pytest.approx(loss0, rel=1e-12)
    assert rel(net.get_grads().astype(np.float64), G0) <= 1e-5
    np.testing.assert_array_equal(w1, w0)
    net.close()
