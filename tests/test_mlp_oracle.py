"""Pins of the warm-start network oracle (oracle/mlp.py) against facts that do not come from it:
tabulated normal-CDF values, a routing network with a closed-form output, central finite
differences of the loss, the closed form of Adam's first steps, bfloat16 rounding of exact ties
(and torch's own bfloat16 conversion), and features of fields with known discrete Laplacians."""
import math

import numpy as np
import pytest

import oracle.mlp as om
from paper_2312_14839_gb300 import scenes as S

# Standard normal CDF at 1 and 2 (printed tables, e.g. Abramowitz and Stegun Table 26.1).
PHI1 = 0.8413447460685429
PHI2 = 0.9772498680518208


def test_gelu_tabulated_and_symmetry():
    assert om.gelu(np.array([1.0]))[0] == pytest.approx(PHI1, rel=1e-14)
    assert om.gelu(np.array([-1.0]))[0] == pytest.approx(-(1.0 - PHI1), rel=1e-13)
    assert om.gelu(np.array([2.0]))[0] == pytest.approx(2.0 * PHI2, rel=1e-14)
    assert om.gelu(np.array([0.0]))[0] == 0.0
    x = np.random.default_rng(0).normal(0, 3, 200)
    # Phi(-x) = 1 - Phi(x)  =>  GELU(-x) = GELU(x) - x
    np.testing.assert_allclose(om.gelu(-x), om.gelu(x) - x, rtol=1e-12, atol=1e-12)


def test_gelu_grad_central_differences():
    x = np.linspace(-6, 6, 97)
    h = 1e-5
    fd = (om.gelu(x + h) - om.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(om.gelu_grad(x), fd, rtol=1e-8, atol=1e-9)


def _routing_params():
    """x5 -> hidden1[0] (weight 2) -> hidden2[7] -> hidden3[3] -> output[2]; every hidden bias 10
    keeps GELU in its linear range (x (1 - Phi(x)) < 1e-14 for x >= 8)."""
    layers = [(np.zeros((o, i)), np.zeros(o)) for i, o in om.LAYERS]
    layers[0][0][0, 5] = 2.0
    layers[1][0][7, 0] = 1.0
    layers[2][0][3, 7] = 1.0
    layers[3][0][2, 3] = 1.0
    for l in range(3):
        layers[l][1][:] = 10.0
    layers[3][1][2] = -30.0
    return om.pack(layers)


def test_routing_network_closed_form():
    p = _routing_params()
    x = np.random.default_rng(1).uniform(-0.9, 0.9, (17, om.N_IN))
    y, _ = om.forward(p, x)
    np.testing.assert_allclose(y[:, 2], 2.0 * x[:, 5], atol=1e-12)
    others = np.delete(y, 2, axis=1)
    assert np.abs(others).max() == 0.0


def test_zero_network_loss():
    p = np.zeros(om.n_params())
    rng = np.random.default_rng(2)
    X, T = rng.normal(size=(9, 28)), rng.normal(size=(9, 12))
    norm = (X.mean(0), X.std(0), T.mean(0), T.std(0))
    loss, g = om.loss_and_grads(p, X, T, norm)
    tn = (T - T.mean(0)) / T.std(0)
    # zero weights and biases output 0: the loss is the mean square of the normalised targets (= 1)
    assert loss == pytest.approx(float(np.mean(tn * tn)), rel=1e-14)
    assert loss == pytest.approx(1.0, rel=1e-12)


def test_gradients_central_differences():
    rng = np.random.default_rng(3)
    p = S.mlp_init_params(5, last_scale=1.0).astype(np.float64)
    X, T = rng.normal(size=(8, 28)), rng.normal(size=(8, 12))
    norm = (X.mean(0), X.std(0) * 0.5, T.mean(0), T.std(0))
    _, g = om.loss_and_grads(p, X, T, norm)
    # sample parameters from every weight matrix and bias vector
    offs, idx = 0, []
    for fi, fo in om.LAYERS:
        idx += list(offs + rng.integers(0, fi * fo, 12)) + list(offs + fi * fo + rng.integers(0, fo, 4))
        offs += fi * fo + fo
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (om.loss_and_grads(pp, X, T, norm)[0] - om.loss_and_grads(pm, X, T, norm)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9), k


def test_adam_closed_form_steps():
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    m = v = np.zeros(50)
    lr = 1e-3
    # first step: m_hat = g, v_hat = g^2, so every parameter moves by lr g / (|g| + eps)
    p1, m, v = om.adam(p0, g, m, v, 1, lr)
    np.testing.assert_allclose(p1 - p0, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9)
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    p2, m, v = om.adam(p1, g, m, v, 2, lr)
    np.testing.assert_allclose(p2 - p1, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_round_bf16_ties_and_torch():
    e = 2.0 ** -8
    cases = {1.0 + e: 1.0,                    # tie, even neighbour below
             1.0 + 3 * e: 1.0 + 4 * e,        # tie, even neighbour above
             1.0 + e + 2.0 ** -20: 1.0 + 2 * e,
             -(1.0 + 3 * e): -(1.0 + 4 * e),
             1.5: 1.5, 2.0 ** -100: 2.0 ** -100}
    for x, want in cases.items():
        assert om.round_bf16(np.array([x]))[0] == want, x
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).normal(0, 10, 4000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(om.round_bf16(x), ref)


def test_features_rest_state_and_neighbour_speed():
    """At rest every feature is 0. A uniform position velocity c gives the neighbour-mean speed |c|
    at every node (corners, edges, interior, and on the periodic annulus); a velocity linear in x,
    v_x = (x, 0, 0) with x >= 0, gives the interior mean of x - h, x + h, x, x: x itself."""
    g, rest = S.flat_sheet(5, 3)
    X = om.node_features(g, rest, rest, np.zeros_like(rest))
    assert np.abs(X).max() == 0.0
    c = np.array([0.3, -0.4, 1.2])
    v = np.zeros_like(rest)
    v[:, 0:3] = c
    v[:, 3:12] = 7.0                       # derivative velocities do not enter the speed feature
    X = om.node_features(g, rest, rest, v)
    np.testing.assert_allclose(X[:, 27], np.linalg.norm(c), rtol=1e-15)
    ga, resta = S.annulus(8, 3)
    va = np.zeros_like(resta)
    va[:, 0:3] = c
    Xa = om.node_features(ga, resta, resta, va)
    np.testing.assert_allclose(Xa[:, 27], np.linalg.norm(c), rtol=1e-15)
    r = rest.reshape(-1, 12)
    vl = np.zeros_like(r)
    vl[:, 0] = r[:, 0]
    Xl = om.node_features(g, rest, rest, vl)
    inner = np.array([(j * g.n1 + i) for j in range(1, g.n2 - 1) for i in range(1, g.n1 - 1)])
    np.testing.assert_allclose(Xl[inner, 27], r[inner, 0], rtol=1e-14)


def test_features_affine_and_quadratic_fields():
    n = 6
    g, rest = S.flat_sheet(n, n)
    r = rest.reshape(-1, 12)
    x, y = r[:, 0], r[:, 1]
    hx = 1.0 / n
    rng = np.random.default_rng(6)
    A, c = rng.normal(size=(3, 2)), rng.normal(size=3)
    q = r.copy()
    q[:, 0:3] += (A @ np.stack([x, y])).T + c           # affine displacement
    q[:, 3:12] += rng.normal(size=(r.shape[0], 9))       # derivative DOFs do not enter
    v = rng.normal(size=r.shape)
    X = om.node_features(g, rest, q.reshape(-1), v.reshape(-1))
    inner = np.array([(j * g.n1 + i) for j in range(1, g.n2 - 1) for i in range(1, g.n1 - 1)])
    np.testing.assert_allclose(X[inner, 24:27], 0.0, atol=1e-13)
    np.testing.assert_allclose(X[:, 0:12], (q - r), rtol=0, atol=0)
    np.testing.assert_allclose(X[:, 12:24], v, rtol=0, atol=0)
    q2 = r.copy()
    q2[:, 2] += x * x                                    # u_z = x^2: mean of 4 neighbours = hx^2 / 2
    X2 = om.node_features(g, rest, q2.reshape(-1), np.zeros(g.n_dof))
    np.testing.assert_allclose(X2[inner, 26], hx * hx / 2, rtol=1e-12)
    np.testing.assert_allclose(X2[inner, 24:26], 0.0, atol=0)


def test_warm_targets_constant_velocity():
    rng = np.random.default_rng(7)
    q, v = rng.normal(size=120), rng.normal(size=120)
    dt = 1e-3
    t = om.warm_targets(q + dt * v, q, v, dt)
    assert t.shape == (10, 12)
    np.testing.assert_allclose(t, 0.0, atol=1e-15)
    a = rng.normal(size=120)
    np.testing.assert_allclose(om.warm_targets(q + dt * v + dt * dt * a, q, v, dt).reshape(-1), dt * dt * a,
                               rtol=1e-6, atol=1e-15)
