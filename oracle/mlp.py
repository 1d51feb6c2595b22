"""FP64 oracle of the learned warm start (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU baseline may import this module; the
product path never does. The paper has no learning component, so nothing here follows a passage
of it: every function restates a textbook definition in plain numpy, one step after the other.

* GELU(x) = x Phi(x), Phi the standard normal CDF (Hendrycks and Gimpel, 2016).
* Dense layers y = W x + b, W [fan_out, fan_in]; hidden layers apply GELU.
* Mean squared error over all rows and the 12 outputs, on per-column normalised targets.
* Back-propagation by the chain rule, layer by layer.
* Adam (Kingma and Ba, 2015, Algorithm 1) with bias-corrected moments.
* Node features and warm-start targets of a shell state (the feature definition of the library's
  warm-start interface): u = q - q_rest, v, the mean of u_nb - u over present edge neighbours for
  the position DOFs, and the mean over the same neighbours of their position speed |v_nb|; targets
  q^{n+1} - q^n - dt v^n.

``bf16=True`` rounds, to the nearest bfloat16 (ties to even), exactly the quantities that the CUDA
kernels store in BF16: the normalised input, the weights used in products, each hidden GELU
activation and each back-propagated dZ used in a product. Everything else stays FP64.

Parity pins: tests/test_mlp_oracle.py (routing network with a closed-form output, GELU at
tabulated points and its symmetry identity, central finite differences of the loss for the
gradients, the first Adam steps' closed form, bfloat16 rounding of exactly representable ties,
features of affine and quadratic displacement fields).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

LAYERS = ((28, 256), (256, 256), (256, 256), (256, 12))
N_IN, N_OUT = 28, 12


def n_params() -> int:
    return sum(i * o + o for i, o in LAYERS)


def unpack(params):
    """Packed vector -> [(W [fan_out, fan_in], b [fan_out]), ...] (FP64 copies)."""
    params = np.asarray(params, dtype=np.float64)
    out, off = [], 0
    for fi, fo in LAYERS:
        W = params[off:off + fi * fo].reshape(fo, fi).copy()
        off += fi * fo
        b = params[off:off + fo].copy()
        off += fo
        out.append((W, b))
    assert off == params.size
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def round_bf16(x):
    """Round to the nearest bfloat16 value, ties to even. The value is first rounded to FP32, as
    the kernels round FP32 values."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    # d/dx [x Phi(x)] = Phi(x) + x phi(x)
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def normalise(x, mean, std):
    std = np.where(np.asarray(std) > 0, std, 1.0)
    return (np.asarray(x, dtype=np.float64) - mean) / std


def forward(params, xn, bf16=False):
    """Forward pass on normalised inputs xn [rows, 28]. Returns (output [rows, 12], cache) where
    cache holds, per layer, the layer input a (as used in the product) and pre-activation z."""
    r = round_bf16 if bf16 else (lambda t: t)
    a = r(np.asarray(xn, dtype=np.float64))
    cache = []
    layers = unpack(params)
    for l, (W, b) in enumerate(layers):
        z = a @ r(W).T + b
        cache.append((a, z))
        a = r(gelu(z)) if l < len(layers) - 1 else z
    return a, cache


def loss_and_grads(params, X, T, norm, bf16=False):
    """MSE loss on normalised targets and its gradient (packed like params).

    norm = (in_mean, in_std, out_mean, out_std). X [rows, 28], T [rows, 12] raw values."""
    in_mean, in_std, out_mean, out_std = norm
    xn = normalise(X, in_mean, in_std)
    tn = normalise(T, out_mean, out_std)
    y, cache = forward(params, xn, bf16)
    rows = y.shape[0]
    diff = y - tn
    loss = float(np.mean(diff * diff))
    dz = 2.0 * diff / (rows * N_OUT)
    r = round_bf16 if bf16 else (lambda t: t)
    layers = unpack(params)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a, _ = cache[l]
        dzr = r(dz)
        grads[l] = (dzr.T @ a, dz.sum(axis=0))
        if l == 0:
            break
        da = dzr @ r(W)
        dz = da * gelu_grad(cache[l - 1][1])
    return loss, pack(grads)


def adam(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1). Returns (params, m, v) as new arrays."""
    m = b1 * m + (1.0 - b1) * grads
    v = b2 * v + (1.0 - b2) * grads * grads
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def predict(params, X, norm, bf16=False):
    """De-normalised network output for raw features X."""
    in_mean, in_std, out_mean, out_std = norm
    y, _ = forward(params, normalise(X, in_mean, in_std), bf16)
    std = np.where(np.asarray(out_std) > 0, out_std, 1.0)
    return y * std + out_mean


def node_features(grid, rest, q, v):
    """[n_nodes, 28] features of a shell state (plain loops over nodes)."""
    n1, n2 = grid.n1, grid.n2
    u = (np.asarray(q, dtype=np.float64).reshape(-1) - np.asarray(rest, dtype=np.float64).reshape(-1))
    u = u.reshape(n1 * n2, 12)
    vv = np.asarray(v, dtype=np.float64).reshape(n1 * n2, 12)
    X = np.zeros((n1 * n2, N_IN))
    for j in range(n2):
        for i in range(n1):
            node = j * n1 + i
            X[node, 0:12] = u[node]
            X[node, 12:24] = vv[node]
            diffs, speeds = [], []
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                a, b = i + di, j + dj
                if grid.periodic_u:
                    a %= n1
                if grid.periodic_v:
                    b %= n2
                if not (0 <= a < n1 and 0 <= b < n2) or (a == i and b == j):
                    continue
                diffs.append(u[b * n1 + a, 0:3] - u[node, 0:3])
                speeds.append(np.linalg.norm(vv[b * n1 + a, 0:3]))
            if diffs:
                X[node, 24:27] = np.mean(diffs, axis=0)
                X[node, 27] = np.mean(speeds)
    return X


def warm_targets(q_next, q, v, dt):
    """q^{n+1} - q^n - dt v^n per DOF, as [n_nodes, 12]."""
    t = np.asarray(q_next, dtype=np.float64) - np.asarray(q, dtype=np.float64) - dt * np.asarray(v, dtype=np.float64)
    return t.reshape(-1, 12)
