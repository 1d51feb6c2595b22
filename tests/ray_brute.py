"""Independent checks for the ray-patch intersection (Sec. 5), written without the oracle.

The patch is evaluated straight from the textbook cubic Hermite basis
h00 = 2t^3 - 3t^2 + 1, h10 = t^3 - 2t^2 + t, h01 = -2t^3 + 3t^2, h11 = t^3 - t^2
(no Bezier form), and intersections are found by Newton's method from a grid of starts in every
patch, vectorised with numpy. Nothing here shares code with the oracle or the CUDA path.
"""
from __future__ import annotations

import numpy as np


def hermite_basis(t, deriv: int = 0):
    """[4, n] values (or first derivatives) of h00, h10, h01, h11 at t."""
    t = np.asarray(t, dtype=np.float64)
    if deriv == 0:
        return np.stack([2 * t**3 - 3 * t**2 + 1, t**3 - 2 * t**2 + t, -2 * t**3 + 3 * t**2, t**3 - t**2])
    return np.stack([6 * t**2 - 6 * t, 3 * t**2 - 4 * t + 1, -6 * t**2 + 6 * t, 3 * t**2 - 2 * t])


def patch_corners(g, patch: int):
    """Node ids of corners (0,0), (1,0), (0,1), (1,1) of a patch, with periodic wrap."""
    pu, pv = patch % g.nu, patch // g.nu
    n1 = g.nu if g.periodic_u else g.nu + 1
    n2 = g.nv if g.periodic_v else g.nv + 1
    return [((pv + b) % n2) * n1 + (pu + a) % n1 for b in (0, 1) for a in (0, 1)]


def patch_coeffs(g, q, patch: int):
    """C[a, b, 3]: a indexes (h00, h10, h01, h11) in theta1, b the same in theta2."""
    q = np.asarray(q, dtype=np.float64).reshape(-1, 12)
    nd = patch_corners(g, patch)
    C = np.zeros((4, 4, 3))
    for k, (a0, b0) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
        X = q[nd[k]]
        # basis order along one direction: value at 0, slope at 0, value at 1, slope at 1
        ia, ib = 2 * a0, 2 * b0
        C[ia, ib] = X[0:3]
        C[ia + 1, ib] = X[3:6] * g.dxi1
        C[ia, ib + 1] = X[6:9] * g.dxi2
        C[ia + 1, ib + 1] = X[9:12] * g.dxi1 * g.dxi2
    return C


def evaluate(C, u, v):
    """(x, x_u, x_v) [n, 3] at local parameters u, v [n]."""
    Hu, Hv = hermite_basis(u), hermite_basis(v)
    dHu, dHv = hermite_basis(u, 1), hermite_basis(v, 1)
    x = np.einsum("an,bn,abc->nc", Hu, Hv, C)
    xu = np.einsum("an,bn,abc->nc", dHu, Hv, C)
    xv = np.einsum("an,bn,abc->nc", Hu, dHv, C)
    return x, xu, xv


def all_roots(g, q, o, d, starts: int = 6, iters: int = 40):
    """Every root (tau, patch, u, v) of x(u, v) = o + tau d with tau >= 0 that Newton reaches
    from a starts x starts grid in each patch."""
    o, d = np.asarray(o, dtype=np.float64), np.asarray(d, dtype=np.float64)
    out = []
    s = (np.arange(starts) + 0.5) / starts
    U0, V0 = np.meshgrid(s, s, indexing="ij")
    for p in range(g.nu * g.nv):
        C = patch_coeffs(g, q, p)
        u, v = U0.ravel().copy(), V0.ravel().copy()
        x, _, _ = evaluate(C, u, v)
        t = (x - o) @ d
        for _ in range(iters):
            x, xu, xv = evaluate(C, u, v)
            F = x - o - t[:, None] * d
            J = np.stack([xu, xv, -np.broadcast_to(d, xu.shape)], axis=2)
            ok = np.abs(np.linalg.det(J)) > 1e-300
            step = np.zeros_like(F)
            step[ok] = np.linalg.solve(J[ok], -F[ok][..., None])[..., 0]
            u, v, t = u + step[:, 0], v + step[:, 1], t + step[:, 2]
            u, v = np.clip(u, -0.5, 1.5), np.clip(v, -0.5, 1.5)
        x, _, _ = evaluate(C, u, v)
        r = np.linalg.norm(x - o - t[:, None] * d, axis=1)
        good = (r < 1e-12) & (u >= 0) & (u <= 1) & (v >= 0) & (v <= 1) & (t >= 0)
        out += [(t[i], p, u[i], v[i]) for i in np.flatnonzero(good)]
    return out


def nearest(g, q, o, d, **kw):
    """Nearest root (tau, patch, u, v), or None."""
    roots = all_roots(g, q, o, d, **kw)
    return min(roots) if roots else None


def all_contacts(g, q, dq, x0, dx, starts: int = 5, s_starts=(0.1, 0.5, 0.9), iters: int = 40):
    """Every root (s, patch, u, v) in [0, 1] x patch of X(u, v) + s D(u, v) = x0 + s dx (a shell
    moving linearly from q to q + dq, a point moving from x0 to x0 + dx) that Newton reaches from
    a starts x starts x len(s_starts) grid in each patch."""
    x0, dx = np.asarray(x0, dtype=np.float64), np.asarray(dx, dtype=np.float64)
    out = []
    g1 = (np.arange(starts) + 0.5) / starts
    U0, V0, S0 = np.meshgrid(g1, g1, np.asarray(s_starts, dtype=np.float64), indexing="ij")
    for p in range(g.nu * g.nv):
        C = patch_coeffs(g, q, p)
        Cd = patch_coeffs(g, dq, p)
        u, v, s = U0.ravel().copy(), V0.ravel().copy(), S0.ravel().copy()
        for _ in range(iters):
            X, Xu, Xv = evaluate(C, u, v)
            D, Du, Dv = evaluate(Cd, u, v)
            F = X + s[:, None] * D - x0 - s[:, None] * dx
            J = np.stack([Xu + s[:, None] * Du, Xv + s[:, None] * Dv, D - dx], axis=2)
            ok = np.abs(np.linalg.det(J)) > 1e-300
            step = np.zeros_like(F)
            step[ok] = np.linalg.solve(J[ok], -F[ok][..., None])[..., 0]
            u, v, s = u + step[:, 0], v + step[:, 1], s + step[:, 2]
            u, v, s = np.clip(u, -0.5, 1.5), np.clip(v, -0.5, 1.5), np.clip(s, -1.0, 2.0)
        X, _, _ = evaluate(C, u, v)
        D, _, _ = evaluate(Cd, u, v)
        r = np.linalg.norm(X + s[:, None] * D - x0 - s[:, None] * dx, axis=1)
        good = (r < 1e-12) & (u >= 0) & (u <= 1) & (v >= 0) & (v <= 1) & (s >= 0) & (s <= 1)
        out += [(s[i], p, u[i], v[i]) for i in np.flatnonzero(good)]
    return out


def earliest_contact(g, q, dq, x0, dx, **kw):
    roots = all_contacts(g, q, dq, x0, dx, **kw)
    return min(roots) if roots else None
