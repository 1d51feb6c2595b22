"""Second-order forward-mode automatic differentiation (value, gradient, dense Hessian).

Test helper: differentiates the plain energy definition of Sec. 3.3 (thickness-integrated St.
Venant-Kirchhoff areal density, 4x4 Gauss rule of App. A.2) exactly, to roundoff, with no
truncation error. The oracle's gradient and Hessian follow the closed forms of App. B; comparing
the two pins those closed forms to the energy they are meant to differentiate.
"""
from __future__ import annotations

import math

import numpy as np


class Jet:
    __slots__ = ("v", "g", "H")

    def __init__(self, v, g, H):
        self.v, self.g, self.H = v, g, H

    @staticmethod
    def const(v, n):
        return Jet(float(v), np.zeros(n), None)

    def _h(self):
        return self.H if self.H is not None else 0.0

    def __add__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.v + o, self.g, self.H)
        H = None if self.H is None and o.H is None else self._h() + o._h()
        return Jet(self.v + o.v, self.g + o.g, H)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.g, None if self.H is None else -self.H)

    def __sub__(self, o):
        return self + (-o if isinstance(o, Jet) else -o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if not isinstance(o, Jet):
            return Jet(self.v * o, self.g * o, None if self.H is None else self.H * o)
        og = np.outer(self.g, o.g)
        H = self.v * o._h() + o.v * self._h() + og + og.T
        return Jet(self.v * o.v, self.v * o.g + o.v * self.g, H)

    __rmul__ = __mul__

    def _chain(self, f0, f1, f2):
        H = f1 * self._h() + f2 * np.outer(self.g, self.g)
        return Jet(f0, f1 * self.g, H)

    def inv(self):
        x = self.v
        return self._chain(1.0 / x, -1.0 / x ** 2, 2.0 / x ** 3)

    def sqrt(self):
        x = self.v
        s = math.sqrt(x)
        return self._chain(s, 0.5 / s, -0.25 / (x * s))

    def __truediv__(self, o):
        if not isinstance(o, Jet):
            return self * (1.0 / o)
        return self * o.inv()


def _hermite(p, r, t, d):
    f = [lambda t: 2 * t ** 3 - 3 * t ** 2 + 1, lambda t: 6 * t ** 2 - 6 * t, lambda t: 12 * t - 6]
    g = [lambda t: t ** 3 - 2 * t ** 2 + t, lambda t: 3 * t ** 2 - 4 * t + 1, lambda t: 6 * t - 4]
    if (p, r) == (0, 0):
        return f[d](t)
    if (p, r) == (1, 0):
        return (-1) ** d * f[d](1 - t)
    if (p, r) == (0, 1):
        return g[d](t)
    return -((-1) ** d) * g[d](1 - t)


def shape_table(d1, d2, t1, t2):
    """[16, 6]: Phi, Phi_1, Phi_2, Phi_11, Phi_22, Phi_12, local I = (p+2q)*4 + (r+2s)."""
    out = np.zeros((16, 6))
    for q in range(2):
        for p in range(2):
            for s in range(2):
                for r in range(2):
                    I = (p + 2 * q) * 4 + (r + 2 * s)
                    sc = (d1 if r else 1.0) * (d2 if s else 1.0)
                    u = [_hermite(p, r, t1, k) for k in range(3)]
                    v = [_hermite(q, s, t2, k) for k in range(3)]
                    out[I] = sc * np.array([u[0] * v[0], u[1] * v[0] / d1, u[0] * v[1] / d2,
                                            u[2] * v[0] / d1 ** 2, u[0] * v[2] / d2 ** 2,
                                            u[1] * v[1] / (d1 * d2)])
    return out


def gauss4():
    a = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))
    b = math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
    wa, wb = (18 + math.sqrt(30)) / 36, (18 - math.sqrt(30)) / 36
    return [-b, -a, a, b], [wb, wa, wa, wb]


def _lin(q48, phi_col):
    """3-vector of jets sum_I phi_I q_I (linear in the DOFs: zero Hessian)."""
    out = []
    for c in range(3):
        g = np.zeros(48)
        g[c::3] = phi_col
        out.append(Jet(float(phi_col @ q48[c::3]), g, None))
    return out


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def energy_jet(q48, qb48, d1, d2, young, poisson, h, pseudo=False):
    """Jet of the patch energy E(q) (value, d/dq [48], d^2/dq^2 [48, 48]).

    pseudo=True linearises the bending strain B = (b - b_bar) / 2 at q (its jet keeps the value
    and first derivatives, with a zero Hessian): the Hessian is then the membrane Hessian plus the
    Gauss-Newton bending term, i.e. the exact Hessian without the second derivatives of beta."""
    lam = young * poisson / (1 - poisson ** 2)
    mu = young / (2 * (1 + poisson))
    gx, gw = gauss4()
    E = Jet(0.0, np.zeros(48), np.zeros((48, 48)))
    for j in range(4):
        for i in range(4):
            phi = shape_table(d1, d2, (1 + gx[i]) / 2, (1 + gx[j]) / 2)
            W = (d1 * gw[i] / 2) * (d2 * gw[j] / 2)
            # rest geometry (constants)
            ra1 = phi[:, 1] @ qb48.reshape(16, 3)
            ra2 = phi[:, 2] @ qb48.reshape(16, 3)
            rc = [phi[:, 3 + m] @ qb48.reshape(16, 3) for m in range(3)]
            rn = np.cross(ra1, ra2)
            ra3 = rn / np.linalg.norm(rn)
            abar = np.array([[ra1 @ ra1, ra1 @ ra2], [ra1 @ ra2, ra2 @ ra2]])
            bbar = np.array([[rc[0] @ ra3, rc[2] @ ra3], [rc[2] @ ra3, rc[1] @ ra3]])
            ainv = np.linalg.inv(abar)
            sqab = math.sqrt(np.linalg.det(abar))
            # deformed geometry (jets)
            a1 = _lin(q48, phi[:, 1])
            a2 = _lin(q48, phi[:, 2])
            cc = [_lin(q48, phi[:, 3 + m]) for m in range(3)]
            n = _cross(a1, a2)
            sqa = _dot(n, n).sqrt()
            a3 = [nk / sqa for nk in n]
            a = [[_dot(a1, a1), _dot(a1, a2)], [_dot(a1, a2), _dot(a2, a2)]]
            b11, b22, b12 = _dot(cc[0], a3), _dot(cc[1], a3), _dot(cc[2], a3)
            b = [[b11, b12], [b12, b22]]
            A = [[(a[x][y] - abar[x, y]) * 0.5 for y in range(2)] for x in range(2)]
            B = [[(b[x][y] - bbar[x, y]) * 0.5 for y in range(2)] for x in range(2)]
            if pseudo:
                B = [[Jet(B[x][y].v, B[x][y].g, None) for y in range(2)] for x in range(2)]
            V = Jet(0.0, np.zeros(48), None)
            for al in range(2):
                for be in range(2):
                    for ga in range(2):
                        for de in range(2):
                            Hc = lam / 2 * ainv[al, be] * ainv[ga, de] + mu * ainv[be, ga] * ainv[al, de]
                            V = V + (A[al][be] * A[ga][de] * h + B[al][be] * B[ga][de] * (h ** 3 / 3)) * Hc
            E = E + V * (W * sqab)
    return E
