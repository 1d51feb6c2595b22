"""Pins of the ray-patch intersection oracle (Sec. 5) against references other than itself:
the textbook Hermite basis, exact rational slab clipping, the plane's closed form and an
independent multi-start Newton search on curved shells."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

import ray_brute as RB


def _random_shell(seed=5):
    g, rest, q = S.sheet_noisy(3, 2e-2, seed)
    return g, q


def test_bezier_form_equals_hermite_patch():
    """Step 1 (Bezier points b1 = a + a'/3, b2 = b - b'/3 and the twist term) reproduces the
    Hermite patch and its first derivatives at random points."""
    for g, q in (_random_shell(), S.cylinder(5, 3)):
        rng = np.random.default_rng(0)
        for p in range(g.nu * g.nv):
            P = O.bezier_patch(g, q, p)
            C = RB.patch_coeffs(g, q, p)
            u, v = rng.random(6), rng.random(6)
            x, xu, xv = RB.evaluate(C, u, v)
            for k in range(6):
                bx, bxu, bxv = O.bezier_eval(P, u[k], v[k])
                np.testing.assert_allclose(bx, x[k], rtol=0, atol=1e-14)
                np.testing.assert_allclose(bxu, xu[k], rtol=0, atol=1e-13)
                np.testing.assert_allclose(bxv, xv[k], rtol=0, atol=1e-13)


def test_bezier_corners_interpolate_nodes():
    """Corner control points are the nodal positions (Bezier endpoint interpolation)."""
    g, q = _random_shell(7)
    qn = q.reshape(-1, 12)
    for p in range(g.nu * g.nv):
        P = O.bezier_patch(g, q, p)
        nd = RB.patch_corners(g, p)
        for k, (i, j) in enumerate(((0, 0), (3, 0), (0, 3), (3, 3))):
            np.testing.assert_array_equal(P[i, j], qn[nd[k], 0:3])


def test_de_casteljau_piece_is_a_reparametrisation():
    """A sub-patch [u0, u1] x [v0, v1] evaluated at (s, t) is the patch at
    (u0 + s (u1 - u0), v0 + t (v1 - v0)); its derivatives carry the chain-rule factors."""
    rng = np.random.default_rng(1)
    P = rng.normal(size=(4, 4, 3))
    for u0, u1, v0, v1 in ((0.0, 1.0, 0.0, 1.0), (0.25, 0.5, 0.5, 1.0), (0.1234, 0.1299, 0.77, 0.91)):
        Sb = O.bezier_sub(P, u0, u1, v0, v1)
        for s, t in rng.random((5, 2)):
            a, au, av = O.bezier_eval(Sb, s, t)
            b, bu, bv = O.bezier_eval(P, u0 + s * (u1 - u0), v0 + t * (v1 - v0))
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)
            np.testing.assert_allclose(au, bu * (u1 - u0), rtol=0, atol=1e-12)
            np.testing.assert_allclose(av, bv * (v1 - v0), rtol=0, atol=1e-12)
    # the whole range reproduces the net exactly
    np.testing.assert_array_equal(O.bezier_sub(P, 0.0, 1.0, 0.0, 1.0), P)


def _exact_slab(lo, hi, o, d):
    """Liang-Barsky clipping in exact rational arithmetic: tau interval (>= 0) or None."""
    t0, t1 = Fraction(0), None
    for k in range(3):
        ok, dk = Fraction(o[k]), Fraction(d[k])
        if dk == 0:
            if ok < Fraction(lo[k]) or ok > Fraction(hi[k]):
                return None
            continue
        a, b = (Fraction(lo[k]) - ok) / dk, (Fraction(hi[k]) - ok) / dk
        if a > b:
            a, b = b, a
        t0 = max(t0, a)
        t1 = b if t1 is None else min(t1, b)
    if t1 is not None and t0 > t1:
        return None
    return t0, t1


def test_ray_box_matches_exact_clipping():
    """Eq. ineqray: the slab interval against exact rational clipping of the control points'
    box, including an axis-parallel ray, an origin inside the box and a box behind the ray."""
    rng = np.random.default_rng(2)
    cases = []
    for _ in range(200):
        Sb = rng.normal(size=(4, 4, 3))
        o = rng.normal(size=3) * 3
        d = rng.normal(size=3)
        cases.append((Sb, o, d / np.linalg.norm(d)))
    Sb = rng.random((4, 4, 3))
    cases.append((Sb, np.array([0.5, 0.5, -2.0]), np.array([0.0, 0.0, 1.0])))   # axis-parallel, hit
    cases.append((Sb, np.array([5.0, 0.5, -2.0]), np.array([0.0, 0.0, 1.0])))   # axis-parallel, miss
    cases.append((Sb, Sb.reshape(-1, 3).mean(0), np.array([0.6, 0.0, 0.8])))    # origin inside
    cases.append((Sb, np.array([0.5, 0.5, 3.0]), np.array([0.0, 0.6, 0.8])))    # box behind
    hits = 0
    for Sb, o, d in cases:
        lo, hi = Sb.reshape(-1, 3).min(0), Sb.reshape(-1, 3).max(0)
        ref = _exact_slab(lo, hi, o, d)
        hit, t0, t1, ext = O.ray_box(Sb, o, d)
        assert hit == (ref is not None)
        if hit:
            hits += 1
            assert ext == float(max(hi - lo))
            assert t0 == pytest.approx(float(ref[0]), rel=1e-14, abs=1e-15)
            assert t1 == pytest.approx(float(ref[1]), rel=1e-14, abs=1e-15)
    assert hits > 10


@pytest.mark.parametrize("use_newton", [True, False])
def test_plane_closed_form(use_newton):
    """A flat 10 x 10 sheet in z = 0: tau = -o_z / d_z, patch and local parameters from the hit
    point's (x, y); rays that point away or run parallel to the sheet miss."""
    g, q, eye, tgt = S.ray_scenes()["plane"]
    o, d = S.camera_rays(24, 18, eye, tgt)
    tau, patch, uv, flags = O.trace_rays(g, q, o, d, use_newton)
    t = -o[:, 2] / d[:, 2]
    X = o + t[:, None] * d
    inside = (X[:, 0] >= 0) & (X[:, 0] <= 1) & (X[:, 1] >= 0) & (X[:, 1] <= 1) & (t > 0)
    assert inside.sum() > 50 and (~inside).sum() > 50
    assert np.array_equal(flags & 1 == 1, inside)
    assert not (flags & 2).any()
    tol = 1e-12 if use_newton else 2e-9
    np.testing.assert_allclose(tau[inside], t[inside], rtol=0, atol=tol)
    i = np.minimum((X[inside, 0] / g.dxi1).astype(int), g.nu - 1)
    j = np.minimum((X[inside, 1] / g.dxi2).astype(int), g.nv - 1)
    interior = (np.abs(X[inside, 0] / g.dxi1 - np.round(X[inside, 0] / g.dxi1)) > 1e-6) & \
               (np.abs(X[inside, 1] / g.dxi2 - np.round(X[inside, 1] / g.dxi2)) > 1e-6)
    assert np.array_equal(patch[inside][interior], (j * g.nu + i)[interior])
    lu = X[inside, 0] / g.dxi1 - i
    lv = X[inside, 1] / g.dxi2 - j
    np.testing.assert_allclose(uv[inside][interior, 0], lu[interior], atol=1e-8)
    np.testing.assert_allclose(uv[inside][interior, 1], lv[interior], atol=1e-8)
    # away from the sheet and parallel to it
    o2 = np.array([[0.5, 0.5, 1.0], [0.5, 0.5, 0.1]])
    d2 = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    _, p2, _, f2 = O.trace_rays(g, q, o2, d2, use_newton)
    assert not (f2 & 1).any() and (p2 == -1).all()


@pytest.mark.parametrize("scene", ["cylinder", "drape"])
def test_curved_scenes_against_multistart_newton(scene):
    """Hit or miss, the nearest tau and its patch agree with an independent multi-start Newton
    search over every patch. Newton variant within 1e-11; the midpoint variant within 1e-8 (its
    refined box is at most EPS_TAU = 1e-9 on each side)."""
    g, q, eye, tgt = S.ray_scenes()[scene]
    if scene == "drape":
        g, _, q = S.sheet_sinusoid(6, 3, amplitude=0.05)
    o, d = S.camera_rays(10, 8, eye, tgt)
    res = {nw: O.trace_rays(g, q, o, d, nw) for nw in (True, False)}
    n_hit = 0
    for k in range(len(o)):
        ref = RB.nearest(g, q, o[k], d[k])
        for nw, tol in ((True, 1e-11), (False, 1e-8)):
            tau, patch, uv, flags = (a[k] for a in res[nw])
            assert bool(flags & 1) == (ref is not None), (scene, k, nw)
            if ref is not None:
                assert abs(tau - ref[0]) <= tol, (scene, k, nw, tau, ref)
                assert patch == ref[1]
                if nw:
                    assert abs(uv[0] - ref[2]) <= 1e-8 and abs(uv[1] - ref[3]) <= 1e-8
        n_hit += ref is not None
    assert 10 < n_hit < len(o)


def test_hit_point_lies_on_ray_and_surface():
    """x(u, v) of the reported patch equals o + tau d (Eq. ray) for every hit, evaluated with the
    Hermite basis."""
    g, q, eye, tgt = S.ray_scenes()["drape"]
    o, d = S.camera_rays(16, 12, eye, tgt)
    tau, patch, uv, flags = O.trace_rays(g, q, o, d, True)
    hit = np.flatnonzero(flags & 1)
    assert len(hit) > 20
    for k in hit:
        x, _, _ = RB.evaluate(RB.patch_coeffs(g, q, patch[k]), np.array([uv[k, 0]]), np.array([uv[k, 1]]))
        np.testing.assert_allclose(x[0], o[k] + tau[k] * d[k], atol=1e-11)


def test_newton_variant_splits_fewer_candidates():
    """Fig. subany against Fig. submid: same hits, fewer candidates split with Newton."""
    g, q, eye, tgt = S.ray_scenes()["cylinder"]
    o, d = S.camera_rays(24, 18, eye, tgt)
    a = O.trace_rays(g, q, o, d, True, want_stats=True)
    b = O.trace_rays(g, q, o, d, False, want_stats=True)
    assert np.array_equal(a[1], b[1])
    assert a[4][:, 0].sum() < 0.5 * b[4][:, 0].sum()
