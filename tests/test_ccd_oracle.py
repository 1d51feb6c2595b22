"""Pins of the point-patch continuous collision oracle (Sec. 5, Eq. ineqccd) against references
other than itself: dense time sampling of the box condition, the closed form of a translating
plane, the static case against the pinned ray search, and an independent multi-start Newton
search in (u, v, s) on a deforming shell."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

import ray_brute as RB


def _inside_box(S_, dS, x0, dx, s):
    """Brute force: is x0 + s dx inside the box of the control points S + s dS, per sample s."""
    P = S_.reshape(-1, 3)[None, :, :] + s[:, None, None] * dS.reshape(-1, 3)[None, :, :]
    x = x0[None, :] + s[:, None] * dx[None, :]
    return np.all((P.min(1) <= x) & (x <= P.max(1)), axis=1)


def test_feasible_times_against_dense_sampling():
    """Eq. ineqccd: the union/intersection of half-lines equals the set of sampled times at which
    the point is inside the moving box, away from the interval ends; random nets and motions,
    including nets with a zero displacement component and points resting on a face."""
    rng = np.random.default_rng(3)
    s = np.linspace(0.0, 1.0, 20001)
    n_nonempty = n_split = 0
    for trial in range(300):
        S_ = rng.normal(size=(4, 4, 3)) * 0.3
        dS = rng.normal(size=(4, 4, 3)) * 0.5
        if trial % 10 == 0:
            dS[..., 2] = 0.0                       # b = 0 control points
        x0 = rng.normal(size=3) * 0.5
        dx = rng.normal(size=3) * 0.8
        if trial % 15 == 0:
            x0[1] = S_[..., 1].min()               # on a face at s = 0
            dx[1] = dS[..., 1].reshape(-1)[np.argmin(S_[..., 1])]
        iv = O.ccd_feasible(S_, dS, x0, dx)
        inside = _inside_box(S_, dS, x0, dx, s)
        member = np.zeros_like(inside)
        near = np.zeros_like(inside)
        for lo, hi in iv:
            assert 0.0 <= lo <= hi <= 1.0
            member |= (s >= lo) & (s <= hi)
            near |= (np.abs(s - lo) < 1e-9) | (np.abs(s - hi) < 1e-9)
        assert np.array_equal(member[~near], inside[~near]), trial
        assert all(iv[i][1] < iv[i + 1][0] for i in range(len(iv) - 1))
        n_nonempty += bool(iv)
        n_split += len(iv) > 1
    assert n_nonempty > 30 and n_split > 0


@pytest.mark.parametrize("use_newton", [True, False])
def test_translating_plane_closed_form(use_newton):
    """A flat sheet translating up by 2 cm: contact at s = (z0 - 0) / (dx_z - 0.02) when that is
    in [0, 1] and the contact point is over the sheet; patch and (u, v) from that point."""
    g, q, dq, x0, dx = S.ccd_scene("plane", 1500)
    s, patch, uv, flags = O.ccd_points(g, q, dq, x0, dx, use_newton)
    with np.errstate(divide="ignore", invalid="ignore"):
        sc = (0.0 - x0[:, 2]) / (dx[:, 2] - 0.02)
    X = x0 + sc[:, None] * dx
    hit = (sc >= 0) & (sc <= 1) & (X[:, 0] >= 0) & (X[:, 0] <= 1) & (X[:, 1] >= 0) & (X[:, 1] <= 1)
    assert hit.sum() > 100 and (~hit).sum() > 100
    assert np.array_equal((flags & 1) == 1, hit)
    tol = 1e-12 if use_newton else 1e-7
    np.testing.assert_allclose(s[hit], sc[hit], rtol=0, atol=tol)
    i = np.minimum((X[hit, 0] / g.dxi1).astype(int), g.nu - 1)
    j = np.minimum((X[hit, 1] / g.dxi2).astype(int), g.nv - 1)
    interior = (np.abs(X[hit, 0] / g.dxi1 - np.round(X[hit, 0] / g.dxi1)) > 1e-6) & \
               (np.abs(X[hit, 1] / g.dxi2 - np.round(X[hit, 1] / g.dxi2)) > 1e-6)
    assert np.array_equal(patch[hit][interior], (j * g.nu + i)[interior])
    np.testing.assert_allclose(uv[hit][interior, 0], (X[hit, 0] / g.dxi1 - i)[interior], atol=1e-6)


def test_static_shell_reduces_to_ray_search():
    """With dq = 0 a moving point is a ray segment: s |dx| equals the ray search's tau wherever
    the ray hits within the segment, with the same patch (Newton split on both)."""
    g, q, dq, x0, dx = S.ccd_scene("static", 800)
    s, patch, uv, flags = O.ccd_points(g, q, dq, x0, dx, True)
    L = np.linalg.norm(dx, axis=1)
    tau, rp, ruv, rf = O.trace_rays(g, q, x0, dx / L[:, None], True)
    within = ((rf & 1) == 1) & (tau <= L)
    assert within.sum() > 50
    assert np.array_equal((flags & 1) == 1, within)
    np.testing.assert_allclose(s[within] * L[within], tau[within], rtol=0, atol=1e-10)
    assert np.array_equal(patch[within], rp[within])


@pytest.mark.parametrize("use_newton,tol", [(True, 1e-9), (False, 1e-7)])
def test_deforming_shell_against_multistart_newton(use_newton, tol):
    """The deforming drape on a 6 x 6-patch sheet: contact or not, the earliest s and its patch
    agree with an independent multi-start Newton search in (u, v, s) over every patch.
    Tolerances from the stopping rules: the Newton split stops at a residual of
    1e-12 (1 + |x0| + |dx|), about 2e-12 here, which moves s by that over the normal relative
    speed (down to about 1e-2 per step): 1e-9. The midpoint split stops at a box of 1e-9 per
    axis crossed at such speeds: 1e-7."""
    g, _, q = S.sheet_sinusoid(6, 3, 0.05)
    _, _, q1 = S.sheet_sinusoid(6, 7, 0.05)
    q1 = q1.copy()
    q1[:, 2] -= 0.02
    dq = q1 - q
    _, _, _, x0, dx = S.ccd_scene("drape", 60, seed=21)
    s, patch, uv, flags = O.ccd_points(g, q, dq, x0, dx, use_newton)
    n_hit = 0
    for k in range(len(x0)):
        ref = RB.earliest_contact(g, q, dq, x0[k], dx[k])
        assert bool(flags[k] & 1) == (ref is not None), k
        if ref is not None:
            n_hit += 1
            assert abs(s[k] - ref[0]) <= tol, (k, s[k], ref)
            assert patch[k] == ref[1]
    assert 5 < n_hit < len(x0)


def test_contact_point_lies_on_the_moving_surface():
    """For every contact of the Newton split, X(u, v) + s D(u, v) = x0 + s dx to 1e-11
    (Hermite basis, independent of the Bezier form)."""
    g, q, dq, x0, dx = S.ccd_scene("drape", 300)
    s, patch, uv, flags = O.ccd_points(g, q, dq, x0, dx, True)
    hits = np.flatnonzero(flags & 1)
    assert len(hits) > 30
    for k in hits:
        X, _, _ = RB.evaluate(RB.patch_coeffs(g, q, patch[k]), uv[k:k + 1, 0], uv[k:k + 1, 1])
        D, _, _ = RB.evaluate(RB.patch_coeffs(g, dq, patch[k]), uv[k:k + 1, 0], uv[k:k + 1, 1])
        np.testing.assert_allclose(X[0] + s[k] * D[0], x0[k] + s[k] * dx[k], atol=1e-11)


def test_newton_split_needs_fewer_splits():
    g, q, dq, x0, dx = S.ccd_scene("drape", 1000)
    a = O.ccd_points(g, q, dq, x0, dx, True, want_stats=True)
    b = O.ccd_points(g, q, dq, x0, dx, False, want_stats=True)
    assert np.array_equal(a[3] & 1, b[3] & 1)
    assert a[4][:, 0].sum() < 0.7 * b[4][:, 0].sum()


def test_breathing_cylinder_against_multistart_newton():
    """A periodic cylinder expanding radially (patches across the u seam included): contact or
    not, earliest s and patch against the independent multi-start Newton search."""
    g, q, dq, x0, dx = S.ccd_scene("cylinder", 40, seed=5)
    s, patch, uv, flags = O.ccd_points(g, q, dq, x0, dx, True)
    n_hit = 0
    for k in range(len(x0)):
        ref = RB.earliest_contact(g, q, dq, x0[k], dx[k], starts=4, s_starts=(0.2, 0.8))
        assert bool(flags[k] & 1) == (ref is not None), k
        if ref is not None:
            n_hit += 1
            assert abs(s[k] - ref[0]) <= 1e-9 and patch[k] == ref[1]
    assert 5 < n_hit < len(x0)
