"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: values the paper prints,
closed forms, invariants, exact AD of the energy definition, finite differences, a dense direct
solve, or brute force on tiny meshes.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from ad_jet import energy_jet
from paper_2312_14839_gb300 import scenes as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
MAT = S.SHEET_MATERIAL


# --------------------------------------------------------------------------------------------
# App. A.1: Hermite basis
# --------------------------------------------------------------------------------------------
def test_hermite_endpoint_identities():
    """f(0)=1, f(1)=0, g(0)=g(1)=0, f'(0)=f'(1)=0, g'(0)=1, g'(1)=0 (App. A.1)."""
    want = GOLD["hermite_endpoints"]["value"]
    f = lambda t, d=0: O.hermite_w(0, 0, t, d)
    g = lambda t, d=0: O.hermite_w(0, 1, t, d)
    got = {"f(0)": f(0), "f(1)": f(1), "g(0)": g(0), "g(1)": g(1),
           "f'(0)": f(0, 1), "f'(1)": f(1, 1), "g'(0)": g(0, 1), "g'(1)": g(1, 1)}
    for k, v in want.items():
        assert got[k] == pytest.approx(v, abs=1e-15), k


def test_hermite_derivatives_match_finite_differences():
    for p in (0, 1):
        for r in (0, 1):
            for t in (0.1, 0.37, 0.8):
                e = 1e-6
                d1 = (O.hermite_w(p, r, t + e) - O.hermite_w(p, r, t - e)) / (2 * e)
                d2 = (O.hermite_w(p, r, t + e, 1) - O.hermite_w(p, r, t - e, 1)) / (2 * e)
                assert O.hermite_w(p, r, t, 1) == pytest.approx(d1, abs=1e-8)
                assert O.hermite_w(p, r, t, 2) == pytest.approx(d2, abs=1e-8)


def _bicubic(rng):
    C = rng.normal(size=(4, 4, 3))

    def P(x, y, dx=0, dy=0):
        out = np.zeros(3)
        for i in range(4):
            for j in range(4):
                if i < dx or j < dy:
                    continue
                ci = math.factorial(i) / math.factorial(i - dx)
                cj = math.factorial(j) / math.factorial(j - dy)
                out += C[i, j] * ci * cj * x ** (i - dx) * y ** (j - dy)
        return out
    return P


@pytest.mark.parametrize("d1,d2,x0,y0", [(1.0, 1.0, 0.0, 0.0), (0.3, 0.7, 0.4, -0.2), (2.0, 0.05, 1.0, 3.0)])
def test_hermite_reproduces_bicubics_exactly(d1, d2, x0, y0):
    """Bicubic Hermite interpolation (Eq. hermite) is exact on bicubic polynomials, with the
    derivative DOFs taken w.r.t. the global parameters; all 6 shape-derivative kinds agree."""
    rng = np.random.default_rng(1)
    P = _bicubic(rng)
    q = np.zeros(48)
    for qq in range(2):
        for p in range(2):
            x, y = x0 + p * d1, y0 + qq * d2
            c = p + 2 * qq
            q[c * 12:c * 12 + 3] = P(x, y)
            q[c * 12 + 3:c * 12 + 6] = P(x, y, 1, 0)
            q[c * 12 + 6:c * 12 + 9] = P(x, y, 0, 1)
            q[c * 12 + 9:c * 12 + 12] = P(x, y, 1, 1)
    for t1, t2 in [(0.2, 0.9), (0.55, 0.1), (1.0, 0.5)]:
        phi = O.shape(d1, d2, t1, t2)
        x, y = x0 + t1 * d1, y0 + t2 * d2
        Q = q.reshape(16, 3)
        for k, (dx, dy) in enumerate([(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1)]):
            want = P(x, y, dx, dy)
            got = phi[:, k] @ Q
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * (1 + np.abs(want).max())), (k, got, want)


def test_c1_continuity_across_shared_edge():
    """x, a_1 and a_2 agree across a shared edge (App. A.1: C^1 smoothness)."""
    g, rest = S.flat_sheet(2, 1, 1.0, 0.5)
    q = S.noisy(rest, 0.05, 3)
    left, right = O.gather(g, q, 0).reshape(16, 3), O.gather(g, q, 1).reshape(16, 3)
    for t2 in (0.0, 0.3, 0.77, 1.0):
        pl = O.shape(g.dxi1, g.dxi2, 1.0, t2)
        pr = O.shape(g.dxi1, g.dxi2, 0.0, t2)
        for k in range(3):
            assert np.allclose(pl[:, k] @ left, pr[:, k] @ right, atol=1e-13)


# --------------------------------------------------------------------------------------------
# App. A.2: Gauss rule
# --------------------------------------------------------------------------------------------
def test_gauss_nodes_match_printed_values():
    x, w = O.gauss4()
    want = GOLD["gauss_nodes_unit"]["value"]
    assert x[2] == pytest.approx(want[0], abs=5e-7)
    assert x[3] == pytest.approx(want[1], abs=5e-7)
    assert np.allclose(x, -x[::-1]) and w.sum() == pytest.approx(2.0, abs=1e-15)
    # inner lines carry (18 + sqrt 30)/72 of the extent
    assert w[1] / 2 == pytest.approx((18 + math.sqrt(30)) / 72, abs=1e-15)


def test_gauss_exact_to_degree_seven():
    x, w = O.gauss4()
    for k in range(8):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert (w * x ** k).sum() == pytest.approx(exact, abs=1e-14)
    assert abs((w * x ** 8).sum() - 2.0 / 9) > 1e-4   # degree 8 is not integrated exactly


# --------------------------------------------------------------------------------------------
# Sec. 3.3: energy
# --------------------------------------------------------------------------------------------
def _assembled_energy(g, rest, q, mat=MAT):
    E, grad, _ = O.assemble(g, mat, rest, q, want_hess=False)
    return E, grad


@pytest.mark.parametrize("build", [lambda: S.flat_sheet(3, 2, 0.7, 0.4), lambda: S.annulus(8, 2)])
def test_energy_zero_at_rest_and_rigid_invariance(build):
    g, rest = build()
    E0, g0 = _assembled_energy(g, rest, rest)
    assert abs(E0) < 1e-20 and np.abs(g0).max() < 1e-12
    # rotate every 3-vector (x, x_1, x_2, x_12) by R and translate x
    ang = [0.3, -1.1, 0.7]
    Rx = np.array([[1, 0, 0], [0, math.cos(ang[0]), -math.sin(ang[0])], [0, math.sin(ang[0]), math.cos(ang[0])]])
    Rz = np.array([[math.cos(ang[1]), -math.sin(ang[1]), 0], [math.sin(ang[1]), math.cos(ang[1]), 0], [0, 0, 1]])
    R = Rz @ Rx
    q = (rest.reshape(-1, 4, 3) @ R.T).reshape(-1, 12)
    q[:, 0:3] += np.array([0.5, -2.0, 3.0])
    E, grad = _assembled_energy(g, rest, q)
    assert abs(E) < 1e-16 and np.abs(grad).max() < 1e-10


@pytest.mark.parametrize("s1,s2", [(1.1, 1.0), (1.05, 0.97), (1.3, 1.2)])
def test_energy_uniform_stretch_closed_form(s1, s2):
    """x = (s1 xi1, s2 xi2, 0): E = L1 L2 h [lambda/2 (A11 + A22)^2 + mu (A11^2 + A22^2)]."""
    L1, L2 = 0.7, 0.4
    g, rest = S.flat_sheet(3, 2, L1, L2)
    q = rest.copy()
    q[:, 0] *= s1
    q[:, 1] *= s2
    q[:, 3] = s1
    q[:, 7] = s2
    lam = MAT.young * MAT.poisson / (1 - MAT.poisson ** 2)
    mu = MAT.young / (2 * (1 + MAT.poisson))
    A11, A22 = (s1 ** 2 - 1) / 2, (s2 ** 2 - 1) / 2
    want = L1 * L2 * MAT.thickness * (lam / 2 * (A11 + A22) ** 2 + mu * (A11 ** 2 + A22 ** 2))
    E, _ = _assembled_energy(g, rest, q)
    assert E == pytest.approx(want, rel=1e-13)


def test_energy_pure_bending_against_adaptive_quadrature():
    """Cylinder-like bending z = kappa xi1^2 / 2 on one patch: the 4x4 Gauss energy against an
    adaptive 1D quadrature of the exact integrand (Sec. 3.3 density; a11 = 1 + kappa^2 xi^2,
    b11 = kappa / sqrt(1 + kappa^2 xi^2))."""
    kappa, d1, d2 = 0.5, 0.1, 0.2
    mat = S.Material(1e5, 0.3, 2e-2, 200.0)
    q, qb = np.zeros(48), np.zeros(48)
    for qq in range(2):
        for p in range(2):
            c, x, y = p + 2 * qq, p * d1, qq * d2
            qb[c * 12:c * 12 + 12] = [x, y, 0, 1, 0, 0, 0, 1, 0, 0, 0, 0]
            q[c * 12:c * 12 + 12] = [x, y, kappa * x * x / 2, 1, 0, kappa * x, 0, 1, 0, 0, 0, 0]
    lam = mat.young * mat.poisson / (1 - mat.poisson ** 2)
    mu = mat.young / (2 * (1 + mat.poisson))
    h = mat.thickness

    def dens(x):
        A11 = kappa ** 2 * x ** 2 / 2
        B11 = 0.5 * kappa / math.sqrt(1 + kappa ** 2 * x ** 2)
        return (lam / 2 + mu) * (h * A11 ** 2 + h ** 3 / 3 * B11 ** 2)
    want = integrate.quad(dens, 0, d1, epsabs=0, epsrel=1e-13)[0] * d2
    got = O.element_energy(q, qb, d1, d2, mat)
    assert got == pytest.approx(want, rel=1e-9)


# --------------------------------------------------------------------------------------------
# App. B: gradient and Hessian
# --------------------------------------------------------------------------------------------
CASES = [
    ("sheet", lambda: S.flat_sheet(3, 2, 0.6, 0.5), 1e-3, 2e-2),
    ("sheet-thick", lambda: S.flat_sheet(2, 2), 0.5, 3e-2),
    ("annulus", lambda: S.annulus(10, 3), 1e-3, 1e-2),
    ("annulus-thick", lambda: S.annulus(10, 3), 0.3, 2e-2),
]


@pytest.mark.parametrize("name,build,h,sigma", CASES)
def test_gradient_and_hessian_match_exact_ad(name, build, h, sigma):
    """App. B's closed forms against second-order forward AD of the Sec. 3.3 energy."""
    g, rest = build()
    mat = S.Material(1e5, 0.3, h, 200.0)
    q = S.noisy(rest, sigma, 17)
    for p in (0, g.n_patches - 1):
        q48, qb48 = O.gather(g, q, p), O.gather(g, rest, p)
        E, G, H = O.element_egh(q48, qb48, g.dxi1, g.dxi2, mat)
        J = energy_jet(q48, qb48, g.dxi1, g.dxi2, mat.young, mat.poisson, mat.thickness)
        assert E == pytest.approx(J.v, rel=1e-12)
        assert np.linalg.norm(G - J.g) <= 1e-12 * np.linalg.norm(J.g)
        assert np.linalg.norm(H - J.H) <= 1e-12 * np.linalg.norm(J.H)


def test_bending_hessian_terms_match_ad_in_isolation():
    """Bending-only check: subtract the membrane contribution (h -> h with bending scaled away)
    by differencing two thicknesses, so a dropped bending term cannot hide under membrane."""
    g, rest = S.annulus(10, 3)
    q = S.noisy(rest, 2e-2, 5)
    q48, qb48 = O.gather(g, q, 7), O.gather(g, rest, 7)

    def parts(h):
        mat = S.Material(1e5, 0.3, h, 200.0)
        _, G, H = O.element_egh(q48, qb48, g.dxi1, g.dxi2, mat)
        J = energy_jet(q48, qb48, g.dxi1, g.dxi2, 1e5, 0.3, h)
        return G, H, J.g, J.H
    # energy = h M(q) + h^3/12 Bn(q): eliminate M with h and 2h
    G1, H1, JG1, JH1 = parts(0.1)
    G2, H2, JG2, JH2 = parts(0.2)
    Hb, JHb = H2 - 2 * H1, JH2 - 2 * JH1
    Gb, JGb = G2 - 2 * G1, JG2 - 2 * JG1
    assert np.linalg.norm(Hb - JHb) <= 1e-9 * np.linalg.norm(JHb)
    assert np.linalg.norm(Gb - JGb) <= 1e-9 * np.linalg.norm(JGb)


@pytest.mark.parametrize("name,build,h,sigma", CASES)
def test_pseudo_hessian_matches_gauss_newton_ad(name, build, h, sigma):
    """The pseudo Hessian (App. B, "The pseudo Hessian": the exact one without the second
    derivatives of beta) against AD of the energy with the bending strain linearised at q: the
    membrane Hessian plus the Gauss-Newton bending term. Energy and gradient are unchanged."""
    g, rest = build()
    mat = S.Material(1e5, 0.3, h, 200.0)
    q = S.noisy(rest, sigma, 19)
    for p in (0, g.n_patches - 1):
        q48, qb48 = O.gather(g, q, p), O.gather(g, rest, p)
        E, G, Hp = O.element_egh(q48, qb48, g.dxi1, g.dxi2, mat, pseudo=True)
        _, _, He = O.element_egh(q48, qb48, g.dxi1, g.dxi2, mat)
        J = energy_jet(q48, qb48, g.dxi1, g.dxi2, mat.young, mat.poisson, mat.thickness, pseudo=True)
        assert E == pytest.approx(J.v, rel=1e-12)
        assert np.linalg.norm(G - J.g) <= 1e-12 * np.linalg.norm(J.g)
        assert np.linalg.norm(Hp - J.H) <= 1e-12 * np.linalg.norm(J.H)
        # the dropped term is present in this bent state (not a vacuous comparison)
        assert np.linalg.norm(He - Hp) > 1e-8 * np.linalg.norm(He)


def test_pseudo_hessian_equals_exact_without_bending_strain():
    """Where beta = 0 (H beta = 0) the dropped term vanishes: the curved rest state of the annulus
    and a uniform in-plane stretch of a flat sheet."""
    mat = S.Material(1e5, 0.3, 0.05, 200.0)
    g, rest = S.annulus(10, 3)
    for p in (0, 13):
        qb48 = O.gather(g, rest, p)
        _, _, He = O.element_egh(qb48, qb48, g.dxi1, g.dxi2, mat)
        _, _, Hp = O.element_egh(qb48, qb48, g.dxi1, g.dxi2, mat, pseudo=True)
        assert np.linalg.norm(He - Hp) <= 1e-13 * np.linalg.norm(He)
    g, rest = S.flat_sheet(2, 2)
    q = rest.reshape(-1, 12).copy()
    q[:, 0] *= 1.1                                    # x -> 1.1 x, y -> 0.95 y: membrane strain only
    q[:, 1] *= 0.95
    q[:, 3] *= 1.1
    q[:, 7] *= 0.95
    q48, qb48 = O.gather(g, q, 3), O.gather(g, rest, 3)
    _, _, He = O.element_egh(q48, qb48, g.dxi1, g.dxi2, mat)
    _, _, Hp = O.element_egh(q48, qb48, g.dxi1, g.dxi2, mat, pseudo=True)
    assert np.linalg.norm(He - Hp) <= 1e-13 * np.linalg.norm(He)


def test_gradient_and_hessian_central_differences():
    g, rest = S.flat_sheet(2, 2)
    mat = S.Material(1e5, 0.3, 0.05, 200.0)
    q = S.noisy(rest, 2e-2, 9)
    q48, qb48 = O.gather(g, q, 2), O.gather(g, rest, 2)
    E, G, H = O.element_egh(q48, qb48, g.dxi1, g.dxi2, mat)
    e = 1e-6
    Gfd, Hfd = np.zeros(48), np.zeros((48, 48))
    for i in range(48):
        qp, qm = q48.copy(), q48.copy()
        qp[i] += e
        qm[i] -= e
        Gfd[i] = (O.element_energy(qp, qb48, g.dxi1, g.dxi2, mat) - O.element_energy(qm, qb48, g.dxi1, g.dxi2, mat)) / (2 * e)
        Hfd[:, i] = (O.element_egh(qp, qb48, g.dxi1, g.dxi2, mat)[1] - O.element_egh(qm, qb48, g.dxi1, g.dxi2, mat)[1]) / (2 * e)
    assert np.linalg.norm(G - Gfd) <= 1e-7 * np.linalg.norm(G)
    assert np.linalg.norm(H - Hfd) <= 1e-7 * np.linalg.norm(H)


def test_hessian_symmetric_and_rigid_modes_in_null_space_at_rest():
    g, rest = S.annulus(6, 2)
    for p in (0, 4):
        q48 = O.gather(g, rest, p)
        _, _, H = O.element_egh(q48, q48, g.dxi1, g.dxi2, MAT)
        assert np.linalg.norm(H - H.T) <= 1e-14 * np.linalg.norm(H)
        Q = q48.reshape(16, 3)
        modes = []
        for c in range(3):   # translations: only value DOFs move
            t = np.zeros((16, 3))
            t[0::4, c] = 1.0
            modes.append(t.ravel())
        for axis in np.eye(3):   # infinitesimal rotations act on every 3-vector
            modes.append(np.cross(axis, Q).ravel())
        for v in modes:
            assert np.linalg.norm(H @ v) <= 1e-12 * np.linalg.norm(H) * np.linalg.norm(v)
        # flat rest: exactly 6 zero eigenvalues is not claimed (bending has more); check PSD
        ev = np.linalg.eigvalsh(H)
        assert ev.min() >= -1e-10 * ev.max()


# --------------------------------------------------------------------------------------------
# Sec. 4.3: mass and gravity
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("build,area", [(lambda: S.flat_sheet(4, 3, 0.8, 0.6), 0.48),
                                        (lambda: S.flat_sheet(1, 1, 0.3, 0.2), 0.06)])
def test_mass_partition_of_unity_and_psd(build, area):
    g, rest = build()
    pat = O.bsr_pattern(g)
    mval, fs = O.mass(g, MAT, rest, pat)
    rho_h = MAT.density * MAT.thickness
    M = O.bsr_to_dense(pat[0], pat[1], mval)          # [n*4, n*4] scalar
    pos = np.zeros(g.n_nodes * 4)
    pos[0::4] = 1.0
    assert pos @ M @ pos == pytest.approx(rho_h * area, rel=1e-13)
    assert fs[:, 0].sum() == pytest.approx(rho_h * area, rel=1e-13)
    assert np.allclose(M @ pos, fs.ravel(), rtol=1e-12, atol=1e-18)   # M 1_pos = F/g
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > -1e-15 * ev.max()


def test_mass_annulus_area():
    """Annulus area from the Hermite-interpolated rest midsurface (polar map; not exactly
    pi (r1^2 - r0^2) because the interpolant is only cubic in the angle)."""
    g, rest = S.annulus(64, 4, 0.2, 0.7)
    mval, fs = O.mass(g, MAT, rest)
    area = fs[:, 0].sum() / (MAT.density * MAT.thickness)
    assert area == pytest.approx(math.pi * (0.7 ** 2 - 0.2 ** 2), rel=1e-6)


# --------------------------------------------------------------------------------------------
# BSR pattern and printed counts (Sec. 7, Table 2)
# --------------------------------------------------------------------------------------------
def test_dof_counts_and_twisting_nnz():
    for row in GOLD["dofs"]["value"]:
        nu, nv = row["patches"]
        g = S.annulus(nu, nv)[0] if row.get("periodic_u") else S.flat_sheet(nu, nv)[0]
        if "dofs" in row:
            assert g.n_dof == row["dofs"]
        else:
            assert round(g.n_dof, -2) == row["dofs_rounded"]
    g, _ = S.flat_sheet(30, 30)
    row_ptr, col = O.bsr_pattern(g)
    nnz = col.size * 144
    assert nnz == (3 * 30 + 1) ** 2 * 144 == 1192464
    assert float(f"{nnz:.2e}") == GOLD["nnz_twisting"]["value"]


def test_bsr_pattern_structure():
    for g in (S.flat_sheet(5, 4)[0], S.annulus(7, 3)[0]):
        row_ptr, col = O.bsr_pattern(g)
        assert np.all(np.diff(row_ptr) <= 9)
        for i in range(g.n_nodes):
            cols = col[row_ptr[i]:row_ptr[i + 1]]
            assert np.all(np.diff(cols) > 0) and i in cols
        # symmetric pattern
        pairs = {(i, j) for i in range(g.n_nodes) for j in col[row_ptr[i]:row_ptr[i + 1]]}
        assert all((j, i) in pairs for i, j in pairs)


def test_assembled_equals_sum_of_elements():
    g, rest = S.annulus(5, 2)
    q = S.noisy(rest, 1e-2, 2)
    pat = O.bsr_pattern(g)
    E, grad, (rp, col, val) = O.assemble(g, MAT, rest, q, mass_scale=3.0, pattern=pat)
    mval, _ = O.mass(g, MAT, rest, pat)
    Ke = np.zeros((g.n_dof, g.n_dof))
    ge = np.zeros(g.n_dof)
    Ee = 0.0
    for p in range(g.n_patches):
        e, gg, H = O.element_egh(O.gather(g, q, p), O.gather(g, rest, p), g.dxi1, g.dxi2, MAT)
        idx = np.concatenate([np.arange(n * 12, n * 12 + 12) for n in O.patch_nodes(g, p)])
        Ke[np.ix_(idx, idx)] += H
        ge[idx] += gg
        Ee += e
    Md = np.kron(O.bsr_to_dense(rp, col, mval), np.eye(3))
    # reorder M from (node, kind, comp) scalar-kron layout
    assert E == pytest.approx(Ee, rel=1e-13)
    assert np.allclose(grad, ge, rtol=1e-12, atol=1e-14)
    A = O.bsr_to_dense(rp, col, val)
    assert np.allclose(A, Ke + 3.0 * Md, rtol=1e-12, atol=1e-12 * np.abs(Ke).max())


# --------------------------------------------------------------------------------------------
# Sec. 6.1: PCG, Newton, implicit Euler
# --------------------------------------------------------------------------------------------
def test_pcg_matches_dense_solve():
    g, rest = S.flat_sheet(3, 3)
    q = S.noisy(rest, 1e-3, 4)
    _, grad, (rp, col, val) = O.assemble(g, MAT, rest, q, mass_scale=1e6)
    mask = S.pinned_mask(g, [0, g.n_nodes - 1])
    A = O.bsr_to_dense(rp, col, val)
    free = mask == 0
    b = -grad
    x, it, st = O.pcg(rp, col, val, b, mask=mask, rtol=1e-13, max_iter=5000)
    assert st == 0
    xd = np.zeros_like(b)
    xd[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert np.all(x[~free] == 0.0)


def test_pcg_detects_negative_curvature():
    g, rest = S.flat_sheet(2, 2)
    _, grad, (rp, col, val) = O.assemble(g, MAT, rest, S.noisy(rest, 1e-3, 4), mass_scale=1e6)
    x, it, st = O.pcg(rp, col, -val, np.ones(g.n_dof), rtol=1e-10)
    assert st == 100


def test_newton_free_fall_is_exact():
    """Rest sheet, no constraints, gravity: the implicit-Euler solution is a rigid translation,
    v^{n} = n dt g on position DOFs and 0 on derivative DOFs, one Newton iteration per step."""
    g, rest = S.flat_sheet(3, 2, 0.6, 0.4)
    q, v = rest.ravel().copy(), np.zeros(g.n_dof)
    P = O.step_params(dt=1e-2, gravity=(0.0, 0.0, -9.81), pcg_rtol=1e-14, pcg_max=5000)
    for n in range(1, 4):
        q, v, st = O.newton_step(g, MAT, rest, q, v, P)
        assert st["status"] == 0 and st["newton_iters"] == 1
        V = v.reshape(-1, 12)
        assert np.allclose(V[:, 2], -9.81 * 1e-2 * n, rtol=1e-9)
        assert np.abs(V[:, [0, 1]]).max() < 1e-9 and np.abs(V[:, 3:]).max() < 1e-9


def test_newton_affine_patch_test():
    """All boundary nodes prescribed (positions and derivatives) by a uniform stretch, interior
    perturbed, no gravity, inertia negligible: Newton returns the affine state and its
    closed-form energy."""
    s1, s2 = 1.08, 1.05
    g, rest = S.flat_sheet(4, 4)
    aff = rest.copy()
    aff[:, 0] *= s1
    aff[:, 1] *= s2
    aff[:, 3] = s1
    aff[:, 7] = s2
    bnd = [j * g.n1 + i for j in range(g.n2) for i in range(g.n1)
           if i in (0, g.n1 - 1) or j in (0, g.n2 - 1)]
    mask = S.pinned_mask(g, bnd, kinds=(0, 1, 2, 3))
    q0 = aff.copy()
    rng = np.random.default_rng(0)
    interior = [n for n in range(g.n_nodes) if n not in bnd]
    q0[interior, 0:3] += rng.normal(0, 3e-3, size=(len(interior), 3))
    P = O.step_params(dt=1e3, gravity=(0.0, 0.0, 0.0), pcg_rtol=1e-12, pcg_max=5000)
    q, v, st = O.newton_step(g, MAT, rest, q0.ravel(), np.zeros(g.n_dof), P, mask=mask, qfix=aff.ravel())
    assert st["status"] == 0
    assert np.abs(q - aff.ravel()).max() < 1e-8
    lam = MAT.young * MAT.poisson / (1 - MAT.poisson ** 2)
    mu = MAT.young / (2 * (1 + MAT.poisson))
    A11, A22 = (s1 ** 2 - 1) / 2, (s2 ** 2 - 1) / 2
    want = MAT.thickness * (lam / 2 * (A11 + A22) ** 2 + mu * (A11 ** 2 + A22 ** 2))
    E, _ = _assembled_energy(g, rest, q)
    assert E == pytest.approx(want, rel=1e-9)


def test_newton_quadratic_convergence_with_exact_hessian():
    g, rest, q0 = S.sheet_noisy(4, sigma=1e-3, seed=1)
    mask = S.pinned_mask(g, S.corner_nodes(g)[::3])
    res = []
    for k in range(1, 5):
        P = O.step_params(dt=1e-3, pcg_rtol=1e-14, pcg_max=20000, newton_max=k, newton_rtol=1e-300)
        _, _, st = O.newton_step(g, MAT, rest, q0.ravel(), np.zeros(g.n_dof), P, mask=mask,
                                 qfix=q0.ravel())
        res.append(st["res_final"] / st["res0"])
    # r_{k+1} <~ C r_k^2 until roundoff: the rate improves each iteration
    assert res[1] < 1e-2 * res[0] or res[1] < 1e-12
    assert res[2] < res[1] ** 1.5 * 1e3 or res[2] < 1e-12


def test_newton_step_config1_converges():
    g, rest, q0 = S.sheet_noisy(10, 1e-3, 1)
    mask = S.pinned_mask(g, [S.corner_nodes(g)[0], S.corner_nodes(g)[3]])
    P = O.step_params(dt=1e-3)
    q, v, st = O.newton_step(g, MAT, rest, q0.ravel(), np.zeros(g.n_dof), P, mask=mask, qfix=q0.ravel())
    assert st["status"] == 0 and 1 <= st["newton_iters"] <= 20
    assert st["res_final"] <= 1e-8 * st["res0"]
