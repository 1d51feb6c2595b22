"""Pins of the oracle's Newton policies (Sec. 6.1): the backtracking line search ("quadratic and
cubic line searches") and the diagonal regulariser ("a diagonal regularizer is added to make the
matrix positive definite"). The paper gives neither formulas nor constants; the readings pinned
here are: Armijo (c1 = 1e-4) from alpha = 1, the quadratic then the cubic interpolant's minimiser
(Nocedal-Wright Sec. 3.5) clamped to [0.1, 0.5] of the last trial; every free diagonal entry
A_ii <= 0 replaced by max(-A_ii, 1e-8 D_k); tau from a tenth of the previous iteration's tau,
times 10 per negative curvature, beyond 1e4 a failure. Each expected value below is a closed
form written from those definitions, not a re-call of the oracle."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

MAT = S.SHEET_MATERIAL
ARMIJO = 1e-4


# --------------------------------------------------------------------------------------------
# Line search
# --------------------------------------------------------------------------------------------
def test_first_backtrack_is_the_exact_minimiser_of_a_quadratic():
    """phi(a) = gd a + c a^2 / 2 fails Armijo at a = 1 when its minimiser a* = -gd / c < ~0.5;
    the quadratic model through phi(0), phi'(0), phi(1) is phi itself, so the first backtrack is
    a* and a* passes Armijo (phi(a*) = gd a* / 2)."""
    for gd, c in ((-1.0, 3.0), (-2.5, 9.0), (-1e-3, 4e-3)):
        astar = -gd / c
        alpha, bt, tried = O.line_search(gd, lambda a: gd * a + 0.5 * c * a * a)
        assert bt == 1 and tried[0] == 1.0
        assert alpha == pytest.approx(astar, rel=1e-14)


def test_second_backtrack_is_the_minimiser_of_the_cubic():
    """phi(a) = -a + 4 a^2 - 2.5 a^3: a = 1 fails, the quadratic step 1/3 fails, and the cubic
    through phi(0), phi'(0), phi(1), phi(1/3) is phi itself, so the third trial is phi's local
    minimiser (-4 + sqrt(16 - 7.5)) / -7.5, which passes."""
    phi = lambda a: -a + 4 * a * a - 2.5 * a ** 3
    alpha, bt, tried = O.line_search(-1.0, phi)
    assert bt == 2
    assert tried[1] == pytest.approx(1.0 / 3.0, rel=1e-14)
    want = (-4.0 + math.sqrt(16.0 - 7.5)) / -7.5
    assert alpha == pytest.approx(want, rel=1e-12)
    assert 3.0 * -2.5 * alpha ** 2 + 8.0 * alpha - 1.0 == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("trial,alpha,phi,gd,a_prev,f_prev,want", [
    (0, 1.0, 100.0, -1.0, 0.0, 0.0, 0.1),        # quadratic minimiser 1/202 clamped up to 0.1 alpha
    (0, 1.0, -0.5e-4, -1.0, 0.0, 0.0, 0.5),      # quadratic minimiser 0.500025 clamped down
    (0, 0.8, float("nan"), -1.0, 0.0, 0.0, 0.4),  # non-finite energy: halve
    (3, 0.2, float("inf"), -1.0, 0.4, 1.0, 0.1),
    (0, 0.5, 0.25, -2.0, 0.0, 0.0, 0.5 * 0.5 * 2.0 / (2.0 * (0.25 + 1.0))),
])
def test_next_trial_closed_forms_and_clamps(trial, alpha, phi, gd, a_prev, f_prev, want):
    assert O.ls_next_alpha(trial, alpha, phi, gd, a_prev, f_prev) == pytest.approx(want, rel=1e-14)


def test_cubic_with_no_real_minimiser_halves():
    """Trials of the cubic c a^3 + b a^2 + gd a with b = c = gd = -1: the fitted cubic is that
    cubic, whose derivative 3 c a^2 + 2 b a + gd has no real root (b^2 - 3 c gd = -2 < 0), so the
    step halves."""
    b, c, gd = -1.0, -1.0, -1.0
    a0, a1 = 1.0, 0.4
    f0 = c * a0 ** 3 + b * a0 ** 2 + gd * a0
    f1 = c * a1 ** 3 + b * a1 ** 2 + gd * a1
    assert O.ls_next_alpha(1, a1, f1, gd, a0, f0) == pytest.approx(0.5 * a1, rel=1e-14)


def test_accepted_step_satisfies_armijo_and_every_earlier_trial_fails_it():
    rng = np.random.default_rng(5)
    for _ in range(200):
        gd = -10 ** rng.uniform(-3, 1)
        k = rng.uniform(0.5, 40.0) * -gd
        w = rng.uniform(1.0, 30.0)
        amp = rng.uniform(0.0, 2.0) * -gd
        phi = lambda a: gd * a + 0.5 * k * a * a + amp * (1.0 - math.cos(w * a)) / w
        alpha, bt, tried = O.line_search(gd, phi)
        assert alpha is not None
        assert phi(alpha) <= ARMIJO * alpha * gd
        assert bt == len(tried) - 1
        for a in tried[:-1]:
            assert not (phi(a) <= ARMIJO * a * gd)
        for a0, a1 in zip(tried, tried[1:]):
            assert 0.1 * a0 * (1 - 1e-15) <= a1 <= 0.5 * a0 * (1 + 1e-15)


def test_line_search_gives_up_after_twenty_trials():
    alpha, bt, tried = O.line_search(-1.0, lambda a: 1.0 + a)
    assert alpha is None and bt == 20 and len(tried) == 20


# --------------------------------------------------------------------------------------------
# Regulariser
# --------------------------------------------------------------------------------------------
def _free_kind_means(rp, col, val, mask):
    n = rp.size - 1
    sums, cnt = np.zeros(4), np.zeros(4)
    for i in range(n):
        k = [kk for kk in range(rp[i], rp[i + 1]) if col[kk] == i][0]
        for a in range(12):
            if mask[i * 12 + a]:
                continue
            sums[a // 3] += abs(val[k, a, a])
            cnt[a // 3] += 1
    return np.where(cnt > 0, sums / np.maximum(cnt, 1), 1.0)


def test_local_fix_replaces_non_positive_free_diagonal_by_its_magnitude():
    g, rest = S.flat_sheet(2, 2)
    _, _, (rp, col, val) = O.assemble(g, MAT, rest, S.noisy(rest, 1e-3, 2), mass_scale=1e3)
    mask = S.pinned_mask(g, [4])
    val = val.copy()
    diag_k = [[kk for kk in range(rp[i], rp[i + 1]) if col[kk] == i][0] for i in range(g.n_nodes)]
    # plant non-positive entries: negative, zero, tiny negative, and one on a prescribed DOF
    plants = {(0, 1): -3.0 * val[diag_k[0], 1, 1], (2, 7): 0.0, (5, 10): -1e-30, (4, 0): -5.0}
    for (nd, a), v in plants.items():
        val[diag_k[nd], a, a] = v
    D = _free_kind_means(rp, col, val, mask)
    fixed, cnt = O.fix_diagonal(rp, col, val, mask)
    assert cnt == 3
    want = val.copy()
    for (nd, a), v in plants.items():
        if mask[nd * 12 + a]:
            continue
        want[diag_k[nd], a, a] = max(-v, 1e-8 * D[a // 3])
    assert np.array_equal(fixed, want)


def _coupled_pair(c):
    """Two nodes, A = [[I, c I], [c I, I]] (12x12 blocks): diagonal blocks SPD, eigenvalues
    1 - c and 1 + c, so A + tau I (D = 1 for every kind) is positive definite iff tau > c - 1."""
    rp = np.array([0, 2, 4], dtype=np.int32)
    col = np.array([0, 1, 0, 1], dtype=np.int32)
    I = np.eye(12)
    val = np.stack([I, c * I, c * I, I])
    e = np.linspace(1.0, 2.0, 12)
    rhs = np.concatenate([e, -e])   # the eigenvector of eigenvalue 1 - c
    return rp, col, val, rhs


def test_regulariser_ladder_climbs_by_ten_from_zero():
    """c = 1.5: every solve with tau < 0.5 meets p^T A p < 0 at its first iteration (rhs is the
    negative eigenvector); the ladder 0, 1e-8, ..., 1e-1 fails, tau = 1 succeeds, with 9 shifted
    solves, and d = rhs / (1 + 1 - 1.5)."""
    rp, col, val, rhs = _coupled_pair(1.5)
    d, st, tau, it, regs, fixes = O.newton_direction(rp, col, val, rhs, rtol=1e-12)
    assert st == 0 and fixes == 0
    assert tau == pytest.approx(1.0, rel=1e-12)
    assert regs == 9 and it == 1
    assert np.allclose(d, rhs / 0.5, rtol=1e-12)


@pytest.mark.parametrize("carry,start_regs", [(1.0, 2), (1e-7, 9), (5e-8, 9), (30.0, 1)])
def test_regulariser_starts_at_a_tenth_of_the_carried_tau(carry, start_regs):
    """carry 1 -> start 0.1 (fails) -> 1: 2 shifted solves; carry 1e-7 -> start 1e-8: 9 shifted
    solves; carry 5e-8 -> a tenth is below 1e-8, start at 0 (unshifted) -> 9 shifted solves;
    carry 30 -> start 3 passes at once."""
    rp, col, val, rhs = _coupled_pair(1.5)
    d, st, tau, it, regs, fixes = O.newton_direction(rp, col, val, rhs, tau_carry=carry, rtol=1e-12)
    assert st == 0 and regs == start_regs
    want_tau = 3.0 if carry == 30.0 else 1.0
    assert tau == pytest.approx(want_tau, rel=1e-12)
    assert np.allclose(d, rhs / (2.0 + want_tau - 1.5 - 1.0), rtol=1e-12)


def test_regulariser_gives_up_beyond_1e4():
    rp, col, val, rhs = _coupled_pair(1e5 + 1.0)
    d, st, tau, it, regs, fixes = O.newton_direction(rp, col, val, rhs, rtol=1e-12)
    assert st == 8   # OG_ERR_INDEFINITE: tau = 1e4 still meets negative curvature
    assert regs == 13   # 1e-8 .. 1e4


def test_non_spd_block_falls_back_to_the_inverse_of_its_diagonal():
    """One node whose 12x12 block has a positive diagonal but is indefinite: the preconditioner is
    diag(1/A_ii), so one fixed PCG iteration from 0 gives x = (r.z / z.A z) z with z = r / diag."""
    rng = np.random.default_rng(3)
    dg = np.linspace(1.0, 3.0, 12)
    A = np.diag(dg)
    A[0, 5] = A[5, 0] = 4.0   # 1 * 2.09 < 16: the block is not positive definite
    assert np.linalg.eigvalsh(A).min() < 0
    rp = np.array([0, 1], dtype=np.int32)
    col = np.array([0], dtype=np.int32)
    b = rng.normal(size=12)
    x, it, st = O.pcg(rp, col, A[None], b, fixed_iters=1)
    z = b / dg
    pAp = z @ A @ z
    assert pAp > 0 and it == 1
    assert np.allclose(x, (b @ z) / pAp * z, rtol=1e-13)


# --------------------------------------------------------------------------------------------
# Newton with the regulariser
# --------------------------------------------------------------------------------------------
def test_in_plane_twist_keeps_the_sheet_planar_and_converges_quadratically():
    """A flat sheet twisted about its normal stays in its plane (the energy is even in the normal
    displacement and nothing breaks the symmetry), while compression can make normal diagonal
    entries negative. The local fix leaves the in-plane DOFs unshifted: each step converges in a
    few Newton iterations with no shifted solve, and the normal components stay exactly 0."""
    g, rest = S.flat_sheet(10, 10)
    q, v = rest.ravel().copy(), np.zeros(g.n_dof)
    P = O.step_params(dt=2e-3, gravity=(0.0, 0.0, 0.0), newton_max=30)
    fixes = 0
    for k in range(1, 21):
        mask, qfix = S.twist_prescription(g, rest, k, deg_per_step=8.0)
        q, v, st = O.newton_step(g, MAT, rest, q, v, P, mask=mask, qfix=qfix)
        assert st["status"] == 0 and st["newton_iters"] <= 4, (k, st)
        assert st["regularizations"] == 0
        fixes += st["diag_fixes"]
        Q = q.reshape(-1, 12)
        assert np.all(Q[:, 2::3] == 0.0)
    assert fixes > 0
