"""Direct solver comparator (Sec. 6.1's LDL^T, here a banded FP64 Cholesky over the node rows of the
grid, hand-written kernels) for the Newton systems, against the block-Jacobi PCG path at a tight
tolerance and the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rollout(g, rest, q0, mask, P, solver, steps):
    from paper_2312_14839_gb300.bhem import Shell
    dev = "cuda"
    with Shell(g, S.SHEET_MATERIAL, torch.as_tensor(rest.reshape(-1), device=dev), precision="fp64",
               solver=solver) as sh:
        q = torch.as_tensor(q0.reshape(-1).copy(), device=dev)
        v = torch.zeros_like(q)
        m = torch.as_tensor(mask, device=dev)
        qf = q.clone()
        its = []
        for _ in range(steps):
            st = sh.newton_step(q, v, P, mask=m, q_fixed=qf)
            assert st["status"] == 0, st
            its.append((st["newton_iters"], st["regularizations"]))
        torch.cuda.synchronize()
        return q.cpu().numpy(), its


def test_config1_newton_iterations_match_pcg_and_oracle():
    """10 implicit-Euler steps of the 10 x 10 noisy sheet, corners (0,0), (1,1) pinned: the direct
    solve takes the same Newton iterations per step as PCG at eta = 1e-13 and as the FP64
    oracle at that tolerance, and ends in the same state (to 1e-9 of its size)."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest, q0 = S.sheet_noisy(10, 1e-3, 1)
    mask = S.pinned_mask(g, [0, g.n_nodes - 1])
    P = step_params(dt=1e-3, newton_rtol=1e-8, pcg_rtol=1e-13, pcg_max=5000)
    qd, itd = _rollout(g, rest, q0, mask, P, "direct", 10)
    qp, itp = _rollout(g, rest, q0, mask, P, "pcg", 10)
    assert [a for a, _ in itd] == [a for a, _ in itp], (itd, itp)
    assert np.linalg.norm(qd - qp) <= 1e-9 * np.linalg.norm(qp)
    # FP64 oracle (its own PCG at the same tolerance)
    q, v = q0.reshape(-1).copy(), np.zeros(g.n_dof)
    its_o = []
    for _ in range(10):
        q, v, so = O.newton_step(g, S.SHEET_MATERIAL, rest, q, v,
                                 O.step_params(dt=1e-3, newton_rtol=1e-8, pcg_rtol=1e-13, pcg_max=5000),
                                 mask=mask, qfix=q0.reshape(-1))
        its_o.append(so["newton_iters"])
    assert [a for a, _ in itd] == its_o
    assert np.linalg.norm(qd - q) <= 1e-9 * np.linalg.norm(q)


def test_indefinite_system_takes_the_regulariser_ladder():
    """A 6 x 6 sheet compressed in plane to 97% with its edges x = 0 and x = 1 held: the Hessian
    is indefinite, Cholesky fails, the regulariser grows tenfold until it succeeds, and the step
    still reaches the Newton tolerance."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest = S.flat_sheet(6, 6)
    q0 = rest.copy()
    q0[:, 0] *= 0.97
    q0[:, 3] *= 0.97
    rng = np.random.default_rng(2)
    q0[:, 2] += rng.normal(0.0, 1e-4, size=g.n_nodes)
    edge = [j * g.n1 for j in range(g.n2)] + [j * g.n1 + g.n1 - 1 for j in range(g.n2)]
    mask = S.pinned_mask(g, edge, kinds=(0, 1, 2, 3))
    P = step_params(dt=1e-2, gravity=(0.0, 0.0, 0.0), newton_rtol=1e-8, newton_max=100)
    _, its = _rollout(g, rest, q0, mask, P, "direct", 2)
    assert sum(r for _, r in its) >= 1


@pytest.mark.parametrize("name,make", [
    ("sheet12x4 (rows along u)", lambda: _rect_noisy(12, 4)),
    ("annulus16x3 (periodic rows)", lambda: _annulus_noisy(16, 3)),
])
def test_both_row_orientations_match_pcg(name, make):
    """The band runs along the narrower non-periodic direction: a 12 x 4 sheet is factorised by
    node columns, a periodic annulus by node rows that wrap around. Both give the Newton
    iterations and the state of PCG at eta = 1e-13."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest, q0 = make()
    mask = S.pinned_mask(g, [0])
    P = step_params(dt=1e-3, newton_rtol=1e-8, pcg_rtol=1e-13, pcg_max=20000)
    qd, itd = _rollout(g, rest, q0, mask, P, "direct", 3)
    qp, itp = _rollout(g, rest, q0, mask, P, "pcg", 3)
    assert [a for a, _ in itd] == [a for a, _ in itp], (itd, itp)
    assert np.linalg.norm(qd - qp) <= 1e-9 * np.linalg.norm(qp)


def _rect_noisy(nu, nv):
    g, rest = S.flat_sheet(nu, nv, 1.0, nv / nu)
    return g, rest, S.noisy(rest, 1e-3, 7)


def _annulus_noisy(nu, nv):
    g, rest = S.annulus(nu, nv)
    return g, rest, S.noisy(rest, 1e-3, 8)


def test_sheet_30x30_factorises_well_under_a_second():
    """The 30 x 30 noisy sheet under gravity, two corners pinned (11,532 DOF, the paper's 30 x 30
    scene size): the first implicit-Euler step with the banded direct solve takes the Newton
    iterations of PCG at eta = 1e-13 and of the FP64 oracle, and each factorisation of the step
    takes well under a second."""
    import time
    from paper_2312_14839_gb300.bhem import step_params
    g, rest, q0 = S.sheet_noisy(30, 1e-3, 1)
    mask = S.pinned_mask(g, [0, g.n_nodes - 1])
    P = step_params(dt=1e-3, newton_rtol=1e-8, newton_max=50, pcg_rtol=1e-13, pcg_max=20000)
    _rollout(g, rest, q0, mask, P, "direct", 1)   # first call: allocation
    t0 = time.perf_counter()
    qd, itd = _rollout(g, rest, q0, mask, P, "direct", 1)
    sec = time.perf_counter() - t0
    qp, itp = _rollout(g, rest, q0, mask, P, "pcg", 1)
    assert itd[0][0] == itp[0][0], (itd, itp)
    assert np.linalg.norm(qd - qp) <= 1e-8 * np.linalg.norm(qp)
    _, _, so = O.newton_step(g, S.SHEET_MATERIAL, rest, q0.reshape(-1), np.zeros(g.n_dof),
                             O.step_params(dt=1e-3, newton_rtol=1e-8, newton_max=50, pcg_rtol=1e-13,
                                           pcg_max=20000), mask=mask, qfix=q0.reshape(-1))
    assert itd[0][0] == so["newton_iters"]
    assert sec / max(1, sum(1 + r for _, r in itd)) < 0.5, sec


def test_direct_solver_rejects_unsupported_shells():
    """Rows of more than 4096 unknowns (a 350 x 350 sheet: 351 nodes per row either way) are
    rejected before any factorisation."""
    from paper_2312_14839_gb300.bhem import Shell, ShellError, step_params
    g, rest = S.flat_sheet(350, 350)
    with Shell(g, S.SHEET_MATERIAL, torch.as_tensor(rest.reshape(-1), device="cuda"), precision="fp64",
               solver="direct") as sh:
        q = torch.as_tensor(S.noisy(rest, 1e-3, 3).reshape(-1), device="cuda")
        v = torch.zeros_like(q)
        with pytest.raises(ShellError) as ei:
            sh.newton_step(q, v, step_params(dt=1e-3), raise_on_error=True)
        assert ei.value.status == 1


def test_direct_solver_rejects_a_grid_periodic_in_both_directions():
    """A torus (periodic in u and v) couples the first and last node rows in both directions, so
    no row ordering makes its matrix block tridiagonal: the direct step returns SHELL_ERR_ARG."""
    import math
    from paper_2312_14839_gb300.bhem import Shell, ShellError, step_params
    nu, nv, R, r = 12, 8, 0.5, 0.2
    g = S.Grid(nu, nv, True, True, 2 * math.pi / nu, 2 * math.pi / nv)
    rest = np.zeros((g.n_nodes, 12))
    for j in range(g.n2):
        for i in range(g.n1):
            th, ph = i * g.dxi1, j * g.dxi2
            rho = R + r * math.cos(ph)
            rest[j * g.n1 + i] = [rho * math.cos(th), rho * math.sin(th), r * math.sin(ph),
                                  -rho * math.sin(th), rho * math.cos(th), 0.0,
                                  -r * math.sin(ph) * math.cos(th), -r * math.sin(ph) * math.sin(th), r * math.cos(ph),
                                  r * math.sin(ph) * math.sin(th), -r * math.sin(ph) * math.cos(th), 0.0]
    with Shell(g, S.SHEET_MATERIAL, torch.as_tensor(rest.reshape(-1), device="cuda"), precision="fp64",
               solver="direct") as sh:
        q = torch.as_tensor(S.noisy(rest, 1e-3, 4).reshape(-1), device="cuda")
        v = torch.zeros_like(q)
        with pytest.raises(ShellError) as ei:
            sh.newton_step(q, v, step_params(dt=1e-3, gravity=(0.0, 0.0, 0.0)), raise_on_error=True)
        assert ei.value.status == 1
