"""Direct solver comparator (Sec. 6.1's LDL^T, here a dense FP64 Cholesky through cuSOLVER) for
the Newton systems, against the block-Jacobi PCG path at a tight tolerance and the FP64 oracle."""
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


def test_direct_solver_rejects_large_shells():
    from paper_2312_14839_gb300.bhem import Shell, ShellError, step_params
    g, rest, q0 = S.sheet_sinusoid(80, 3)   # 6,561 nodes, 78,732 DOF
    with Shell(g, S.SHEET_MATERIAL, torch.as_tensor(rest.reshape(-1), device="cuda"), precision="fp64",
               solver="direct") as sh:
        q = torch.as_tensor(q0.reshape(-1).copy(), device="cuda")
        v = torch.zeros_like(q)
        with pytest.raises(ShellError):
            sh.newton_step(q, v, step_params(dt=1e-3), raise_on_error=True)
