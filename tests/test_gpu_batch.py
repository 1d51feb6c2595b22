"""Batched shells (shell_batch_*) against the FP64 oracle and against the single-shell solver:
every shell of a batch runs its own Newton to its own 1e-8 residual."""
import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_shells():
    """Uneven sizes and materials, flat sheets with pinned corners and a periodic annulus."""
    out = []
    specs = [(4, S.Material(1e5, 0.3, 1e-3, 200.0)), (7, S.Material(3e4, 0.3, 2e-3, 200.0)),
             (3, S.Material(1e6, 0.3, 5e-4, 200.0)), (10, S.Material(1e5, 0.3, 1e-3, 200.0))]
    for k, (n, mat) in enumerate(specs):
        g, rest = S.flat_sheet(n, n)
        q = S.noisy(rest, 1e-3, 20 + k)
        c = S.corner_nodes(g)
        mask = S.pinned_mask(g, [c[0], c[3]])
        out.append((g, mat, rest, q, mask))
    g, rest = S.annulus(8, 3)
    q = S.noisy(rest, 1e-3, 30)
    mask = S.pinned_mask(g, [0])
    out.append((g, S.Material(2e5, 0.4, 1e-3, 300.0), rest, q, mask))
    return out


def run_batch(shells, steps=1, autotune=False):
    from paper_2312_14839_gb300.bhem import Batch, step_params
    B = Batch([(g, m, r) for g, m, r, _, _ in shells])
    q = torch.as_tensor(np.concatenate([x[3].reshape(-1) for x in shells]), device="cuda")
    v = torch.zeros_like(q)
    mask = torch.as_tensor(np.concatenate([x[4] for x in shells]), device="cuda")
    qfix = q.clone()
    if autotune:
        B.autotune(q)
    P = step_params(dt=1e-3)
    hist = []
    for _ in range(steps):
        st = B.newton_step(q, v, P, mask=mask, q_fixed=qfix)
        hist.append((st, q.cpu().numpy().copy(), v.cpu().numpy().copy()))
    off = B.node_offsets.copy()
    B.close()
    return hist, off


def test_batch_matches_oracle_per_shell():
    shells = make_shells()
    hist, off = run_batch(shells, steps=2)
    Po = O.step_params(dt=1e-3)
    states = [(x[3].reshape(-1).copy(), np.zeros(x[0].n_dof)) for x in shells]
    for st, qb, vb in hist:
        for s, (g, mat, rest, q0, mask) in enumerate(shells):
            a, b = off[s] * 12, off[s + 1] * 12
            qo, vo, so = O.newton_step(g, mat, rest, states[s][0], states[s][1], Po, mask=mask, qfix=q0.reshape(-1))
            assert st[s]["status"] == 0 and so["status"] == 0
            assert abs(st[s]["newton_iters"] - so["newton_iters"]) <= 1, (s, st[s], so)
            assert st[s]["res_final"] <= 1e-8 * st[s]["res0"]
            assert rel(vb[a:b], vo) <= 1e-5, (s, rel(vb[a:b], vo))
            states[s] = (qb[a:b].copy(), vb[a:b].copy())   # continue the oracle from the GPU state


def test_batch_of_one_equals_shell_inside_batch():
    shells = make_shells()
    full, off = run_batch(shells, steps=1)
    for s in (1, 4):
        alone, _ = run_batch([shells[s]], steps=1)
        a, b = off[s] * 12, off[s + 1] * 12
        assert alone[0][0][0]["newton_iters"] == full[0][0][s]["newton_iters"]
        assert rel(alone[0][2], full[0][2][a:b]) <= 1e-6


def test_batch_matches_single_shell_solver():
    from paper_2312_14839_gb300.bhem import Shell, step_params
    shells = make_shells()
    hist, off = run_batch(shells, steps=1)
    for s, (g, mat, rest, q0, mask) in enumerate(shells):
        sh = Shell(g, mat, torch.as_tensor(rest.reshape(-1), device="cuda"), precision="mixed")
        q = torch.as_tensor(q0.reshape(-1), device="cuda")
        v = torch.zeros_like(q)
        st = sh.newton_step(q, v, step_params(dt=1e-3), mask=torch.as_tensor(mask, device="cuda"), q_fixed=q.clone())
        a, b = off[s] * 12, off[s + 1] * 12
        assert abs(st["newton_iters"] - hist[0][0][s]["newton_iters"]) <= 1
        assert rel(hist[0][2][a:b], v.cpu().numpy()) <= 1e-5


def test_autotune_keeps_results():
    shells = make_shells()
    base, off = run_batch(shells, steps=1)
    tuned, _ = run_batch(shells, steps=1, autotune=True)
    for s in range(len(shells)):
        assert abs(base[0][0][s]["newton_iters"] - tuned[0][0][s]["newton_iters"]) <= 1
    assert rel(tuned[0][2], base[0][2]) <= 1e-5
