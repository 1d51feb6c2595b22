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


def run_batch(shells, steps=1, autotune=False, assembly="atomic"):
    from paper_2312_14839_gb300.bhem import Batch, step_params
    B = Batch([(g, m, r) for g, m, r, _, _ in shells], assembly=assembly)
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


def test_graph_step_equals_host_driven_step(monkeypatch):
    """A batch step is one CUDA graph launch whose WHILE nodes take the host's loop decisions
    on the device; with BHEM_BATCH_HOST_LOOP set the same kernels run in the same order with the
    decisions taken on the host. The per-shell dot products are summed across CTAs with FP64
    atomics, whose order varies from run to run, so a PCG solve may stop one iteration apart:
    the two forms agree in status and Newton counts, PCG totals within one per Newton iteration,
    and the states to 1e-6, for two steps (the second replays the captured graph)."""
    shells = make_shells()
    monkeypatch.delenv("BHEM_BATCH_HOST_LOOP", raising=False)
    graph, off = run_batch(shells, steps=2)
    monkeypatch.setenv("BHEM_BATCH_HOST_LOOP", "1")
    host, _ = run_batch(shells, steps=2)
    for (sg, qg, vg), (sh_, qh, vh) in zip(graph, host):
        for s in range(len(shells)):
            for key in ("status", "newton_iters", "ls_backtracks", "regularizations", "diag_fixes"):
                assert sg[s][key] == sh_[s][key], (s, key, sg[s], sh_[s])
            assert abs(sg[s]["pcg_iters_total"] - sh_[s]["pcg_iters_total"]) <= sg[s]["newton_iters"]
        assert rel(qg, qh) <= 1e-6 and rel(vg, vh) <= 1e-6


def test_config4_sample_of_32_sheets_against_the_oracle():
    """32 seeded sheets of the 512-sheet recipe (n x n patches, n ~ U{4..40}, log10 E ~ U[4, 6],
    h ~ U[0.5, 2] mm, corners (0,0) and (1,1) pinned, gravity): one batched step (one graph
    launch) against the FP64 oracle sheet by sheet: every sheet converges to 1e-8, Newton counts
    agree to within one (FP32 Hessians), and the velocities agree to the solver's tolerance."""
    sheets = S.batch_sheets(512, seed=4)[::16]
    shells = []
    for g, mat, rest, q in sheets:
        c = S.corner_nodes(g)
        shells.append((g, mat, rest, q, S.pinned_mask(g, [c[0], c[3]])))
    assert len(shells) == 32 and len({g.nu for g, *_ in shells}) > 10
    hist, off = run_batch(shells, steps=1)
    st, qb, vb = hist[0]
    Po = O.step_params(dt=1e-3)
    for s, (g, mat, rest, q0, mask) in enumerate(shells):
        a, b = off[s] * 12, off[s + 1] * 12
        qo, vo, so = O.newton_step(g, mat, rest, q0.reshape(-1), np.zeros(g.n_dof), Po, mask=mask,
                                   qfix=q0.reshape(-1))
        assert st[s]["status"] == 0 and so["status"] == 0, (s, g.nu, st[s], so)
        assert abs(st[s]["newton_iters"] - so["newton_iters"]) <= 1, (s, g.nu, st[s], so)
        assert st[s]["res_final"] <= 1e-8 * st[s]["res0"]
        assert rel(vb[a:b], vo) <= 1e-5, (s, g.nu, rel(vb[a:b], vo))


def test_colour_assembly_on_odd_periodic_grids_equals_atomic():
    """Annuli periodic in u with 7 and 13 patches around (1 mod 3, where a pu mod 3 colouring put
    the seam patch and patch 0 on one colour) and 5 (2 mod 3), stepped with colour-ordered
    assembly (plain writes, one launch per colour) and with atomic assembly: the same Newton
    counts and the same states to the rounding of the atomic sums."""
    shells = []
    for k, nu in enumerate((7, 13, 5)):
        g, rest = S.annulus(nu, 3)
        q = S.noisy(rest, 1e-3, 40 + k)
        shells.append((g, S.Material(1e5, 0.3, 1e-3, 200.0), rest, q, S.pinned_mask(g, [0])))
    col, off = run_batch(shells, steps=2, assembly="color")
    ato, _ = run_batch(shells, steps=2, assembly="atomic")
    for (sc, qc, vc), (sa, qa, va) in zip(col, ato):
        for s in range(len(shells)):
            assert sc[s]["status"] == sa[s]["status"] == 0
            assert sc[s]["newton_iters"] == sa[s]["newton_iters"], (s, sc[s], sa[s])
        assert rel(qc, qa) <= 1e-6 and rel(vc, va) <= 1e-5
