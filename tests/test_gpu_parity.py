"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

Tolerances (normwise relative, per patch / per quantity): <= 1e-11 for FP64 results, <= 1e-5 for
FP32 element quantities; index work (BSR pattern) bit-exact; Newton iteration counts identical
for the FP64 path.
"""
import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "mixed": 1e-5}


def dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def make_shell(g, mat, rest, **kw):
    from paper_2312_14839_gb300.bhem import Shell
    return Shell(g, mat, dev(rest.reshape(-1)), **kw)


THIN = S.SHEET_MATERIAL
THICK = S.Material(1e5, 0.3, 0.05, 200.0)

CASES = {
    "sheet10x10-noisy": lambda: (*S.sheet_noisy(10, 1e-3, 1), THIN),
    "sheet1x1": lambda: (*S.sheet_noisy(1, 1e-2, 2), THIN),
    "sheet3x2-rect-thick": lambda: (lambda g, r: (g, r, S.noisy(r, 2e-2, 3), THICK))(*S.flat_sheet(3, 2, 0.6, 0.4)),
    "annulus12x3": lambda: (lambda g, r: (g, r, S.noisy(r, 1e-2, 4), THIN))(*S.annulus(12, 3)),
    "annulus7x2-odd-thick": lambda: (lambda g, r: (g, r, S.noisy(r, 1e-2, 5), THICK))(*S.annulus(7, 2)),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_element_parity(case, prec):
    g, rest, q, mat = CASES[case]()
    E0, G0, H0 = O.elements(g, mat, rest, q)
    sh = make_shell(g, mat, rest, precision=prec)
    E, G, H = sh.element_egh(dev(q.reshape(-1)), precision=prec)
    torch.cuda.synchronize()
    E, G, H = host(E), host(G), host(H)
    tol = TOL[prec]
    assert np.abs(E - E0).max() <= tol * np.abs(E0).sum()
    for p in range(g.n_patches):
        assert rel(G[p], G0[p]) <= tol, (p, rel(G[p], G0[p]))
        assert rel(H[p], H0[p]) <= tol, (p, rel(H[p], H0[p]))
        assert np.abs(H[p] - H[p].T).max() <= tol * np.abs(H0[p]).max() * 4


@pytest.mark.parametrize("case", ["sheet3x2-rect-thick", "annulus7x2-odd-thick"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_pseudo_hessian_element_parity(case, prec):
    """The pseudo Hessian (App. B: without the second derivatives of beta) against the oracle's."""
    g, rest, q, mat = CASES[case]()
    E0, G0, H0 = O.elements(g, mat, rest, q, pseudo=True)
    _, _, Hx = O.elements(g, mat, rest, q)
    sh = make_shell(g, mat, rest, precision=prec, hessian="pseudo")
    E, G, H = sh.element_egh(dev(q.reshape(-1)), precision=prec)
    torch.cuda.synchronize()
    E, G, H = host(E), host(G), host(H)
    tol = TOL[prec]
    assert np.abs(E - E0).max() <= tol * np.abs(E0).sum()
    for p in range(g.n_patches):
        assert rel(G[p], G0[p]) <= tol, (p, rel(G[p], G0[p]))
        assert rel(H[p], H0[p]) <= tol, (p, rel(H[p], H0[p]))
    # the case has bending strain: the pseudo Hessian differs from the exact one beyond tolerance
    assert max(rel(H0[p], Hx[p]) for p in range(g.n_patches)) > 100 * tol


def test_newton_pseudo_hessian_fp64_identical_iteration_counts():
    """Implicit-Euler steps with the pseudo Hessian: FP64 GPU against the oracle, same counts."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest, q0 = S.sheet_noisy(6, 2e-2, 3)
    mat = S.Material(1e5, 0.3, 0.01, 200.0)
    c = S.corner_nodes(g)
    mask = S.pinned_mask(g, [c[0], c[3]])
    qfix = q0.reshape(-1).copy()
    sh = make_shell(g, mat, rest, precision="fp64", hessian="pseudo")
    P = step_params(dt=1e-2)
    Po = O.step_params(dt=1e-2, pseudo_hessian=True)
    q, v = dev(q0.reshape(-1)), torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    qo, vo = q0.reshape(-1).copy(), np.zeros(g.n_dof)
    for _ in range(3):
        st = sh.newton_step(q, v, P, mask=dev(mask, torch.uint8), q_fixed=dev(qfix))
        qo, vo, so = O.newton_step(g, mat, rest, qo, vo, Po, mask=mask, qfix=qfix)
        assert st["status"] == 0 and so["status"] == 0
        assert st["newton_iters"] == so["newton_iters"], (st, so)
        assert rel(host(q), qo) <= 1e-11


@pytest.mark.parametrize("case", ["sheet10x10-noisy", "annulus12x3", "annulus7x2-odd-thick", "sheet1x1"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("assembly", ["atomic", "color"])
def test_assembled_parity(case, prec, assembly):
    g, rest, q, mat = CASES[case]()
    ms = 1e6
    pat = O.bsr_pattern(g)
    E0, g0, (rp0, col0, val0) = O.assemble(g, mat, rest, q, mass_scale=ms, pattern=pat)
    sh = make_shell(g, mat, rest, precision=prec, assembly=assembly)
    E, G = sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=ms)
    rp, col, val = sh.bsr()
    torch.cuda.synchronize()
    assert np.array_equal(host(rp).astype(np.int64), rp0) and np.array_equal(host(col).astype(np.int64), col0)
    # energy and gradient are FP64 in both precisions
    assert abs(host(E)[0] - E0) <= 1e-11 * abs(E0)
    assert rel(host(G), g0) <= 1e-11
    val = host(val)
    assert rel(val, val0) <= TOL[prec]
    for i in range(g.n_nodes):   # every block row
        a, b = rp0[i], rp0[i + 1]
        assert rel(val[a:b], val0[a:b]) <= TOL[prec] * 4, i


@pytest.mark.parametrize("case", ["sheet10x10-noisy", "annulus7x2-odd-thick"])
def test_mass_and_gravity_parity(case):
    g, rest, q, mat = CASES[case]()
    M0, F0 = O.mass(g, mat, rest)
    sh = make_shell(g, mat, rest)
    M, F = sh.mass()
    torch.cuda.synchronize()
    assert rel(host(M), M0) <= 1e-13
    assert rel(host(F), F0) <= 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_spmv_matches_dense_product(prec):
    g, rest, q, mat = CASES["annulus12x3"]()
    sh = make_shell(g, mat, rest, precision=prec)
    sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=1e6)
    rp, col, val = sh.bsr()
    A = O.bsr_to_dense(host(rp).astype(np.int64), host(col).astype(np.int64), host(val))
    x = np.random.default_rng(0).normal(size=g.n_dof)
    y = host(sh.spmv(dev(x)))
    assert rel(y, A @ x) <= (1e-13 if prec == "fp64" else 1e-5)
    if prec == "mixed":   # FP32 input: the single-launch form
        x32 = x.astype(np.float32)
        y32 = host(sh.spmv(dev(x32, torch.float32)))
        assert rel(y32, A @ x32.astype(np.float64)) <= 1e-5


SPMV_GRIDS = {
    "annulus12x3": lambda: CASES["annulus12x3"](),
    "sheet1x1": lambda: CASES["sheet1x1"](),
    "sheet3x2": lambda: CASES["sheet3x2-rect-thick"](),
    "sheet61x37": lambda: (lambda g, r: (g, r, S.noisy(r, 1e-2, 9), THIN))(*S.flat_sheet(61, 37)),
    "sheet256-sinusoid": lambda: (*S.sheet_sinusoid(256, 3), THIN),
}


@pytest.mark.parametrize("case", list(SPMV_GRIDS))
def test_spmv_tma_identical_to_plain(case, monkeypatch):
    """The TMA-pipelined FP32 SpMV computes every row with the arithmetic and order of the plain
    kernel that streams both triangles (BHEM_SPMV_SYM=0): outputs are bit-identical (empty tail
    groups, one-group grids, full size). The matrices come from the colour-ordered assembly,
    which is deterministic."""
    monkeypatch.setenv("BHEM_SPMV_SYM", "0")
    g, rest, q, mat = SPMV_GRIDS[case]()
    ys = []
    x32 = dev(np.random.default_rng(1).normal(size=g.n_dof), torch.float32)
    for variant in ("plain", "tma"):
        sh = make_shell(g, mat, rest, precision="mixed", spmv=variant, assembly="color")
        sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=1e6, want_energy=False, want_grad=False)
        ys.append(host(sh.spmv(x32)))
        sh.close()
    assert np.array_equal(ys[0], ys[1])


@pytest.mark.parametrize("assembly", ["color", "atomic"])
@pytest.mark.parametrize("case", ["annulus12x3", "sheet1x1", "sheet61x37", "sheet256-sinusoid"])
def test_spmv_symmetric_reads_match_both_triangles(monkeypatch, case, assembly):
    """The FP32 SpMV that reads each node row's blocks left of the diagonal as the transposes of
    the blocks (j, i) of earlier rows (BHEM_SPMV_SYM=1) against the default one, which streams
    both triangles (BHEM_SPMV_SYM=0). The colour-ordered assembly adds the patches into blocks
    (i, j) and (j, i) in the same order and each patch's 48x48 Hessian is exactly symmetric, so that assembled
    matrix is exactly symmetric (checked block by block) and the products, summed in the same
    order by both kernels, are bit-identical; the atomic assembly's sums run in arbitrary order,
    so its triangles, and the products, agree to FP32 rounding."""
    g, rest, q, mat = SPMV_GRIDS[case]()
    x32 = dev(np.random.default_rng(2).normal(size=g.n_dof), torch.float32)
    ys = {}
    for sym in ("1", "0"):
        monkeypatch.setenv("BHEM_SPMV_SYM", sym)
        sh = make_shell(g, mat, rest, precision="mixed", spmv="plain", assembly=assembly)
        sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=1e6, want_energy=False, want_grad=False)
        ys[sym] = host(sh.spmv(x32))
        if sym == "1" and assembly == "color" and g.n_patches <= 4096:
            rp, col, val = sh.bsr()
            rp, col, val = host(rp).astype(np.int64), host(col).astype(np.int64), host(val)
            for i in range(g.n_nodes):
                for k in range(rp[i], rp[i + 1]):
                    j = col[k]
                    kt = rp[j] + int(np.searchsorted(col[rp[j]:rp[j + 1]], i))
                    assert col[kt] == i and np.array_equal(val[k], val[kt].T), (i, j)
        sh.close()
    if assembly == "color":
        assert np.array_equal(ys["1"], ys["0"])
    else:
        assert rel(ys["1"], ys["0"]) <= 1e-6


def test_pcg_mixed_tma_matches_plain(monkeypatch):
    """PCG with the TMA SpMV (in the graph-loop form of the solve, which launches the shell's SpMV
    kernel): same iteration count, and the solution agrees to the solver tolerance (only the
    order of the p.Ap partial sums differs)."""
    monkeypatch.setenv("BHEM_PCG_LOOP", "graph")
    g, rest, q, mat = CASES["sheet10x10-noisy"]()
    mask = dev(S.pinned_mask(g, [0, g.n_nodes - 1]), torch.uint8)
    res = []
    for variant in ("plain", "tma"):
        sh = make_shell(g, mat, rest, precision="mixed", spmv=variant)
        _, G = sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=1e6)
        x, it, neg = sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=1000)
        res.append((host(x), it, neg))
        sh.close()
    assert res[0][2] == res[1][2] == 0
    assert abs(res[0][1] - res[1][1]) <= 1
    assert rel(res[1][0], res[0][0]) <= 1e-5


def test_tma_spmv_wait_timeout_is_reported_and_the_shell_recovers(monkeypatch):
    """The bulk-copy SpMV's stage waits are bounded. With a zero budget every stage wait expires:
    the solve (in its graph-loop form, which launches the shell's SpMV kernel) returns
    SHELL_ERR_TIMEOUT (the kernel still drains the copies it issued, with the default budget, so
    nothing is left in flight), and after the default budget is restored the same shell solves
    the system as before."""
    from paper_2312_14839_gb300.bhem import ShellError
    monkeypatch.setenv("BHEM_PCG_LOOP", "graph")
    g, rest, q, mat = CASES["sheet10x10-noisy"]()
    mask = dev(S.pinned_mask(g, [0, g.n_nodes - 1]), torch.uint8)
    sh = make_shell(g, mat, rest, precision="mixed", spmv="tma")
    _, G = sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=1e6)
    x0, it0, neg0 = sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=1000)
    sh.set_wait_budget(0)
    with pytest.raises(ShellError) as ei:
        sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=20)
    assert ei.value.status == 9   # SHELL_ERR_TIMEOUT
    sh.set_wait_budget(-1)
    x1, it1, neg1 = sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=1000)
    assert it1 == it0 and neg1 == neg0 == 0
    assert np.array_equal(host(x1), host(x0))
    sh.close()


def test_pcg_parity_fp64():
    g, rest, q, mat = CASES["sheet10x10-noisy"]()
    dt = 1e-3
    pat = O.bsr_pattern(g)
    _, grad0, (rp0, col0, val0) = O.assemble(g, mat, rest, q, mass_scale=1 / dt ** 2, pattern=pat)
    mask = S.pinned_mask(g, [0, g.n_nodes - 1])
    x0, it0, st0 = O.pcg(rp0, col0, val0, -grad0, mask=mask, rtol=1e-6, max_iter=1000)
    sh = make_shell(g, mat, rest, precision="fp64")
    _, G = sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=1 / dt ** 2)
    x, it, neg = sh.pcg_solve(-G, mask=dev(mask, torch.uint8), rtol=1e-6, max_iter=1000)
    assert st0 == 0 and neg == 0
    assert it == it0
    assert rel(host(x), x0) <= 1e-9


def _config1_run(prec, steps=10, host_buffers=False):
    g, rest, q0 = S.sheet_noisy(10, 1e-3, 1)
    mat = THIN
    c = S.corner_nodes(g)
    mask = S.pinned_mask(g, [c[0], c[3]])
    qfix = q0.reshape(-1).copy()
    sh = make_shell(g, mat, rest, precision=prec)
    P = __import__("paper_2312_14839_gb300.bhem", fromlist=["step_params"]).step_params(dt=1e-3)
    if host_buffers:
        q, v = q0.reshape(-1).copy(), np.zeros(g.n_dof)
        m, qf = mask, qfix
    else:
        q, v = dev(q0.reshape(-1)), torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
        m, qf = dev(mask, torch.uint8), dev(qfix)
    out = []
    for _ in range(steps):
        st = sh.newton_step(q, v, P, mask=m, q_fixed=qf)
        qq = q.copy() if host_buffers else host(q)
        vv = v.copy() if host_buffers else host(v)
        out.append((st, qq, vv))
    return g, mat, rest, q0, mask, qfix, out


def test_newton_config1_fp64_identical_iteration_counts():
    g, mat, rest, q0, mask, qfix, out = _config1_run("fp64")
    Po = O.step_params(dt=1e-3)
    q, v = q0.reshape(-1).copy(), np.zeros(g.n_dof)
    for st, qg, vg in out:
        q, v, so = O.newton_step(g, mat, rest, q, v, Po, mask=mask, qfix=qfix)
        assert st["status"] == 0 and so["status"] == 0
        assert st["newton_iters"] == so["newton_iters"]
        assert st["pcg_iters_total"] == so["pcg_iters_total"]
        assert st["res_final"] <= 1e-8 * st["res0"]
        assert rel(qg, q) <= 1e-11
        assert rel(vg, v) <= 1e-7


def test_newton_config1_mixed_precision():
    g, mat, rest, q0, mask, qfix, out = _config1_run("mixed")
    Po = O.step_params(dt=1e-3)
    q, v = q0.reshape(-1).copy(), np.zeros(g.n_dof)
    for st, qg, vg in out:
        q, v, so = O.newton_step(g, mat, rest, q, v, Po, mask=mask, qfix=qfix)
        assert st["status"] == 0
        assert abs(st["newton_iters"] - so["newton_iters"]) <= 1
        assert st["res_final"] <= 1e-8 * st["res0"]
        assert rel(vg, v) <= 1e-5
        q, v = qg.copy(), vg.copy()   # continue the oracle from the GPU state (no drift)


@pytest.mark.parametrize("hessian", ["exact", "pseudo"])
def test_config2_twist_mixed_against_fp64_oracle(hessian):
    """Config 2 (30x30 sheet, centre twist 2 deg/step, no gravity, dt = 2 ms): all 200
    mixed-precision GPU steps against the FP64 oracle, each step started from the GPU state.
    Newton counts agree to within one (FP32 Hessians), every step meets 1e-8, and the states agree
    to the solver's tolerance."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest = S.flat_sheet(30, 30)
    mat = THIN
    sh = make_shell(g, mat, rest, precision="mixed", hessian=hessian)
    P = step_params(dt=2e-3, gravity=(0.0, 0.0, 0.0))
    Po = O.step_params(dt=2e-3, gravity=(0.0, 0.0, 0.0), pseudo_hessian=hessian == "pseudo")
    q, v = dev(rest.reshape(-1)), torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    steps = 200   # through the buckling regime (from about step 18) to the end of the twist
    fixes = 0
    for k in range(1, steps + 1):
        mask, vals = S.twist_prescription(g, rest, k)
        q_prev, v_prev = host(q), host(v)
        st = sh.newton_step(q, v, P, mask=dev(mask, torch.uint8), q_fixed=dev(vals))
        qo, vo, so = O.newton_step(g, mat, rest, q_prev, v_prev, Po, mask=mask, qfix=vals)
        assert st["status"] == 0 and so["status"] == 0, (k, st, so)
        assert abs(st["newton_iters"] - so["newton_iters"]) <= 1, (k, st, so)
        assert st["res_final"] <= 1e-8 * st["res0"]
        dq_g, dq_o = host(q) - q_prev, qo - q_prev
        err = rel(dq_g, dq_o)
        print(f"twist step {k}: newton {st['newton_iters']} (oracle {so['newton_iters']}), "
              f"diagonal fixes {st['diag_fixes']} ({so['diag_fixes']}), step error {err:.2e}")
        assert err <= 1e-5, (k, err)
        fixes += so["diag_fixes"]
    assert fixes > 0   # the run reaches the regime where normal diagonal entries turn negative


def _fp64_step_against_oracle(g, mat, rest, q0, P, Po, mask=None, qfix=None, v0=None):
    sh = make_shell(g, mat, rest, precision="fp64")
    v0 = np.zeros(g.n_dof) if v0 is None else v0
    q, v = dev(q0.reshape(-1)), dev(v0)
    kw = {} if mask is None else {"mask": dev(mask, torch.uint8), "q_fixed": dev(qfix)}
    st = sh.newton_step(q, v, P, **kw)
    qo, vo, so = O.newton_step(g, mat, rest, q0.reshape(-1), v0, Po, mask=mask, qfix=qfix)
    return st, so, host(q), qo


def _q_bound(st, so):
    """State bound of an FP64 step against the oracle: rounding when every PCG solve stopped at the
    same iteration, else the Newton criterion's (see the test below)."""
    return 1e-11 if st["pcg_iters_total"] == so["pcg_iters_total"] else 1e-9


def test_newton_backtracking_and_regulariser_ladder_fp64_identical():
    """16x16 sheet relaxing from the 5 cm sinusoid under gravity: the FP64 step meets negative
    curvature (regulariser ladder) and rejects line-search trials (quadratic and cubic
    backtracks). The GPU takes the same decisions as the oracle: identical Newton, backtrack,
    regularisation and diagonal-fix counts, and the same state within the FP64 tolerance. The
    GPU's FP64 Hessian and gradient are sums of patch contributions in atomic order, so their last
    bits vary from run to run; over this step's ~600 PCG iterations a solve whose residual ends
    within rounding of its tolerance can stop one iteration apart (seen: 624 against 625 in one
    of several runs), so the PCG totals may differ by at most one per Newton iteration. The states
    then agree to FP64 rounding (1e-11) when the PCG totals are equal; when one solve stopped an
    iteration apart, the two iterates differ by that solve's remainder, which the step's Newton
    criterion (relative residual 1e-8, with PCG at eta = 1e-6) bounds, and the bound is 1e-9."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest, q0 = S.sheet_sinusoid(16, 3, 0.05)
    st, so, qg, qo = _fp64_step_against_oracle(g, THIN, rest, q0, step_params(dt=1e-3, newton_max=50),
                                                O.step_params(dt=1e-3, newton_max=50))
    assert so["status"] == 0 and so["ls_backtracks"] >= 2 and so["regularizations"] >= 2
    for key in ("status", "newton_iters", "ls_backtracks", "regularizations", "diag_fixes"):
        assert st[key] == so[key], (key, st, so)
    assert abs(st["pcg_iters_total"] - so["pcg_iters_total"]) <= so["newton_iters"], (st, so)
    assert rel(qg, qo) <= _q_bound(st, so), (rel(qg, qo), st["pcg_iters_total"], so["pcg_iters_total"])
    assert so["tau_final"] > 0 and st["tau_final"] == pytest.approx(so["tau_final"], rel=1e-12)
    # the same step with a regulariser level carried in (the first solve starts at 0.1): the same
    # decisions on both sides
    tau = 1.0
    st2, so2, qg2, qo2 = _fp64_step_against_oracle(g, THIN, rest, q0, step_params(dt=1e-3, newton_max=50, tau_carry=tau),
                                                   O.step_params(dt=1e-3, newton_max=50, tau_carry=tau))
    assert so2["status"] == 0
    for key in ("status", "newton_iters", "ls_backtracks", "regularizations", "diag_fixes"):
        assert st2[key] == so2[key], (key, st2, so2)
    assert abs(st2["pcg_iters_total"] - so2["pcg_iters_total"]) <= so2["newton_iters"], (st2, so2)
    assert rel(qg2, qo2) <= _q_bound(st2, so2), (rel(qg2, qo2), st2["pcg_iters_total"], so2["pcg_iters_total"])


def test_newton_planar_twist_diagonal_fix_fp64_identical():
    """10x10 sheet twisted 8 deg per step about its normal: from step 15 normal diagonal entries
    turn negative and are fixed locally; every count, the fixes included, equals the oracle's and
    the sheet stays exactly planar."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest = S.flat_sheet(10, 10)
    mat = THIN
    sh = make_shell(g, mat, rest, precision="fp64")
    P = step_params(dt=2e-3, gravity=(0.0, 0.0, 0.0), newton_max=30)
    Po = O.step_params(dt=2e-3, gravity=(0.0, 0.0, 0.0), newton_max=30)
    q, v = dev(rest.reshape(-1)), torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    qo, vo = rest.reshape(-1).copy(), np.zeros(g.n_dof)
    fixes = 0
    for k in range(1, 21):
        mask, vals = S.twist_prescription(g, rest, k, deg_per_step=8.0)
        st = sh.newton_step(q, v, P, mask=dev(mask, torch.uint8), q_fixed=dev(vals))
        qo, vo, so = O.newton_step(g, mat, rest, qo, vo, Po, mask=mask, qfix=vals)
        for key in ("status", "newton_iters", "pcg_iters_total", "ls_backtracks", "regularizations",
                    "diag_fixes"):
            assert st[key] == so[key], (k, key, st, so)
        assert rel(host(q), qo) <= 1e-11
        assert np.all(host(q).reshape(-1, 12)[:, 2::3] == 0.0)
        fixes += st["diag_fixes"]
    assert fixes > 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_accepted_step_residual_matches_direct_residual(prec):
    """After an accepted full Newton step (alpha = 1 at the first trial), the step forms the
    residual's inertial part from the line search's M d instead of a second mass product. It must
    equal the residual g = M (q' - y) / dt^2 + grad V(q') - F_g of the implicit-Euler equations
    (Sec. 6.1), formed here directly at the returned q' from the oracle's gradient, mass and load,
    within the FP64 tolerance relative to the step's reference residual."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest, q0 = S.sheet_noisy(10, 1e-3, 1)
    mat = THIN
    c = S.corner_nodes(g)
    mask = S.pinned_mask(g, [c[0], c[3]])
    qfix = q0.reshape(-1).copy()
    dt, grav = 1e-3, np.array([0.0, 0.0, -9.81])
    sh = make_shell(g, mat, rest, precision=prec)
    q, v = dev(q0.reshape(-1)), torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    st = sh.newton_step(q, v, step_params(dt=dt, newton_max=1), mask=dev(mask, torch.uint8),
                        q_fixed=dev(qfix))
    assert st["newton_iters"] == 1 and st["ls_backtracks"] == 0
    assert st["res_final"] < st["res0"]
    q1 = host(q)
    y = q0.reshape(-1)   # q^n + dt v^n with v^n = 0
    _, grad, _ = O.assemble(g, mat, rest, q1, want_hess=False)
    mval, fs = O.mass(g, mat, rest)
    rp, col = O.bsr_pattern(g)
    x = (q1 - y).reshape(g.n_nodes, 4, 3)
    Mx = np.zeros_like(x)
    for i in range(g.n_nodes):
        for k in range(rp[i], rp[i + 1]):
            Mx[i] += mval[k] @ x[col[k]]
    res = Mx / dt ** 2 + grad.reshape(g.n_nodes, 4, 3) - fs[:, :, None] * grav[None, None, :]
    res = res.reshape(-1)
    res[mask.astype(bool)] = 0.0
    assert abs(st["res_final"] - np.linalg.norm(res)) <= 1e-11 * st["res0"]


def test_newton_host_buffers_match_device_buffers():
    *_, out_d = _config1_run("fp64", steps=3)
    *_, out_h = _config1_run("fp64", steps=3, host_buffers=True)
    for (sd, qd, vd), (sh_, qh, vh) in zip(out_d, out_h):
        assert sd["newton_iters"] == sh_["newton_iters"]
        assert rel(qh, qd) <= 1e-13 and rel(vh, vd) <= 1e-9


@pytest.mark.parametrize("maker", [lambda: S.sheet_sinusoid(256, 3), lambda: S.annulus_sinusoid(280, 5, 3)])
def test_full_size_sampled_element_parity(maker):
    """Full-size sheets in the bench's configuration: FP32 element outputs of sampled patches
    against the oracle computed patch by patch."""
    g, rest, q = maker()
    mat = THIN
    sh = make_shell(g, mat, rest, precision="mixed")
    E, G, H = sh.element_egh(dev(q.reshape(-1)))
    idx = np.unique(np.concatenate([[0, g.n_patches - 1], np.random.default_rng(7).integers(0, g.n_patches, 40)]))
    ti = torch.as_tensor(idx, device="cuda")
    Es, Gs, Hs = host(E[ti]), host(G[ti]), host(H[ti])
    for k, p in enumerate(idx):
        e0, g0, h0 = O.element_egh(O.gather(g, q, p), O.gather(g, rest, p), g.dxi1, g.dxi2, mat)
        assert abs(Es[k] - e0) <= 1e-5 * abs(e0)
        assert rel(Gs[k], g0) <= 1e-5
        assert rel(Hs[k], h0) <= 1e-5


def test_full_size_sampled_assembly_rows():
    """256x256 BSR: sampled block rows against the sum of the oracle's element blocks of the
    (up to 4) patches around the node."""
    g, rest, q = S.sheet_sinusoid(256, 3)
    mat = THIN
    ms = 1e6
    sh = make_shell(g, mat, rest, precision="mixed")
    sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=ms)
    rp, col, val = sh.bsr()
    rp, col = host(rp).astype(np.int64), host(col).astype(np.int64)
    for node in [0, 257, 33000, g.n_nodes - 1, 12345]:
        i, j = node % g.n1, node // g.n1
        want = {}
        for pv in (j - 1, j):
            for pu in (i - 1, i):
                if not (0 <= pu < g.nu and 0 <= pv < g.nv):
                    continue
                p = pv * g.nu + pu
                nd = O.patch_nodes(g, p)
                _, _, H = O.element_egh(O.gather(g, q, p), O.gather(g, rest, p), g.dxi1, g.dxi2, mat)
                m, _ = O.element_mass(O.gather(g, rest, p), g.dxi1, g.dxi2, mat)
                H = H + ms * np.kron(m, np.eye(3))
                a = list(nd).index(node)
                for b in range(4):
                    blk = H[a * 12:(a + 1) * 12, b * 12:(b + 1) * 12]
                    want[nd[b]] = want.get(nd[b], 0) + blk
        ks = range(rp[node], rp[node + 1])
        assert sorted(want) == [col[k] for k in ks]
        got = np.concatenate([host(val[k]) for k in ks])
        ref = np.concatenate([want[col[k]] for k in ks])
        assert rel(got, ref) <= 1e-5


def test_degenerate_and_nonfinite_inputs_are_reported():
    from paper_2312_14839_gb300.bhem import ShellError, step_params
    g, rest, q, mat = CASES["sheet1x1"]()
    sh = make_shell(g, mat, rest, precision="fp64")
    P = step_params()
    zero = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(ShellError) as e:
        sh.newton_step(zero.clone(), zero.clone(), P)
    assert e.value.status == 4
    bad = dev(q.reshape(-1)).clone()
    bad[5] = float("nan")
    with pytest.raises(ShellError) as e:
        sh.newton_step(bad, zero.clone(), P)
    assert e.value.status in (4, 5)
    # the shell stays usable afterwards
    st = sh.newton_step(dev(q.reshape(-1)), zero.clone(), P)
    assert st["status"] == 0


def test_spmv_rejects_misaligned_x():
    """Every SpMV kernel reads x in 16-byte vectors: a misaligned x is an argument error, raised
    before any launch."""
    from paper_2312_14839_gb300.bhem import ShellError
    g, rest, q, mat = CASES["sheet1x1"]()
    sh = make_shell(g, mat, rest, precision="mixed")
    buf = torch.zeros(g.n_dof + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(ShellError, match="16-byte"):
        sh.spmv(buf[1:1 + g.n_dof])
    y = sh.spmv(buf[4:4 + g.n_dof])   # 16-byte offset: accepted
    torch.cuda.synchronize()
    assert float(y.abs().sum()) == 0.0


@pytest.mark.parametrize("case,mass_scale,fixed", [
    ("sheet10x10-noisy", 1e6, 0),      # converges to rtol
    ("sheet10x10-noisy", 1e6, 7),      # a cap that ends inside a 4-iteration loop body
    ("sinusoid16", 1.0, 0),            # indefinite: stops on negative curvature
])
def test_pcg_device_loop_matches_host_loop(monkeypatch, case, mass_scale, fixed):
    """The graph-loop form of the mixed-precision solve loops on the device (a conditional graph
    node around 4 iterations); BHEM_PCG_HOST_LOOP launches the same iterations from the host.
    Same kernels in the same order: iteration count, curvature flag and solution are identical."""
    if case == "sinusoid16":
        g, rest, q = S.sheet_sinusoid(16, 3)
        mat = THIN
    else:
        g, rest, q, mat = CASES[case]()
    mask = dev(S.pinned_mask(g, [0, g.n_nodes - 1]), torch.uint8)
    res = []
    for host_loop in (False, True):
        if host_loop:
            monkeypatch.setenv("BHEM_PCG_HOST_LOOP", "1")
        else:
            monkeypatch.delenv("BHEM_PCG_HOST_LOOP", raising=False)
            monkeypatch.setenv("BHEM_PCG_LOOP", "graph")
        sh = make_shell(g, mat, rest, precision="mixed", assembly="color")
        _, G = sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=mass_scale)
        x, it, neg = sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=1000, fixed_iters=fixed)
        res.append((host(x), it, neg))
        sh.close()
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2], (res[0][1:], res[1][1:])
    if fixed:
        assert res[0][1] == fixed
    if case == "sinusoid16":
        assert res[0][2] == 1
    assert np.array_equal(res[0][0], res[1][0])


@pytest.mark.parametrize("mode", ["persistent", "cluster"])
@pytest.mark.parametrize("case,mass_scale,fixed", [
    ("sheet10x10-noisy", 1e6, 0),      # converges to rtol
    ("sheet10x10-noisy", 1e6, 7),      # a fixed iteration count
    ("sinusoid16", 1.0, 0),            # indefinite: stops on negative curvature
    ("sinusoid64", 1e6, 0),            # 4,225 nodes: many CTAs, several rows each
    ("annulus280x5", 1e6, 0),          # periodic
])
def test_pcg_single_launch_forms_match_host_loop(monkeypatch, mode, case, mass_scale, fixed):
    """Two mixed-precision solves run as one launch: the persistent cooperative kernel, whose CTAs
    meet at software grid barriers, and the thread-block cluster kernel (BHEM_PCG_LOOP=cluster),
    whose CTAs meet at the hardware cluster barrier and reduce through distributed shared memory. The host-chunked form launches one kernel per phase. Same arithmetic per element,
    partial sums combined in another order: same curvature flag, iteration counts within one (the
    stopping test may fall either side), solutions within the solver's tolerance."""
    if case == "sinusoid16":
        g, rest, q = S.sheet_sinusoid(16, 3)
        mat = THIN
    elif case == "sinusoid64":
        g, rest, q = S.sheet_sinusoid(64, 3, 0.01)
        mat = THIN
    elif case == "annulus280x5":
        g, rest, q = S.annulus_sinusoid(280, 5, 3, 0.01)
        mat = THIN
    else:
        g, rest, q, mat = CASES[case]()
    mask = dev(S.pinned_mask(g, [0]), torch.uint8)
    res = []
    for m in (mode, "host"):
        monkeypatch.setenv("BHEM_PCG_LOOP", m)
        sh = make_shell(g, mat, rest, precision="mixed", assembly="color")
        _, G = sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=mass_scale)
        x, it, neg = sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=1000, fixed_iters=fixed)
        res.append((host(x), it, neg))
        sh.close()
    assert res[0][2] == res[1][2], (res[0][1:], res[1][1:])
    assert abs(res[0][1] - res[1][1]) <= 1, (res[0][1:], res[1][1:])
    if fixed:
        assert res[0][1] == res[1][1] == fixed
    if case == "sinusoid16":
        assert res[0][2] == 1
    else:
        assert rel(res[0][0], res[1][0]) <= 1e-4


def test_pcg_persistent_barrier_timeout_is_reported_and_the_shell_recovers(monkeypatch):
    """The persistent solve's grid barriers are bounded waits. With a zero budget every CTA that
    is not the last to arrive gives up at once: the solve returns SHELL_ERR_TIMEOUT and every CTA
    leaves the kernel. With the default budget restored, the same shell solves the system."""
    from paper_2312_14839_gb300.bhem import ShellError
    monkeypatch.setenv("BHEM_PCG_LOOP", "persistent")
    g, rest, q, mat = CASES["sheet10x10-noisy"]()
    mask = dev(S.pinned_mask(g, [0, g.n_nodes - 1]), torch.uint8)
    sh = make_shell(g, mat, rest, precision="mixed")
    _, G = sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=1e6)
    x0, it0, neg0 = sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=1000)
    sh.set_wait_budget(0)
    with pytest.raises(ShellError) as ei:
        sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=20)
    assert ei.value.status == 9   # SHELL_ERR_TIMEOUT
    sh.set_wait_budget(-1)
    x1, it1, neg1 = sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=1000)
    assert it1 == it0 and neg1 == neg0 == 0
    assert np.array_equal(host(x1), host(x0))
    sh.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_step_converged_at_start_then_step_again(prec):
    """On a shell large enough for the second stream (128 x 128 patches), a step that is converged
    at q (here: newton_rtol = 1, met by the residual at q itself) takes no Newton iteration: the
    first Hessian, assembled beside the residual, is left unused and joined. A degenerate input
    on that path is reported, and the shell then steps as a fresh shell does."""
    from paper_2312_14839_gb300.bhem import ShellError, step_params
    g, rest, q = S.sheet_noisy(128, 1e-3, 1)
    mat = THIN
    c = S.corner_nodes(g)
    mask = dev(S.pinned_mask(g, [c[0], c[3]]), torch.uint8)
    P = step_params(dt=1e-3, gravity=(0.0, 0.0, 0.0), newton_max=3, pcg_fixed_iters=30)
    P0 = step_params(dt=1e-3, gravity=(0.0, 0.0, 0.0), newton_rtol=1.0)
    sh = make_shell(g, mat, rest, precision=prec)
    zero = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    q0 = dev(q.reshape(-1))
    st = sh.newton_step(q0.clone(), zero.clone(), P0, mask=mask, q_fixed=q0)
    assert st["status"] == 0 and st["newton_iters"] == 0, st
    with pytest.raises(ShellError) as e:
        sh.newton_step(zero.clone(), zero.clone(), P0)
    assert e.value.status == 4
    qa, va = q0.clone(), zero.clone()
    st_a = sh.newton_step(qa, va, P, mask=mask, q_fixed=q0)
    fresh = make_shell(g, mat, rest, precision=prec)
    qb, vb = q0.clone(), zero.clone()
    st_b = fresh.newton_step(qb, vb, P, mask=mask, q_fixed=q0)
    assert st_a["status"] in (0, 6) and st_a["status"] == st_b["status"]
    assert st_a["newton_iters"] == st_b["newton_iters"]
    assert rel(host(qa) - host(q0), host(qb) - host(q0)) <= (1e-9 if prec == "fp64" else 1e-4)


def _implicit_euler_residual_and_potential(g, mat, rest, q, y, dt, grav, mask=None):
    """|g_free| and Pi of Eq. implicit at q from the oracle's elastic energy and gradient and its
    consistent mass (assembled here as a scipy sparse matrix over the oracle's 4x4 mass blocks)."""
    import scipy.sparse as sp
    E, grad, _ = O.assemble(g, mat, rest, q, want_hess=False)
    mval, fs = O.mass(g, mat, rest)
    rp, col = O.bsr_pattern(g)
    n = g.n_nodes
    rows = np.repeat(np.arange(n), np.diff(rp))
    bi, bj = np.meshgrid(np.arange(4), np.arange(4), indexing="ij")
    R = (rows[:, None, None] * 4 + bi[None]).reshape(-1)
    Cc = (col[:, None, None] * 4 + bj[None]).reshape(-1)
    Ms = sp.csr_matrix((mval.reshape(-1), (R, Cc)), shape=(4 * n, 4 * n))
    d = (q - y).reshape(n * 4, 3)
    Md = (Ms @ d).reshape(-1)
    F = (fs[:, :, None] * np.asarray(grav)[None, None, :]).reshape(-1)
    res = grad + Md / dt ** 2 - F
    if mask is not None:
        res[mask.astype(bool)] = 0.0
    pot = E + 0.5 * float((q - y) @ Md) / dt ** 2 - float(F @ q)
    return float(np.linalg.norm(res)), pot


def test_full_size_bench_step_residual_and_decrease():
    """The bench's step in its own launch configuration, at full size (256 x 256 sinusoid sheet,
    792,588 DOF, mixed precision, one Newton iteration with 50-iteration PCG solves, the
    regulariser level carried in): the oracle's implicit-Euler residual at the returned state
    equals the step's reported res_final (FP64 parts within 1e-9), the reported res0 equals the
    oracle's residual at the start, and the step lowered the incremental potential Pi."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest, q0 = S.sheet_sinusoid(256, 3)
    dt, grav = 1e-3, (0.0, 0.0, -9.81)
    sh = make_shell(g, THIN, rest, precision="mixed")
    P = step_params(dt=dt, newton_max=1, pcg_fixed_iters=50, tau_carry=1.0)
    q, v = dev(q0.reshape(-1)), torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    st = sh.newton_step(q, v, P)
    assert st["newton_iters"] == 1 and st["status"] in (0, 6), st
    assert st["pcg_iters_total"] >= 50 and st["tau_final"] > 0
    q1 = host(q)
    y = q0.reshape(-1)   # q^n + dt v^n with v^n = 0
    r0, pot0 = _implicit_euler_residual_and_potential(g, THIN, rest, y, y, dt, grav)
    r1, pot1 = _implicit_euler_residual_and_potential(g, THIN, rest, q1, y, dt, grav)
    assert abs(st["res0"] - r0) <= 1e-9 * r0, (st["res0"], r0)
    assert abs(st["res_final"] - r1) <= 1e-9 * r0, (st["res_final"], r1)
    assert r1 < r0 and pot1 < pot0, (r0, r1, pot0, pot1)
    sh.close()


@pytest.mark.parametrize("grid,hessian", [((64, 64), "exact"), ((30, 30), "pseudo"), ((7, 2), "exact")])
def test_fused_first_residual_and_hessian_equal_separate_launches(grid, hessian, monkeypatch):
    """A mixed-precision step evaluates its first FP64 residual and its first FP32 Hessian in one
    element launch (the Hessian's warps also run the FP64 energy and gradient). Against the same
    step with separate launches (BHEM_FUSE_FIRST_HESSIAN=0 at shell creation): the same Newton and
    PCG decisions, the same starting residual to FP64 rounding (the gradient is an atomic sum in
    either form), and the same final state within the mixed-precision tolerance."""
    from paper_2312_14839_gb300.bhem import step_params
    nu, nv = grid
    if nv == 2:
        g, rest = S.annulus(nu, nv)
        q0 = S.noisy(rest, 1e-3, 17)
    else:
        g, rest, q0 = S.sheet_sinusoid(nu, 3, 0.05)
    P = step_params(dt=1e-3, newton_max=8)
    out = {}
    for fuse in ("1", "0"):
        monkeypatch.setenv("BHEM_FUSE_FIRST_HESSIAN", fuse)
        sh = make_shell(g, THIN, rest, precision="mixed", hessian=hessian)
        q, v = dev(q0.reshape(-1)), dev(np.zeros(g.n_dof))
        st = sh.newton_step(q, v, P)
        out[fuse] = (st, host(q))
    (s1, q1), (s0, q0_) = out["1"], out["0"]
    for key in ("status", "newton_iters", "ls_backtracks", "regularizations", "diag_fixes"):
        assert s1[key] == s0[key], (key, s1, s0)
    assert abs(s1["pcg_iters_total"] - s0["pcg_iters_total"]) <= s0["newton_iters"], (s1, s0)
    assert s1["res0"] == pytest.approx(s0["res0"], rel=1e-12)
    assert rel(q1 - q0.reshape(-1), q0_ - q0.reshape(-1)) <= 1e-5


@pytest.mark.parametrize("case,mass_scale,fixed", [
    ("sheet10x10-noisy", 1e6, 0),
    ("sheet10x10-noisy", 1e6, 7),
    ("sinusoid16", 1.0, 0),            # indefinite: negative curvature
    ("annulus280x5", 1e6, 0),
])
def test_pcg_folded_direction_update_matches_separate_kernel(monkeypatch, case, mass_scale, fixed):
    """Small shells fold the PCG's p = z + beta p into the next iteration's SpMV, which gathers z
    and forms Ap as (A + tau D) z + beta Ap. Against the separate p-update kernel
    (BHEM_PCG_PUPDATE=1): the same direction arithmetic, Ap by linearity instead of recomputed, so
    the same curvature flag, iteration counts within one and solutions within the solver's
    tolerance."""
    if case == "sinusoid16":
        g, rest, q = S.sheet_sinusoid(16, 3)
        mat = THIN
    elif case == "annulus280x5":
        g, rest, q = S.annulus_sinusoid(280, 5, 3, 0.01)
        mat = THIN
    else:
        g, rest, q, mat = CASES[case]()
    mask = dev(S.pinned_mask(g, [0]), torch.uint8)
    res = []
    for v in ("0", "1"):
        monkeypatch.setenv("BHEM_PCG_PUPDATE", v)
        sh = make_shell(g, mat, rest, precision="mixed", assembly="color")
        _, G = sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=mass_scale)
        x, it, neg = sh.pcg_solve(-G, mask=mask, rtol=1e-6, max_iter=1000, fixed_iters=fixed)
        res.append((host(x), it, neg))
        sh.close()
    assert res[0][2] == res[1][2], (res[0][1:], res[1][1:])
    assert abs(res[0][1] - res[1][1]) <= 1, (res[0][1:], res[1][1:])
    if fixed:
        assert res[0][1] == res[1][1] == fixed
    if case == "sinusoid16":
        assert res[0][2] == 1
    else:
        assert rel(res[0][0], res[1][0]) <= 1e-4
