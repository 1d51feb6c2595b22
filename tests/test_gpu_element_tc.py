"""GPU: the FP32 element Hessian with its contraction on the tensor cores (tcgen05, kind::tf32,
head-and-tail TF32 products) against the FFMA form of the same kernel and against the FP64 oracle.

The tensor-core form is the default of a mixed-precision shell; BHEM_ELEMENT=ffma at shell creation
selects the FFMA form. Both build the same Gauss-point matrices M_g; they differ in the rounding of
the contraction K = sum_g Phi_g^T M_g Phi_g (App. B.2) only, so they agree within the FP32 bound
of the parity tests (1e-5 normwise per patch), and each agrees with the oracle within it.
"""
import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THIN = S.SHEET_MATERIAL
THICK = S.Material(1e5, 0.3, 0.05, 200.0)


def dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def shell(monkeypatch, form, g, mat, rest, **kw):
    from paper_2312_14839_gb300.bhem import Shell
    if form == "ffma":
        monkeypatch.setenv("BHEM_ELEMENT", "ffma")
    else:
        monkeypatch.delenv("BHEM_ELEMENT", raising=False)
    return Shell(g, mat, dev(rest.reshape(-1)), precision="mixed", **kw)


# patch counts: 1, 9 and 30 (not multiples of the 4 patches of a CTA), 35 (periodic, odd), 4,096
CASES = {
    "sheet1x1": lambda: (*S.sheet_noisy(1, 1e-2, 2), THIN),
    "sheet3x3-thick": lambda: (lambda g, r: (g, r, S.noisy(r, 2e-2, 3), THICK))(*S.flat_sheet(3, 3, 0.6, 0.4)),
    "annulus10x3": lambda: (lambda g, r: (g, r, S.noisy(r, 1e-2, 4), THIN))(*S.annulus(10, 3)),
    "annulus7x5-odd-thick": lambda: (lambda g, r: (g, r, S.noisy(r, 1e-2, 5), THICK))(*S.annulus(7, 5)),
    "sheet64-sinusoid": lambda: (*S.sheet_sinusoid(64, 3), THIN),
}


@pytest.mark.parametrize("hessian", ["exact", "pseudo"])
@pytest.mark.parametrize("case", list(CASES))
def test_tensor_core_hessian_matches_ffma_and_oracle(monkeypatch, case, hessian):
    """Unassembled per-patch outputs: the tensor-core Hessian against the FFMA one and against the
    oracle (sampled patches), exact symmetry, and the FP32 energies and gradients (the same
    Gauss-point code in both kernels; the compiler may contract its multiply-adds differently in
    each, so they agree to FP32 rounding rather than bit for bit)."""
    g, rest, q, mat = CASES[case]()
    out = {}
    for form in ("tc", "ffma"):
        sh = shell(monkeypatch, form, g, mat, rest, hessian=hessian)
        E, G, H = sh.element_egh(dev(q.reshape(-1)))
        torch.cuda.synchronize()
        out[form] = (host(E), host(G), host(H))
        sh.close()
    (Et, Gt, Ht), (Ef, Gf, Hf) = out["tc"], out["ffma"]
    assert np.abs(Et - Ef).max() <= 1e-6 * np.abs(Ef).max()
    assert rel(Gt, Gf) <= 1e-6
    worst = 0.0
    for p in range(g.n_patches):
        worst = max(worst, rel(Ht[p], Hf[p]))
        assert np.array_equal(Ht[p], Ht[p].T), p
    assert worst <= 5e-6, worst
    idx = sorted({0, g.n_patches - 1, g.n_patches // 2, g.n_patches // 3})
    for p in idx:
        _, _, h0 = O.element_egh(O.gather(g, q, p), O.gather(g, rest, p), g.dxi1, g.dxi2, mat,
                                 pseudo=hessian == "pseudo")
        assert rel(Ht[p], h0) <= 1e-5, (p, rel(Ht[p], h0))


@pytest.mark.parametrize("assembly", ["atomic", "color"])
@pytest.mark.parametrize("case", ["annulus7x5-odd-thick", "sheet64-sinusoid"])
def test_tensor_core_assembly_matches_ffma(monkeypatch, case, assembly):
    """Assembled K + mass_scale M (BSR) from the tensor-core pass against the FFMA pass."""
    g, rest, q, mat = CASES[case]()
    vals = {}
    for form in ("tc", "ffma"):
        sh = shell(monkeypatch, form, g, mat, rest, assembly=assembly)
        sh.energy_grad_hess(dev(q.reshape(-1)), mass_scale=1e6)
        _, _, val = sh.bsr()
        vals[form] = host(val)
        sh.close()
    assert rel(vals["tc"], vals["ffma"]) <= 5e-6
    for k in range(0, vals["tc"].shape[0], max(1, vals["tc"].shape[0] // 50)):
        assert rel(vals["tc"][k], vals["ffma"][k]) <= 1e-5, k


def test_tensor_core_newton_step_matches_ffma(monkeypatch):
    """A mixed-precision implicit-Euler step (fused first residual and Hessian, later Hessians
    alone) with either form: the same Newton decisions and the same state within the
    mixed-precision tolerance."""
    from paper_2312_14839_gb300.bhem import step_params
    g, rest, q0 = S.sheet_sinusoid(32, 3, 0.05)
    P = step_params(dt=1e-3, newton_max=8)
    res = {}
    for form in ("tc", "ffma"):
        sh = shell(monkeypatch, form, g, THIN, rest)
        q, v = dev(q0.reshape(-1)), dev(np.zeros(g.n_dof))
        st = sh.newton_step(q, v, P)
        res[form] = (st, host(q))
        sh.close()
    (st, qt), (sf, qf) = res["tc"], res["ffma"]
    for key in ("status", "newton_iters", "ls_backtracks", "regularizations"):
        assert st[key] == sf[key], (key, st, sf)
    assert st["res0"] == pytest.approx(sf["res0"], rel=1e-12)
    assert rel(qt - q0.reshape(-1), qf - q0.reshape(-1)) <= 1e-5


def test_tensor_core_wait_timeout_is_reported_and_the_shell_recovers(monkeypatch):
    """The tensor-core pass waits on an mbarrier for each group of MMAs it commits, with a
    bounded number of polls. With a zero budget the first wait expires: the kernel raises the
    timeout bit, waits (with the full budget) for the MMAs it committed, frees its tensor memory
    and returns, and the step reports SHELL_ERR_TIMEOUT. With the default budget restored the
    same shell evaluates the patch Hessians bit-identically to before."""
    from paper_2312_14839_gb300.bhem import ShellError, step_params
    g, rest, q, mat = CASES["annulus10x3"]()
    sh = shell(monkeypatch, "tc", g, mat, rest)
    qd = dev(q.reshape(-1))
    _, _, H0 = sh.element_egh(qd)
    H0 = host(H0)
    sh.set_wait_budget(0)
    with pytest.raises(ShellError) as ei:
        sh.newton_step(qd.clone(), torch.zeros_like(qd), step_params(dt=1e-3, newton_max=4))
    assert ei.value.status == 9   # SHELL_ERR_TIMEOUT
    sh.set_wait_budget(-1)
    _, _, H1 = sh.element_egh(qd)
    assert np.array_equal(host(H1), H0)
    st = sh.newton_step(qd.clone(), torch.zeros_like(qd), step_params(dt=1e-3, newton_max=4))
    assert st["status"] == 0
    sh.close()


def test_tensor_core_pass_reports_degenerate_and_nonfinite_inputs(monkeypatch):
    """A mixed-precision step (the tensor-core pass with the fused FP64 residual) on a collapsed
    state reports SHELL_ERR_DEGENERATE, on a state with a NaN SHELL_ERR_DEGENERATE or
    SHELL_ERR_NONFINITE; the shell then steps normally."""
    from paper_2312_14839_gb300.bhem import ShellError, step_params
    g, rest, q, mat = CASES["sheet3x3-thick"]()
    sh = shell(monkeypatch, "tc", g, mat, rest)
    P = step_params(dt=1e-3, newton_max=4)
    zero = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(ShellError) as e:
        sh.newton_step(zero.clone(), zero.clone(), P)
    assert e.value.status == 4
    bad = dev(q.reshape(-1)).clone()
    bad[5] = float("nan")
    with pytest.raises(ShellError) as e:
        sh.newton_step(bad, zero.clone(), P)
    assert e.value.status in (4, 5)
    st = sh.newton_step(dev(q.reshape(-1)), zero.clone(), P)
    assert st["status"] == 0
    sh.close()


def test_unassembled_hessians_at_a_misaligned_address(monkeypatch):
    """The FP32 patch Hessians are stored in 16-byte pieces when the output is 16-byte aligned
    and element by element otherwise: an output 4 bytes off alignment receives the same values."""
    from paper_2312_14839_gb300 import bhem
    g, rest, q, mat = CASES["annulus10x3"]()
    sh = shell(monkeypatch, "tc", g, mat, rest)
    qd = dev(q.reshape(-1))
    _, _, H0 = sh.element_egh(qd, want=("h",))
    buf = torch.full((g.n_patches * 2304 + 1,), float("nan"), dtype=torch.float32, device="cuda")
    H1 = buf[1:]
    assert H1.data_ptr() % 16 == 4
    bhem._check(bhem.load().shell_element_egh(sh._h, bhem._ptr(qd), 1, None, None, bhem._ptr(H1)))
    torch.cuda.synchronize()
    assert torch.equal(H1.view(g.n_patches, 48, 48), H0)
    sh.close()


def test_tensor_core_hessians_match_ffma_on_every_patch_at_full_size(monkeypatch):
    """The bench's 256x256 sheet: all 65,536 tensor-core patch Hessians against the FFMA form's
    (which the oracle pins patch by patch on smaller grids and on samples of this one), normwise
    per patch, compared on the device."""
    g, rest, q = S.sheet_sinusoid(256, 3)
    Hs = {}
    for form in ("tc", "ffma"):
        sh = shell(monkeypatch, form, g, THIN, rest)
        _, _, H = sh.element_egh(dev(q.reshape(-1)), want=("h",))
        torch.cuda.synchronize()
        Hs[form] = H
        sh.close()
    d = torch.linalg.norm((Hs["tc"] - Hs["ffma"]).double().reshape(g.n_patches, -1), dim=1)
    ref = torch.linalg.norm(Hs["ffma"].double().reshape(g.n_patches, -1), dim=1)
    worst = float((d / ref).max())
    print(f"full-size tensor-core against FFMA: worst patch {worst:.2e}")
    assert worst <= 5e-6, worst
