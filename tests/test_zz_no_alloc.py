"""The allocation-free energy/gradient entry point (shell_energy_grad_noalloc) against the
allocating one (shell_energy_grad_hess) through the C ABI, on two calls in a row.

It serves callers that cannot allocate device memory while they run (a pool allocator that owns
all device memory, latency-bound loops, fixed-budget plug-ins); its scratch is a fixed device
array shared by all calls, so the second call checks that nothing left over from the first one
changes the result.
"""
import numpy as np
import pytest

from paper_2312_14839_gb300 import scenes as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11   # energy and gradient are FP64 on both entry points


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


CASES = {
    "sheet10x10": lambda: S.sheet_noisy(10, 1e-3, 1),
    "annulus12x3-periodic": lambda: (lambda g, r: (g, r, S.noisy(r, 1e-2, 4)))(*S.annulus(12, 3)),
    "sheet64x64-sinusoid": lambda: S.sheet_sinusoid(64, 3),
}


@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_allocating_entry_point_on_two_calls(case):
    from paper_2312_14839_gb300.bhem import Shell, energy_grad_noalloc
    g, rest, q = CASES[case]()
    mat = S.SHEET_MATERIAL
    rest_d, q1 = _dev(rest), _dev(q)
    q2 = q1 + 1e-3 * torch.sin(torch.arange(q1.numel(), device="cuda", dtype=torch.float64))
    with Shell(g, mat, rest_d, precision="fp64") as sh:
        refs = []
        for qq in (q1, q2):
            E, G = sh.energy_grad_hess(qq, want_hessian=False)
            refs.append((E.clone(), G.clone()))
    for qq, (E_ref, G_ref) in zip((q1, q2), refs):   # two calls in a row, different inputs
        E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        G = torch.full_like(q1, float("nan"))
        energy_grad_noalloc(g, mat, rest_d, qq, E, G)
        torch.cuda.synchronize()
        assert abs(float(E - E_ref)) <= TOL * abs(float(E_ref))
        assert _rel(G, G_ref) <= TOL
    # and the same input twice: identical energy (deterministic reduction)
    E1 = torch.empty(1, dtype=torch.float64, device="cuda")
    E2 = torch.empty(1, dtype=torch.float64, device="cuda")
    energy_grad_noalloc(g, mat, rest_d, q1, E1)
    energy_grad_noalloc(g, mat, rest_d, q1, E2)
    torch.cuda.synchronize()
    assert float(E1) == float(E2)


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2312_14839_gb300.bhem import ShellError, energy_grad_noalloc
    g, _ = S.flat_sheet(400, 400)
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(ShellError) as e:
        energy_grad_noalloc(g, S.SHEET_MATERIAL, x, x, x[:1], None)
    assert e.value.status == 1 and "131072" in str(e.value)
