"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/bhem.h declares
(no GPU needed: nothing here launches a kernel)."""
import os
import re
import subprocess

from paper_2312_14839_gb300 import bhem, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bhem.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SHELL_API\s+[\w\s\*]+?\b(shell_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("shell_create", "shell_destroy", "shell_energy_grad_hess", "shell_newton_step",
                 "shell_element_egh", "shell_pcg_solve", "shell_spmv", "shell_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (shell_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    lib = bhem.load()
    for s in declared_symbols():
        assert getattr(lib, s) is not None


def test_argument_errors_need_no_gpu():
    lib = bhem.load()
    assert lib.shell_create(None, None, None, None, None, None) == 1   # SHELL_ERR_ARG
    assert b"NULL" in lib.shell_last_error()
    assert lib.shell_destroy(None) == 0
    assert lib.shell_trace_rays(None, None, 0, None, None, 1, None, None, None, None, None) == 1
    assert lib.shell_ccd_points(None, None, None, 0, None, None, 1, None, None, None, None, None) == 1


def test_invalid_options_are_rejected_before_any_device_work():
    import ctypes as C
    import numpy as np
    lib = bhem.load()
    g = bhem.shell_grid(2, 2, 0, 0, 0.5, 0.5)
    m = bhem.shell_material(1e5, 0.3, 1e-3, 200.0)
    rest = np.zeros(9 * 12)
    out = C.c_void_p()
    for spmv, solver in ((3, 0), (-1, 0), (0, 2)):
        o = bhem.shell_options(1, 0, 0, spmv, solver)
        rc = lib.shell_create(C.byref(g), C.byref(m), rest.ctypes.data_as(C.c_void_p), C.byref(o), None,
                              C.byref(out))
        assert rc == 1, (spmv, solver)
        assert b"invalid options" in lib.shell_last_error()
        assert not out.value



def _patch_nodes(nu, nv, pu_per, pv_per):
    """Corner node ids of every patch, written from the header's node and patch numbering."""
    n1 = nu if pu_per else nu + 1
    n2 = nv if pv_per else nv + 1
    out = []
    for pv in range(nv):
        for pu in range(nu):
            out.append({((pv + b) % n2) * n1 + (pu + a) % n1 for a in (0, 1) for b in (0, 1)})
    return out


def test_colour_classes_share_no_node():
    """Colour-ordered assembly adds element blocks without atomics, one launch per colour: two
    patches of one colour must never touch the same node, also across a periodic seam with an odd
    patch count (nu = 7, 13, ... put patch nu - 1 and patch 0 on one colour before)."""
    for per_u in (0, 1):
        for per_v in (0, 1):
            for nu in range(1, 21):
                for nv in range(1, 21):
                    col = bhem.grid_colours(nu, nv, per_u, per_v).reshape(-1)
                    assert col.min() >= 0 and col.max() < 9
                    nodes = _patch_nodes(nu, nv, per_u, per_v)
                    for c in set(col.tolist()):
                        seen = set()
                        for p in (col == c).nonzero()[0]:
                            assert not (nodes[p] & seen), (nu, nv, per_u, per_v, c, int(p))
                            seen |= nodes[p]
