"""Plain FP64 CPU oracle of the BHEM hot path (ctypes wrapper around ``bhem_oracle.c``).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library and its Python binding never do, and the
two share no code.

The C sources follow the paper's formulas step by step (``bhem_oracle.c``: Sec. 3, Sec. 4, Sec. 6.1,
App. A, App. B; ``ray_oracle.c``, ``ccd_oracle.c``: Sec. 5); this wrapper only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "bhem_oracle.c"), os.path.join(_HERE, "ray_oracle.c"),
         os.path.join(_HERE, "ccd_oracle.c")]
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Grid(C.Structure):
    _fields_ = [("nu", C.c_int), ("nv", C.c_int), ("periodic_u", C.c_int), ("periodic_v", C.c_int),
                ("dxi1", C.c_double), ("dxi2", C.c_double)]


class Material(C.Structure):
    _fields_ = [("young", C.c_double), ("poisson", C.c_double), ("thickness", C.c_double),
                ("density", C.c_double)]


class StepParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("newton_rtol", C.c_double),
                ("newton_max", C.c_int), ("pcg_rtol", C.c_double), ("pcg_max", C.c_int),
                ("pcg_fixed_iters", C.c_int), ("pseudo_hessian", C.c_int), ("tau_carry", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("pcg_iters_total", C.c_int),
                ("ls_backtracks", C.c_int), ("regularizations", C.c_int), ("status", C.c_int),
                ("diag_fixes", C.c_int), ("res0", C.c_double), ("res_final", C.c_double),
                ("tau_final", C.c_double)]


# phi(alpha, ctx) callback of og_line_search
PHI_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, -fopenmp when available, no target-specific flags) into
    oracle/_lib."""
    with _lock:
        if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS):
            os.makedirs(_LIBDIR, exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"]
            try:   # OpenMP over the independent per-patch and per-row loops, when the compiler has it
                subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
            except subprocess.CalledProcessError:
                subprocess.check_call(base)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        d, i, p = C.c_double, C.c_int, C.c_void_p
        lib.og_hermite_w.restype = d
        lib.og_hermite_w.argtypes = [i, i, d, i]
        lib.og_gauss4.argtypes = [p, p]
        lib.og_shape.argtypes = [d, d, d, d, p]
        lib.og_n_nodes.restype = i
        lib.og_n_nodes.argtypes = [p]
        lib.og_patch_nodes.argtypes = [p, i, p]
        lib.og_element_energy.restype = d
        lib.og_element_energy.argtypes = [p, p, d, d, p]
        lib.og_element_egh.argtypes = [p, p, d, d, p, p, p, p, i]
        lib.og_element_mass.argtypes = [p, d, d, p, p, p]
        lib.og_elements.argtypes = [p, p, p, p, i, i, p, p, p, i]
        lib.og_bsr_pattern.restype = i
        lib.og_bsr_pattern.argtypes = [p, p, p]
        lib.og_assemble.argtypes = [p, p, p, p, p, p, d, p, p, p, i]
        lib.og_mass.argtypes = [p, p, p, p, p, p, p]
        lib.og_pcg.restype = i
        lib.og_pcg.argtypes = [i, p, p, p, p, d, p, p, d, i, i, p, p]
        lib.og_kind_scale.argtypes = [i, p, p, p, p, p]
        lib.og_newton_step.restype = i
        lib.og_set_threads.restype = i
        lib.og_set_threads.argtypes = [i]
        lib.og_fix_diagonal.restype = i
        lib.og_fix_diagonal.argtypes = [i, p, p, p, p, p]
        lib.og_newton_direction.restype = i
        lib.og_newton_direction.argtypes = [i, p, p, p, p, p, d, i, i, p, p, p, p, p]
        lib.og_ls_next_alpha.restype = d
        lib.og_ls_next_alpha.argtypes = [i, d, d, d, d, d]
        lib.og_line_search.restype = i
        lib.og_line_search.argtypes = [d, PHI_FN, p, p, p]
        lib.og_newton_step.argtypes = [p, p, p, p, p, p, p, p, p, p]
        lib.og_bezier_patch.argtypes = [p, p, i, p]
        lib.og_bezier_eval.argtypes = [p, d, d, p, p, p]
        lib.og_bezier_sub.argtypes = [p, d, d, d, d, p]
        lib.og_ray_box.restype = i
        lib.og_ray_box.argtypes = [p, p, p, p, p, p, p]
        lib.og_trace_rays.argtypes = [p, p, i, p, p, i, p, p, p, p, p]
        lib.og_ccd_feasible.restype = i
        lib.og_ccd_feasible.argtypes = [p, p, p, p, p, p]
        lib.og_ccd_points.argtypes = [p, p, p, i, p, p, i, p, p, p, p, p]
        _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's independent loops (n <= 0 leaves the count); returns it."""
    return int(_load().og_set_threads(int(n)))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _grid(g) -> Grid:
    return Grid(int(g.nu), int(g.nv), int(bool(g.periodic_u)), int(bool(g.periodic_v)),
                float(g.dxi1), float(g.dxi2))


def _mat(m) -> Material:
    return Material(float(m.young), float(m.poisson), float(m.thickness), float(m.density))


# ------------------------------------------------------------------------------------------
# App. A
# ------------------------------------------------------------------------------------------
def hermite_w(p: int, r: int, t: float, d: int = 0) -> float:
    return _load().og_hermite_w(p, r, float(t), d)


def gauss4():
    x, w = np.zeros(4), np.zeros(4)
    _load().og_gauss4(_ptr(x), _ptr(w))
    return x, w


def shape(dxi1, dxi2, t1, t2):
    """[16, 6] values Phi, Phi_1, Phi_2, Phi_11, Phi_22, Phi_12 of the 16 shape functions."""
    out = np.zeros((16, 6))
    _load().og_shape(float(dxi1), float(dxi2), float(t1), float(t2), _ptr(out))
    return out


def patch_nodes(g, patch: int):
    nd = np.zeros(4, dtype=np.int32)
    _load().og_patch_nodes(C.byref(_grid(g)), int(patch), _ptr(nd))
    return nd


def gather(g, nodal, patch: int):
    """Patch-local 48-vector: the 12 DOFs of the corners 00, 10, 01, 11."""
    nodal = np.asarray(nodal).reshape(-1, 12)
    return nodal[patch_nodes(g, patch)].reshape(48)


# ------------------------------------------------------------------------------------------
# Element level
# ------------------------------------------------------------------------------------------
def element_energy(q48, qb48, dxi1, dxi2, mat) -> float:
    q48, qb48 = _f64(q48), _f64(qb48)
    return _load().og_element_energy(_ptr(q48), _ptr(qb48), float(dxi1), float(dxi2),
                                     C.byref(_mat(mat)))


def element_egh(q48, qb48, dxi1, dxi2, mat, pseudo: bool = False):
    """(E, grad[48], hess[48, 48]) of one patch; local order corner*12 + kind*3 + component.
    pseudo: the pseudo Hessian (App. B) instead of the exact one."""
    q48, qb48 = _f64(q48), _f64(qb48)
    E = np.zeros(1)
    g = np.zeros(48)
    H = np.zeros((48, 48))
    _load().og_element_egh(_ptr(q48), _ptr(qb48), float(dxi1), float(dxi2), C.byref(_mat(mat)),
                           _ptr(E), _ptr(g), _ptr(H), int(bool(pseudo)))
    return float(E[0]), g, H


def element_mass(qb48, dxi1, dxi2, mat):
    qb48 = _f64(qb48)
    m, f = np.zeros((16, 16)), np.zeros(16)
    _load().og_element_mass(_ptr(qb48), float(dxi1), float(dxi2), C.byref(_mat(mat)), _ptr(m), _ptr(f))
    return m, f


def elements(g, mat, rest, q, p0: int = 0, p1: int | None = None, want_hess: bool = True,
             pseudo: bool = False):
    """Per-patch (E[np], grad[np, 48], hess[np, 48, 48]) for patches p0..p1-1."""
    p1 = g.n_patches if p1 is None else p1
    rest, q = _f64(rest).reshape(-1), _f64(q).reshape(-1)
    n = p1 - p0
    E, G = np.zeros(n), np.zeros((n, 48))
    H = np.zeros((n, 48, 48)) if want_hess else None
    _load().og_elements(C.byref(_grid(g)), C.byref(_mat(mat)), _ptr(rest), _ptr(q), p0, p1,
                        _ptr(E), _ptr(G), _ptr(H), int(bool(pseudo)))
    return E, G, H


# ------------------------------------------------------------------------------------------
# Assembly and solver
# ------------------------------------------------------------------------------------------
def bsr_pattern(g):
    lib = _load()
    gg = _grid(g)
    nb = lib.og_bsr_pattern(C.byref(gg), None, None)
    row_ptr = np.zeros(g.n_nodes + 1, dtype=np.int32)
    col = np.zeros(nb, dtype=np.int32)
    lib.og_bsr_pattern(C.byref(gg), _ptr(row_ptr), _ptr(col))
    return row_ptr, col


def assemble(g, mat, rest, q, mass_scale: float = 0.0, want_hess: bool = True, pattern=None,
             pseudo: bool = False):
    """(energy, grad[n_dof], (row_ptr, col, val[nb, 12, 12]) or None): K + mass_scale * M."""
    row_ptr, col = pattern if pattern is not None else bsr_pattern(g)
    rest, q = _f64(rest).reshape(-1), _f64(q).reshape(-1)
    E = np.zeros(1)
    grad = np.zeros(g.n_dof)
    val = np.zeros((col.size, 12, 12)) if want_hess else None
    _load().og_assemble(C.byref(_grid(g)), C.byref(_mat(mat)), _ptr(rest), _ptr(q), _ptr(row_ptr),
                        _ptr(col), float(mass_scale), _ptr(E), _ptr(grad), _ptr(val), int(bool(pseudo)))
    return float(E[0]), grad, ((row_ptr, col, val) if want_hess else None)


def mass(g, mat, rest, pattern=None):
    """Nodal mass as 4x4 scalar blocks [nb, 4, 4] (M = m (x) I3) and gravity factors [n, 4]."""
    row_ptr, col = pattern if pattern is not None else bsr_pattern(g)
    rest = _f64(rest).reshape(-1)
    mval = np.zeros((col.size, 4, 4))
    fs = np.zeros((g.n_nodes, 4))
    _load().og_mass(C.byref(_grid(g)), C.byref(_mat(mat)), _ptr(rest), _ptr(row_ptr), _ptr(col),
                    _ptr(mval), _ptr(fs))
    return mval, fs


def bsr_to_dense(row_ptr, col, val):
    n = row_ptr.size - 1
    bs = val.shape[1]
    A = np.zeros((n * bs, n * bs))
    for i in range(n):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            j = col[k]
            A[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] += val[k]
    return A


def kind_scale(row_ptr, col, val, mask=None):
    """Regulariser scale per DOF kind: mean |A_ii| over free DOFs of each kind [4]."""
    n = row_ptr.size - 1
    val = _f64(val)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.zeros(4)
    _load().og_kind_scale(n, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(m), _ptr(out))
    return out


def pcg(row_ptr, col, val, b, mask=None, tau=0.0, rtol=1e-6, max_iter=1000, fixed_iters=0):
    """Block-Jacobi PCG from x = 0 on A + tau D (12x12 BSR); returns (x, iters, status)."""
    n = row_ptr.size - 1
    val = _f64(val)
    b = _f64(b).reshape(-1)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    dbar = kind_scale(row_ptr, col, val, m)
    x = np.zeros(n * 12)
    it = C.c_int(0)
    st = _load().og_pcg(n, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(m), float(tau), _ptr(dbar),
                        _ptr(b), float(rtol), int(max_iter), int(fixed_iters), _ptr(x), C.byref(it))
    return x, it.value, st


def fix_diagonal(row_ptr, col, val, mask=None, dbar=None):
    """Local part of the regulariser on a copy of val: (fixed val, entries replaced)."""
    n = row_ptr.size - 1
    v = _f64(val).copy()
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    dbar = kind_scale(row_ptr, col, val, m) if dbar is None else _f64(dbar)
    cnt = _load().og_fix_diagonal(n, _ptr(row_ptr), _ptr(col), _ptr(v), _ptr(m), _ptr(dbar))
    return v, cnt


def newton_direction(row_ptr, col, val, rhs, mask=None, tau_carry=0.0, rtol=1e-6, max_iter=1000,
                     fixed_iters=0):
    """Regularised Newton direction (og_newton_direction). Returns (d, status, tau, pcg iterations,
    solves with tau > 0, diagonal entries replaced)."""
    n = row_ptr.size - 1
    val = _f64(val)
    rhs = _f64(rhs).reshape(-1)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    d = np.zeros(n * 12)
    tau = C.c_double(tau_carry)
    it, regs, fixes = C.c_int(0), C.c_int(0), C.c_int(0)
    st = _load().og_newton_direction(n, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(m), _ptr(rhs), float(rtol),
                                     int(max_iter), int(fixed_iters), C.byref(tau), _ptr(d), C.byref(it),
                                     C.byref(regs), C.byref(fixes))
    return d, st, tau.value, it.value, regs.value, fixes.value


def ls_next_alpha(trial, alpha, phi, gd, a_prev=0.0, f_prev=0.0) -> float:
    return float(_load().og_ls_next_alpha(int(trial), float(alpha), float(phi), float(gd), float(a_prev),
                                          float(f_prev)))


def line_search(gd, phi):
    """Armijo backtracking on a Python function phi(alpha). Returns (alpha or None, backtracks,
    the alphas tried)."""
    tried = []

    def cb(a, _ctx):
        tried.append(a)
        return float(phi(a))
    fn = PHI_FN(cb)
    alpha, bt = C.c_double(0.0), C.c_int(0)
    st = _load().og_line_search(float(gd), fn, None, C.byref(alpha), C.byref(bt))
    return (alpha.value if st == 0 else None), bt.value, tried


def step_params(dt=1e-3, gravity=(0.0, 0.0, -9.81), newton_rtol=1e-8, newton_max=50,
                pcg_rtol=1e-6, pcg_max=1000, pcg_fixed_iters=0, pseudo_hessian=False,
                tau_carry=0.0) -> StepParams:
    return StepParams(float(dt), (C.c_double * 3)(*gravity), float(newton_rtol), int(newton_max),
                      float(pcg_rtol), int(pcg_max), int(pcg_fixed_iters), int(bool(pseudo_hessian)),
                      float(tau_carry))


def newton_step(g, mat, rest, q, v, params: StepParams, mask=None, qfix=None, warm=None):
    """One implicit-Euler step. Returns (q_new, v_new, stats dict)."""
    rest = _f64(rest).reshape(-1)
    q = _f64(q).reshape(-1).copy()
    v = _f64(v).reshape(-1).copy()
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    qf = None if qfix is None else _f64(qfix).reshape(-1)
    w = None if warm is None else _f64(warm).reshape(-1)
    st = StepStats()
    _load().og_newton_step(C.byref(_grid(g)), C.byref(_mat(mat)), _ptr(rest), C.byref(params),
                           _ptr(m), _ptr(qf), _ptr(q), _ptr(v), _ptr(w), C.byref(st))
    stats = {f: getattr(st, f) for f, _ in StepStats._fields_}
    return q, v, stats


# ---------------------------------------------------------------------------------------------
# Static ray-patch intersection (Sec. 5)
# ---------------------------------------------------------------------------------------------
RAY_HIT, RAY_LIMIT = 1, 2


def bezier_patch(g, q, patch: int):
    """Bezier control points [4, 4, 3] of one patch (i along theta1, j along theta2)."""
    q = _f64(q).reshape(-1)
    P = np.zeros((4, 4, 3))
    _load().og_bezier_patch(C.byref(_grid(g)), _ptr(q), int(patch), _ptr(P))
    return P


def bezier_eval(P, u: float, v: float):
    """(x, x_u, x_v) of a Bezier patch at local (u, v) (derivatives with respect to theta)."""
    P = _f64(P)
    x, xu, xv = np.zeros(3), np.zeros(3), np.zeros(3)
    _load().og_bezier_eval(_ptr(P), float(u), float(v), _ptr(x), _ptr(xu), _ptr(xv))
    return x, xu, xv


def bezier_sub(P, u0, u1, v0, v1):
    """Control points [4, 4, 3] of the sub-patch [u0, u1] x [v0, v1] (De Casteljau)."""
    P = _f64(P)
    S = np.zeros((4, 4, 3))
    _load().og_bezier_sub(_ptr(P), float(u0), float(u1), float(v0), float(v1), _ptr(S))
    return S


def ray_box(S, origin, direction):
    """(hit, tau_min, tau_max, largest box side) of Eq. ineqray for control points S [4, 4, 3]."""
    S, o, d = _f64(S), _f64(origin), _f64(direction)
    inv = np.array([1.0 / x if x != 0.0 else 0.0 for x in d])
    t0, t1, ext = C.c_double(), C.c_double(), C.c_double()
    hit = _load().og_ray_box(_ptr(S), _ptr(o), _ptr(d), _ptr(inv), C.byref(t0), C.byref(t1), C.byref(ext))
    return bool(hit), t0.value, t1.value, ext.value


def trace_rays(g, q, origins, dirs, use_newton: bool = True, want_stats: bool = False):
    """Nearest hits of rays o + tau d (unit d) with the shell.

    Returns (tau [n] (inf on a miss), patch [n] (-1), uv [n, 2] local parameters, flags [n]
    (RAY_HIT, RAY_LIMIT)) and, with want_stats, stats [n, 4] = (candidates split, peak heap size,
    sub-patch boxes formed with the patch roots, Newton iterations).
    """
    q = _f64(q).reshape(-1)
    origins, dirs = _f64(origins).reshape(-1, 3), _f64(dirs).reshape(-1, 3)
    n = origins.shape[0]
    tau, uv = np.zeros(n), np.zeros((n, 2))
    patch, flags = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
    stats = np.zeros((n, 4), dtype=np.int32) if want_stats else None
    _load().og_trace_rays(C.byref(_grid(g)), _ptr(q), n, _ptr(origins), _ptr(dirs), int(bool(use_newton)),
                          _ptr(tau), _ptr(patch), _ptr(uv), _ptr(flags), _ptr(stats))
    out = (tau, patch, uv, flags)
    return out + (stats,) if want_stats else out


# ---------------------------------------------------------------------------------------------
# Point-patch continuous collision detection (Sec. 5, dynamic ray-patch intersection)
# ---------------------------------------------------------------------------------------------
def ccd_feasible(S, dS, x0, dx):
    """Feasible normalised times of Eq. ineqccd for the moving net S + s dS ([4, 4, 3] each) and
    the point x0 + s dx: list of closed intervals (lo, hi) in [0, 1], sorted."""
    S, dS, x0, dx = _f64(S), _f64(dS), _f64(x0), _f64(dx)
    lo, hi = np.zeros(8), np.zeros(8)
    n = _load().og_ccd_feasible(_ptr(S), _ptr(dS), _ptr(x0), _ptr(dx), _ptr(lo), _ptr(hi))
    return [(lo[i], hi[i]) for i in range(n)]


def ccd_points(g, q, dq, x0s, dxs, use_newton: bool = True, want_stats: bool = False):
    """Earliest contact of points x0 + s dx (s in [0, 1]) with the shell moving from q to q + dq.

    Returns (s [n] (inf: no contact), patch [n] (-1), uv [n, 2], flags [n] (RAY_HIT, RAY_LIMIT))
    and, with want_stats, stats [n, 4] = (splits, peak heap size, feasibility tests with the patch
    roots that passed the swept-box test, Newton iterations).
    """
    q, dq = _f64(q).reshape(-1), _f64(dq).reshape(-1)
    x0s, dxs = _f64(x0s).reshape(-1, 3), _f64(dxs).reshape(-1, 3)
    n = x0s.shape[0]
    s, uv = np.zeros(n), np.zeros((n, 2))
    patch, flags = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
    stats = np.zeros((n, 4), dtype=np.int32) if want_stats else None
    _load().og_ccd_points(C.byref(_grid(g)), _ptr(q), _ptr(dq), n, _ptr(x0s), _ptr(dxs), int(bool(use_newton)),
                          _ptr(s), _ptr(patch), _ptr(uv), _ptr(flags), _ptr(stats))
    out = (s, patch, uv, flags)
    return out + (stats,) if want_stats else out
