"""Thin ctypes binding of libbhem (include/bhem.h): argument marshalling only.

Every step of the BHEM hot path runs in the library's CUDA kernels; this module passes pointers
(torch CUDA tensors, or host numpy arrays where the C ABI accepts host buffers) and sizes. There
is no CPU fallback: if the library cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

PREC = {"fp64": 0, "mixed": 1}
HESS = {"exact": 0, "pseudo": 1}
ASM = {"atomic": 0, "color": 1}
SPMV = {"auto": 0, "plain": 1, "tma": 2}
SOLVER = {"pcg": 0, "direct": 1}
STATUS = {0: "SHELL_OK", 1: "SHELL_ERR_ARG", 2: "SHELL_ERR_CUDA", 3: "SHELL_ERR_OOM",
          4: "SHELL_ERR_DEGENERATE", 5: "SHELL_ERR_NONFINITE", 6: "SHELL_ERR_NOT_CONVERGED",
          7: "SHELL_ERR_LINESEARCH", 8: "SHELL_ERR_INDEFINITE", 9: "SHELL_ERR_TIMEOUT"}


class ShellError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class shell_grid(C.Structure):
    _fields_ = [("nu", C.c_int), ("nv", C.c_int), ("periodic_u", C.c_int), ("periodic_v", C.c_int),
                ("dxi1", C.c_double), ("dxi2", C.c_double)]


class shell_material(C.Structure):
    _fields_ = [("young", C.c_double), ("poisson", C.c_double), ("thickness", C.c_double),
                ("density", C.c_double)]


class shell_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("hessian", C.c_int), ("assembly", C.c_int),
                ("spmv", C.c_int), ("solver", C.c_int)]


class shell_step_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("newton_rtol", C.c_double),
                ("newton_max", C.c_int), ("pcg_rtol", C.c_double), ("pcg_max", C.c_int),
                ("pcg_fixed_iters", C.c_int), ("tau_carry", C.c_double)]


class shell_step_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("pcg_iters_total", C.c_int),
                ("ls_backtracks", C.c_int), ("regularizations", C.c_int), ("status", C.c_int),
                ("diag_fixes", C.c_int), ("res0", C.c_double), ("res_final", C.c_double),
                ("tau_final", C.c_double)]


class shell_batch_info_t(C.Structure):
    _fields_ = [("n_shells", C.c_int), ("n_nodes", C.c_int), ("n_patches", C.c_int), ("n_blocks", C.c_int),
                ("n_dof", C.c_int), ("patches_per_item", C.c_int), ("assembly", C.c_int),
                ("kernel_launches", C.c_longlong)]


class shell_info_t(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("n_patches", C.c_int), ("n_blocks", C.c_int),
                ("n_dof", C.c_int)]


def library_path() -> str:
    return _build.LIB


def load():
    """Loads libbhem.so, building it with nvcc first when it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libbhem.so not found at {path}")
            lib = C.CDLL(path)
            p, i, d, f, ll = C.c_void_p, C.c_int, C.c_double, C.c_float, C.c_longlong
            sigs = {
                "shell_create": [p, p, p, p, p, p],
                "shell_destroy": [p],
                "shell_info": [p, p],
                "shell_grid_colours": [p, p],
                "shell_set_wait_budget": [p, i],
                "shell_element_egh": [p, p, i, p, p, p],
                "shell_energy_grad_hess": [p, p, d, p, p, i],
                "shell_get_bsr": [p, p, p, p, p],
                "shell_get_mass": [p, p, p],
                "shell_pcg_solve": [p, p, d, p, p, d, i, i, p, p],
                "shell_newton_step": [p, p, p, p, p, p, p, p],
                "shell_spmv": [p, p, i, p],
                "shell_kernel_launches": [p, p],
                "shell_energy_grad_noalloc": [p, p, p, p, p, p, p],
                "shell_batch_create": [i, p, p, p, p, p, p],
                "shell_batch_destroy": [p],
                "shell_batch_info": [p, p, p],
                "shell_batch_autotune": [p, p, i],
                "shell_batch_newton_step": [p, p, p, p, p, p, p, p],
                "shell_mlp_create": [i, p, p],
                "shell_mlp_destroy": [p],
                "shell_mlp_param_count": [p],
                "shell_mlp_set_params": [p, p],
                "shell_mlp_get_params": [p, p, p],
                "shell_mlp_set_normalization": [p, p, p, p, p],
                "shell_mlp_column_stats": [p, p, ll, i, p, p],
                "shell_mlp_forward": [p, p, i, p],
                "shell_mlp_gradients": [p, p, p, ll, p, i, p],
                "shell_mlp_train_step": [p, p, p, ll, p, i, f, p],
                "shell_mlp_kernel_launches": [p, p],
                "shell_mlp_set_wait_budget": [p, C.c_int],
                "shell_node_features": [p, p, p, p],
                "shell_warm_targets": [ll, p, p, p, d, p, p],
                "shell_mlp_warm_start": [p, p, p, p, d, p],
                "shell_measure_fma_peak": [i, i, p, p],
                "shell_measure_mma_peak": [i, i, p, p],
                "shell_trace_rays": [p, p, ll, p, p, i, p, p, p, p, p],
                "shell_ccd_points": [p, p, p, ll, p, p, i, p, p, p, p, p],
            }
            for name, args in sigs.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = C.c_int
            lib.shell_last_error.restype = C.c_char_p
            lib.shell_last_error.argtypes = []
            _lib = lib
        return _lib


def _check(st: int):
    if st != 0:
        raise ShellError(st, load().shell_last_error().decode())


def grid_colours(nu: int, nv: int, periodic_u: int = 0, periodic_v: int = 0):
    """Colour of every patch of the colour-ordered assembly (``shell_grid_colours``), [nv, nu]."""
    g = shell_grid(nu, nv, periodic_u, periodic_v, 1.0, 1.0)
    out = np.zeros(nu * nv, dtype=np.int32)
    _check(load().shell_grid_colours(C.byref(g), out.ctypes.data_as(C.c_void_p)))
    return out.reshape(nv, nu)


def _ptr(t):
    """Raw pointer of a torch tensor (device or host) or numpy array; None stays NULL."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


class _DevArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream, C.c_void_p(stream.cuda_stream)


RAY_VARIANT = {"midpoint": 0, "newton": 1}
RAY_HIT, RAY_LIMIT, RAY_OVERFLOW, RAY_HEAP = 1, 2, 4, 256


def step_params(dt=1e-3, gravity=(0.0, 0.0, -9.81), newton_rtol=1e-8, newton_max=50,
                pcg_rtol=1e-6, pcg_max=1000, pcg_fixed_iters=0, tau_carry=0.0) -> shell_step_params:
    return shell_step_params(float(dt), (C.c_double * 3)(*gravity), float(newton_rtol),
                             int(newton_max), float(pcg_rtol), int(pcg_max), int(pcg_fixed_iters),
                             float(tau_carry))


def energy_grad_noalloc(grid, material, rest, q, energy, grad=None, stream=None):
    """shell_energy_grad_noalloc: elastic energy (into ``energy``, a 1-element FP64 CUDA tensor)
    and gradient (into ``grad`` or None) without any device allocation by the library."""
    _, sh = _stream_handle(stream)
    g = shell_grid(int(grid.nu), int(grid.nv), int(bool(grid.periodic_u)), int(bool(grid.periodic_v)),
                   float(grid.dxi1), float(grid.dxi2))
    m = shell_material(float(material.young), float(material.poisson), float(material.thickness),
                       float(material.density))
    _check(load().shell_energy_grad_noalloc(C.byref(g), C.byref(m), _ptr(rest), _ptr(q), _ptr(energy),
                                            _ptr(grad), sh))


class Shell:
    """One BHEM shell on the current CUDA device (wraps shell_create ... shell_destroy)."""

    def __init__(self, grid, material, rest, precision="mixed", hessian="exact",
                 assembly="atomic", stream=None, spmv="auto", solver="pcg"):
        import torch
        lib = load()
        self.grid = grid
        self.material = material
        self.precision = precision
        self.stream, sh = _stream_handle(stream)
        g = shell_grid(int(grid.nu), int(grid.nv), int(bool(grid.periodic_u)),
                       int(bool(grid.periodic_v)), float(grid.dxi1), float(grid.dxi2))
        m = shell_material(float(material.young), float(material.poisson),
                           float(material.thickness), float(material.density))
        o = shell_options(PREC[precision], HESS[hessian], ASM[assembly], SPMV[spmv], SOLVER[solver])
        if isinstance(rest, np.ndarray):
            rest = np.ascontiguousarray(rest, dtype=np.float64)
        else:
            rest = rest.contiguous().to(torch.float64)
        self._h = C.c_void_p()
        _check(lib.shell_create(C.byref(g), C.byref(m), _ptr(rest), C.byref(o), sh, C.byref(self._h)))
        info = shell_info_t()
        _check(lib.shell_info(self._h, C.byref(info)))
        self.n_nodes, self.n_patches = info.n_nodes, info.n_patches
        self.n_blocks, self.n_dof = info.n_blocks, info.n_dof

    # ------------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().shell_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------------------------
    def element_egh(self, q, precision=None, want=("e", "g", "h")):
        """Unassembled per-patch (E [np], grad [np, 48], hess [np, 48, 48]) as torch tensors."""
        import torch
        prec = PREC[precision or self.precision]
        dev = q.device
        E = torch.empty(self.n_patches, dtype=torch.float64, device=dev) if "e" in want else None
        G = torch.empty(self.n_patches, 48, dtype=torch.float64, device=dev) if "g" in want else None
        hd = torch.float64 if prec == 0 else torch.float32
        H = torch.empty(self.n_patches, 48, 48, dtype=hd, device=dev) if "h" in want else None
        _check(load().shell_element_egh(self._h, _ptr(q), prec, _ptr(E), _ptr(G), _ptr(H)))
        return E, G, H

    def energy_grad_hess(self, q, mass_scale=0.0, want_hessian=True, want_energy=True,
                         want_grad=True):
        """Assembled elastic energy (device scalar), gradient [n_dof]; Hessian into the BSR."""
        import torch
        dev = q.device
        E = torch.empty(1, dtype=torch.float64, device=dev) if want_energy else None
        G = torch.empty(self.n_dof, dtype=torch.float64, device=dev) if want_grad else None
        _check(load().shell_energy_grad_hess(self._h, _ptr(q), float(mass_scale), _ptr(E), _ptr(G),
                                             int(bool(want_hessian))))
        return E, G

    def bsr(self):
        """Copies of (row_ptr [n+1], col [nb], val [nb, 12, 12]) of the assembled matrix."""
        import torch
        rp, col, val, f64 = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_int()
        _check(load().shell_get_bsr(self._h, C.byref(rp), C.byref(col), C.byref(val), C.byref(f64)))
        dev = torch.device("cuda", torch.cuda.current_device())
        t_rp = torch.as_tensor(_DevArray(rp.value, (self.n_nodes + 1,), "<i4"), device=dev).clone()
        t_col = torch.as_tensor(_DevArray(col.value, (self.n_blocks,), "<i4"), device=dev).clone()
        t_val = torch.as_tensor(_DevArray(val.value, (self.n_blocks, 12, 12), "<f8" if f64.value else "<f4"),
                                device=dev).clone()
        return t_rp, t_col, t_val

    def mass(self):
        """Copies of the 4x4-block consistent mass [nb, 4, 4] and gravity factors [n, 4]."""
        import torch
        mb, fg = C.c_void_p(), C.c_void_p()
        _check(load().shell_get_mass(self._h, C.byref(mb), C.byref(fg)))
        dev = torch.device("cuda", torch.cuda.current_device())
        M = torch.as_tensor(_DevArray(mb.value, (self.n_blocks, 4, 4), "<f8"), device=dev).clone()
        F = torch.as_tensor(_DevArray(fg.value, (self.n_nodes, 4), "<f8"), device=dev).clone()
        return M, F

    def pcg_solve(self, rhs, mask=None, tau=0.0, rtol=1e-6, max_iter=1000, fixed_iters=0):
        import torch
        x = torch.empty_like(rhs)
        it, neg = C.c_int(), C.c_int()
        _check(load().shell_pcg_solve(self._h, _ptr(mask), float(tau), _ptr(rhs), _ptr(x), float(rtol),
                                      int(max_iter), int(fixed_iters), C.byref(it), C.byref(neg)))
        return x, it.value, neg.value

    def set_wait_budget(self, polls: int):
        """shell_set_wait_budget: polls of each bounded device-side wait (< 0: the default)."""
        _check(load().shell_set_wait_budget(self._h, int(polls)))

    def kernel_launches(self) -> int:
        n = C.c_longlong()
        _check(load().shell_kernel_launches(self._h, C.byref(n)))
        return n.value

    def spmv(self, x, y=None):
        """y = A x with the assembled BSR on the shell's stream; x, y FP64, or FP32 for a mixed
        shell (then one kernel launch)."""
        import torch
        if y is None:
            y = torch.empty(x.shape, dtype=x.dtype, device=x.device)
        _check(load().shell_spmv(self._h, _ptr(x), int(x.dtype == torch.float32), _ptr(y)))
        return y

    def trace_rays(self, q, origins, dirs, variant="newton", out=None, want_stats=False):
        """Nearest hits of rays o + tau d (unit d) with the shell at q (Sec. 5), on the shell's
        stream. q [n_dof], origins / dirs [n, 3]: FP64 CUDA tensors. Returns a dict of CUDA tensors
        tau [n] (inf on a miss), patch [n] (-1), uv [n, 2], flags [n] (RAY_HIT, RAY_LIMIT,
        RAY_OVERFLOW bits) and, with want_stats, stats [n, 4] (candidates split, peak heap size,
        candidate boxes formed including one root box per patch, Newton iterations).
        out: a dict of the same tensors to fill instead of allocating."""
        import torch
        n = origins.shape[0]
        dev = origins.device
        if out is None:
            out = {"tau": torch.empty(n, dtype=torch.float64, device=dev),
                   "patch": torch.empty(n, dtype=torch.int32, device=dev),
                   "uv": torch.empty((n, 2), dtype=torch.float64, device=dev),
                   "flags": torch.empty(n, dtype=torch.int32, device=dev)}
            if want_stats:
                out["stats"] = torch.empty((n, 4), dtype=torch.int32, device=dev)
        _check(load().shell_trace_rays(self._h, _ptr(q), int(n), _ptr(origins), _ptr(dirs), RAY_VARIANT[variant],
                                       _ptr(out["tau"]), _ptr(out["patch"]), _ptr(out["uv"]), _ptr(out["flags"]),
                                       _ptr(out.get("stats"))))
        return out

    def ccd_points(self, q, dq, x0, dx, variant="newton", out=None, want_stats=False):
        """Earliest contact of points moving from x0 to x0 + dx with the shell moving from q to
        q + dq over one step (Sec. 5, Eq. ineqccd), on the shell's stream. FP64 CUDA tensors:
        q, dq [n_dof], x0, dx [n, 3]. Returns a dict of CUDA tensors s [n] (normalised contact
        time in [0, 1], inf when none), patch [n] (-1), uv [n, 2], flags [n] and, with
        want_stats, stats [n, 4]. out: a dict of the same tensors to fill instead."""
        import torch
        n = x0.shape[0]
        dev = x0.device
        if out is None:
            out = {"s": torch.empty(n, dtype=torch.float64, device=dev),
                   "patch": torch.empty(n, dtype=torch.int32, device=dev),
                   "uv": torch.empty((n, 2), dtype=torch.float64, device=dev),
                   "flags": torch.empty(n, dtype=torch.int32, device=dev)}
            if want_stats:
                out["stats"] = torch.empty((n, 4), dtype=torch.int32, device=dev)
        _check(load().shell_ccd_points(self._h, _ptr(q), _ptr(dq), int(n), _ptr(x0), _ptr(dx), RAY_VARIANT[variant],
                                       _ptr(out["s"]), _ptr(out["patch"]), _ptr(out["uv"]), _ptr(out["flags"]),
                                       _ptr(out.get("stats"))))
        return out

    def newton_step(self, q, v, params: shell_step_params, mask=None, q_fixed=None, warm=None,
                    raise_on_error=False):
        """In-place implicit-Euler step on q, v (torch CUDA tensors or host numpy arrays)."""
        st = shell_step_stats()
        rc = load().shell_newton_step(self._h, C.byref(params), _ptr(mask), _ptr(q_fixed), _ptr(q),
                                      _ptr(v), _ptr(warm), C.byref(st))
        stats = {f: getattr(st, f) for f, _ in shell_step_stats._fields_}
        if rc != 0 and (raise_on_error or rc not in (6, 7, 8)):
            raise ShellError(rc, load().shell_last_error().decode())
        return stats


class Batch:
    """Many shells stepped together (shell_batch_*): shells = [(grid, material, rest), ...].
    State arrays are the shells' arrays concatenated; ``node_offsets[s]`` is shell s's first node."""

    def __init__(self, shells, stream=None, assembly="atomic"):
        import torch
        lib = load()
        S = len(shells)
        self.grids = (shell_grid * S)()
        self.mats = (shell_material * S)()
        for k, (g, m, _) in enumerate(shells):
            self.grids[k] = shell_grid(int(g.nu), int(g.nv), int(bool(g.periodic_u)), int(bool(g.periodic_v)),
                                       float(g.dxi1), float(g.dxi2))
            self.mats[k] = shell_material(float(m.young), float(m.poisson), float(m.thickness), float(m.density))
        rest = np.concatenate([np.ascontiguousarray(r, dtype=np.float64).reshape(-1) for _, _, r in shells])
        stream_obj, sh = (None, C.c_void_p(None)) if stream is None else _stream_handle(stream)
        self.stream = stream_obj
        self._h = C.c_void_p()
        opts = shell_options(PREC["mixed"], HESS["exact"], ASM[assembly], 0, 0)
        _check(lib.shell_batch_create(S, self.grids, self.mats, _ptr(rest), C.byref(opts), sh, C.byref(self._h)))
        self.n_shells = S
        self.node_offsets = np.zeros(S + 1, dtype=np.int32)
        info = self.info()
        self.n_nodes, self.n_patches, self.n_dof = info["n_nodes"], info["n_patches"], info["n_dof"]

    def info(self):
        inf = shell_batch_info_t()
        _check(load().shell_batch_info(self._h, C.byref(inf), _ptr(self.node_offsets)))
        return {f: getattr(inf, f) for f, _ in shell_batch_info_t._fields_}

    def autotune(self, q, repeats=3):
        _check(load().shell_batch_autotune(self._h, _ptr(q), int(repeats)))
        return self.info()

    def newton_step(self, q, v, params: shell_step_params, mask=None, q_fixed=None, warm=None,
                    raise_on_error=False):
        stats = (shell_step_stats * self.n_shells)()
        rc = load().shell_batch_newton_step(self._h, C.byref(params), _ptr(mask), _ptr(q_fixed), _ptr(q),
                                            _ptr(v), _ptr(warm), stats)
        out = [{f: getattr(s, f) for f, _ in shell_step_stats._fields_} for s in stats]
        if rc != 0 and (raise_on_error or rc not in (6, 7, 8)):
            raise ShellError(rc, load().shell_last_error().decode())
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().shell_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Mlp:
    """The warm-start network (shell_mlp_*): a per-node MLP 28 -> 256 -> 256 -> 256 -> 12 whose
    forward, backward and Adam steps run in the library's kernels. Parameters are exchanged as
    one packed FP32 numpy array (per layer W [fan_out, fan_in] row-major, then b)."""

    N_IN, N_OUT, LAYERS = 28, 12, ((28, 256), (256, 256), (256, 256), (256, 12))

    def __init__(self, max_rows, stream=None):
        lib = load()
        self.stream, sh = _stream_handle(stream)
        self.max_rows = int(max_rows)
        self._h = C.c_void_p()
        _check(lib.shell_mlp_create(self.max_rows, sh, C.byref(self._h)))
        n = C.c_longlong()
        _check(lib.shell_mlp_param_count(C.byref(n)))
        self.n_params = n.value

    def close(self):
        if getattr(self, "_h", None):
            load().shell_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32)
        if params.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {params.size}")
        _check(load().shell_mlp_set_params(self._h, _ptr(params)))

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(load().shell_mlp_get_params(self._h, _ptr(out), None))
        return out

    def get_grads(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(load().shell_mlp_get_params(self._h, None, _ptr(out)))
        return out

    def set_normalization(self, in_mean, in_std, out_mean, out_std):
        a = [np.ascontiguousarray(x, dtype=np.float32) for x in (in_mean, in_std, out_mean, out_std)]
        _check(load().shell_mlp_set_normalization(self._h, *[_ptr(x) for x in a]))

    def column_stats(self, X):
        """(mean, std) of each column of a [rows, cols] FP32 CUDA tensor."""
        rows, cols = X.shape
        mean, std = np.empty(cols), np.empty(cols)
        _check(load().shell_mlp_column_stats(self._h, _ptr(X), int(rows), int(cols), _ptr(mean), _ptr(std)))
        return mean, std

    def forward(self, X, Y=None):
        import torch
        if Y is None:
            Y = torch.empty(X.shape[0], self.N_OUT, dtype=torch.float32, device=X.device)
        _check(load().shell_mlp_forward(self._h, _ptr(X), int(X.shape[0]), _ptr(Y)))
        return Y

    def gradients(self, X, T, idx=None, rows=None, want_loss=True):
        rows = int(X.shape[0] if idx is None else idx.shape[0]) if rows is None else int(rows)
        loss = C.c_double()
        _check(load().shell_mlp_gradients(self._h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(idx), rows,
                                          C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def train_step(self, X, T, idx, lr, want_loss=False):
        loss = C.c_double()
        _check(load().shell_mlp_train_step(self._h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(idx),
                                           int(idx.shape[0]), float(lr), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def kernel_launches(self) -> int:
        n = C.c_longlong()
        _check(load().shell_mlp_kernel_launches(self._h, C.byref(n)))
        return n.value

    def set_wait_budget(self, polls: int) -> None:
        """Bound of the tensor-core kernels' device-side waits (< 0: default; 0: every wait expires)."""
        _check(load().shell_mlp_set_wait_budget(self._h, int(polls)))

    def warm_start(self, shell, q, v, dt, warm=None):
        """q + dt v + network(features) for a shell state (FP64 CUDA tensors), on the shell's stream."""
        import torch
        if warm is None:
            warm = torch.empty_like(q)
        _check(load().shell_mlp_warm_start(self._h, shell._h, _ptr(q), _ptr(v), float(dt), _ptr(warm)))
        return warm


def inertial_warm_start(shell, q, v, dt, warm=None):
    """warm = q + dt v (shell_mlp_warm_start without a network), on the shell's stream."""
    import torch
    if warm is None:
        warm = torch.empty_like(q)
    _check(load().shell_mlp_warm_start(None, shell._h, _ptr(q), _ptr(v), float(dt), _ptr(warm)))
    return warm


def node_features(shell, q, v, X=None):
    """Node features [n_nodes, 28] (FP32 CUDA tensor) of a shell state, on the shell's stream."""
    import torch
    if X is None:
        X = torch.empty(shell.n_nodes, Mlp.N_IN, dtype=torch.float32, device=q.device)
    _check(load().shell_node_features(shell._h, _ptr(q), _ptr(v), _ptr(X)))
    return X


def warm_targets(q_next, q, v, dt, T=None, stream=None):
    """T = q_next - q - dt v as FP32 (CUDA tensors of n_dof entries)."""
    import torch
    if T is None:
        T = torch.empty(q.numel(), dtype=torch.float32, device=q.device)
    _, sh = _stream_handle(stream)
    _check(load().shell_warm_targets(int(q.numel()), _ptr(q_next), _ptr(q), _ptr(v), float(dt), _ptr(T), sh))
    return T


def measure_mma_peak(kind: int, iters: int, stream=None) -> float:
    """Measured mma.sync throughput in FLOP/s (shell_measure_mma_peak; 0: TF32, 1: BF16)."""
    _, sh = _stream_handle(stream)
    out = C.c_double()
    _check(load().shell_measure_mma_peak(int(kind), int(iters), sh, C.byref(out)))
    return out.value


def measure_fma_peak(fp64: bool, iters: int, stream=None) -> float:
    """Measured FP32 or FP64 FMA throughput of the current device in FLOP/s
    (shell_measure_fma_peak)."""
    _, sh = _stream_handle(stream)
    out = C.c_double()
    _check(load().shell_measure_fma_peak(int(bool(fp64)), int(iters), sh, C.byref(out)))
    return out.value
