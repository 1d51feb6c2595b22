"""Seeded synthetic inputs for BHEM shells: grids, rest DOFs, deformed states, prescribed DOFs.

This module produces input arrays only. It holds none of the element, assembly or solver
arithmetic; the CUDA library and the CPU oracle each compute everything from these arrays on
their own.

Conventions (Sec. 4.1, Eq. hermite / Eq. shape):
  * A grid of ``nu x nv`` bicubic Hermite patches. Nodes are indexed ``j * n1 + i`` with
    ``i`` along xi^1 (``n1 = nu + 1``, or ``nu`` when periodic in u) and ``j`` along xi^2.
  * Every node stores 12 generalised coordinates ``[x, x_,1, x_,2, x_,12]`` (each in R^3);
    derivative DOFs are derivatives with respect to the global parameters xi^1, xi^2.
  * ``dxi1``, ``dxi2`` are the parameter extents of one patch.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DOF_PER_NODE = 12


@dataclasses.dataclass(frozen=True)
class Grid:
    nu: int
    nv: int
    periodic_u: bool
    periodic_v: bool
    dxi1: float
    dxi2: float

    @property
    def n1(self) -> int:
        return self.nu if self.periodic_u else self.nu + 1

    @property
    def n2(self) -> int:
        return self.nv if self.periodic_v else self.nv + 1

    @property
    def n_nodes(self) -> int:
        return self.n1 * self.n2

    @property
    def n_patches(self) -> int:
        return self.nu * self.nv

    @property
    def n_dof(self) -> int:
        return DOF_PER_NODE * self.n_nodes


@dataclasses.dataclass(frozen=True)
class Material:
    young: float
    poisson: float
    thickness: float
    density: float


def flat_sheet(nu: int, nv: int, l1: float = 1.0, l2: float = 1.0):
    """Flat rectangular sheet in the z=0 plane; xi = rest coordinates in metres."""
    g = Grid(nu, nv, False, False, l1 / nu, l2 / nv)
    rest = np.zeros((g.n_nodes, DOF_PER_NODE))
    j, i = np.meshgrid(np.arange(g.n2), np.arange(g.n1), indexing="ij")
    rest[:, 0] = (i * g.dxi1).ravel()
    rest[:, 1] = (j * g.dxi2).ravel()
    rest[:, 3] = 1.0   # x_,1 = e1
    rest[:, 7] = 1.0   # x_,2 = e2
    return g, rest


def annulus(nu: int, nv: int, r0: float = 0.2, r1: float = 0.7):
    """Flat annulus, periodic in u: xi^1 = angle in [0, 2 pi), xi^2 = radius in [r0, r1].

    Nodal values are the exact polar map and its derivatives, so the rest midsurface is the
    bicubic Hermite interpolant of the circle-sector geometry (C^1 across patches).
    """
    g = Grid(nu, nv, True, False, 2.0 * math.pi / nu, (r1 - r0) / nv)
    j, i = np.meshgrid(np.arange(g.n2), np.arange(g.n1), indexing="ij")
    th = (i * g.dxi1).ravel()
    r = (r0 + j * g.dxi2).ravel()
    c, s = np.cos(th), np.sin(th)
    rest = np.zeros((g.n_nodes, DOF_PER_NODE))
    rest[:, 0], rest[:, 1] = r * c, r * s
    rest[:, 3], rest[:, 4] = -r * s, r * c
    rest[:, 6], rest[:, 7] = c, s
    rest[:, 9], rest[:, 10] = -s, c
    return g, rest


def cylinder(nu: int, nv: int, radius: float = 0.3, length: float = 1.0):
    """Cylinder about the z axis, periodic in u: xi^1 = angle in [0, 2 pi), xi^2 = height in
    [0, length]. Nodal values are the exact map and its derivatives."""
    g = Grid(nu, nv, True, False, 2.0 * math.pi / nu, length / nv)
    j, i = np.meshgrid(np.arange(g.n2), np.arange(g.n1), indexing="ij")
    th = (i * g.dxi1).ravel()
    c, s = np.cos(th), np.sin(th)
    rest = np.zeros((g.n_nodes, DOF_PER_NODE))
    rest[:, 0], rest[:, 1], rest[:, 2] = radius * c, radius * s, (j * g.dxi2).ravel()
    rest[:, 3], rest[:, 4] = -radius * s, radius * c
    rest[:, 8] = 1.0
    return g, rest


def node_params(g: Grid, xi0=(0.0, 0.0)):
    """Parameter coordinates (xi^1, xi^2) of every node."""
    j, i = np.meshgrid(np.arange(g.n2), np.arange(g.n1), indexing="ij")
    return xi0[0] + (i * g.dxi1).ravel(), xi0[1] + (j * g.dxi2).ravel()


def noisy(rest: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """rest + N(0, sigma^2) on all 12 DOFs of every node (PCG64, seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rest + rng.normal(0.0, sigma, size=rest.shape)


def sinusoid_displacement(s: np.ndarray, t: np.ndarray, ds_dxi1: float, dt_dxi2: float,
                          seed: int, amplitude: float = 0.05, n_terms: int = 8):
    """Smooth field u(s,t) = sum_k A_k sin(2 pi (m_k s + n_k t) + phi_k) per component.

    ``s``, ``t`` are normalised coordinates, linear in xi^1, xi^2 with the given slopes.
    Integer wave numbers m_k, n_k in [1, 4] keep the field periodic in s and t. Returns the
    12 nodal DOFs of the displacement [u, u_,1, u_,2, u_,12] (analytic derivatives) with the
    amplitudes scaled so that max over nodes of |u| equals ``amplitude``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    m = rng.integers(1, 5, size=(3, n_terms))
    n = rng.integers(1, 5, size=(3, n_terms))
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(3, n_terms))
    amp = rng.normal(0.0, 1.0, size=(3, n_terms))
    out = np.zeros((s.size, DOF_PER_NODE))
    for c in range(3):
        for k in range(n_terms):
            arg = 2.0 * math.pi * (m[c, k] * s + n[c, k] * t) + ph[c, k]
            ks, kt = 2.0 * math.pi * m[c, k] * ds_dxi1, 2.0 * math.pi * n[c, k] * dt_dxi2
            out[:, c] += amp[c, k] * np.sin(arg)
            out[:, 3 + c] += amp[c, k] * ks * np.cos(arg)
            out[:, 6 + c] += amp[c, k] * kt * np.cos(arg)
            out[:, 9 + c] += -amp[c, k] * ks * kt * np.sin(arg)
    umax = np.max(np.linalg.norm(out[:, 0:3], axis=1))
    return out * (amplitude / umax)


# ---------------------------------------------------------------------------------------
# Workloads (shapes of the paper's 10x10 locking, 30x30 twisting and 280x5 parasol scenes)
# ---------------------------------------------------------------------------------------

SHEET_MATERIAL = Material(young=1e5, poisson=0.3, thickness=1e-3, density=200.0)


def sheet_noisy(n: int = 10, sigma: float = 1e-3, seed: int = 1):
    """n x n patch, 1 m x 1 m sheet with N(0, sigma) noise on all 12 DOFs per node."""
    g, rest = flat_sheet(n, n)
    return g, rest, noisy(rest, sigma, seed)


def sheet_sinusoid(n: int = 256, seed: int = 3, amplitude: float = 0.05):
    """n x n patch 1 m sheet displaced by the smooth 8-term sinusoid field (5 cm max)."""
    g, rest = flat_sheet(n, n)
    x1, x2 = node_params(g)
    u = sinusoid_displacement(x1, x2, 1.0, 1.0, seed, amplitude)
    return g, rest, rest + u


def annulus_sinusoid(nu: int = 280, nv: int = 5, seed: int = 3, amplitude: float = 0.05,
                     r0: float = 0.2, r1: float = 0.7):
    """Periodic annular strip displaced by the sinusoid field in (xi^1 / 2 pi, (xi^2-r0)/(r1-r0))."""
    g, rest = annulus(nu, nv, r0, r1)
    x1, x2 = node_params(g, (0.0, r0))
    u = sinusoid_displacement(x1 / (2.0 * math.pi), (x2 - r0) / (r1 - r0),
                              1.0 / (2.0 * math.pi), 1.0 / (r1 - r0), seed, amplitude)
    return g, rest, rest + u


def corner_nodes(g: Grid):
    """Node ids of the corners (0,0), (1,0), (0,1), (1,1) of a non-periodic grid."""
    n1, n2 = g.n1, g.n2
    return [0, n1 - 1, (n2 - 1) * n1, n2 * n1 - 1]


def pinned_mask(g: Grid, nodes, kinds=(0,)):
    """Prescribed-DOF mask (uint8 [nodes*12]) fixing the given DOF kinds (0=x,1=x_1,2=x_2,3=x_12)."""
    mask = np.zeros(g.n_dof, dtype=np.uint8)
    for nd in nodes:
        for k in kinds:
            mask[nd * DOF_PER_NODE + 3 * k: nd * DOF_PER_NODE + 3 * k + 3] = 1
    return mask


def twist_prescription(g: Grid, rest: np.ndarray, step: int, deg_per_step: float = 2.0):
    """Centre node fixed; its x_,1 and x_,2 rotated about +z by deg_per_step * step.

    Returns (mask uint8 [n_dof], values float64 [n_dof]); values hold the prescribed DOFs and are
    zero elsewhere.
    """
    c = (g.n2 // 2) * g.n1 + g.n1 // 2
    mask = pinned_mask(g, [c], kinds=(0, 1, 2))
    vals = np.zeros(g.n_dof)
    ang = math.radians(deg_per_step * step)
    rot = np.array([[math.cos(ang), -math.sin(ang), 0.0],
                    [math.sin(ang), math.cos(ang), 0.0],
                    [0.0, 0.0, 1.0]])
    base = c * DOF_PER_NODE
    vals[base:base + 3] = rest[c, 0:3]
    vals[base + 3:base + 6] = rot @ rest[c, 3:6]
    vals[base + 6:base + 9] = rot @ rest[c, 6:9]
    return mask, vals


def batch_sheets(n_shells: int = 512, seed: int = 4, n_min: int = 4, n_max: int = 40,
                 sigma: float = 1e-3):
    """Independent square sheets with n ~ U{n_min..n_max}, log10 E ~ U[4,6], h ~ U[0.5,2] mm.

    Returns a list of (grid, material, rest, q0) with seeded N(0, sigma) noise per sheet.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n_shells):
        n = int(rng.integers(n_min, n_max + 1))
        young = 10.0 ** rng.uniform(4.0, 6.0)
        h = rng.uniform(0.5e-3, 2e-3)
        mat = Material(young, 0.3, h, 200.0)
        g, rest = flat_sheet(n, n)
        out.append((g, mat, rest, noisy(rest, sigma, seed * 100003 + k)))
    return out


def corner_twist_rates(seed: int, n: int = 1, max_deg: float = 2.0) -> np.ndarray:
    """Per-trajectory twist rates of the four corners, U[-max_deg, max_deg] degrees per step;
    shape [n, 4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-max_deg, max_deg, size=(n, 4))


def corner_twist_prescription(g: Grid, rest: np.ndarray, step: int, rates) -> tuple[np.ndarray, np.ndarray]:
    """Four corners of a sheet held in place; each corner's x_,1 and x_,2 rotated about +z by
    rates[c] * step degrees. Returns (mask uint8 [n_dof], values float64 [n_dof])."""
    rest = np.asarray(rest, dtype=np.float64).reshape(-1, DOF_PER_NODE)
    corners = corner_nodes(g)
    mask = pinned_mask(g, corners, kinds=(0, 1, 2))
    vals = np.zeros(g.n_dof)
    for c, rate in zip(corners, rates):
        ang = math.radians(float(rate) * step)
        rot = np.array([[math.cos(ang), -math.sin(ang), 0.0],
                        [math.sin(ang), math.cos(ang), 0.0],
                        [0.0, 0.0, 1.0]])
        base = c * DOF_PER_NODE
        vals[base:base + 3] = rest[c, 0:3]
        vals[base + 3:base + 6] = rot @ rest[c, 3:6]
        vals[base + 6:base + 9] = rot @ rest[c, 6:9]
    return mask, vals


# Warm-start network shape: (fan_in, fan_out) per layer, 28 node features in, 12 DOFs out.
MLP_LAYERS = ((28, 256), (256, 256), (256, 256), (256, 12))


def mlp_init_params(seed: int, last_scale: float = 0.1) -> np.ndarray:
    """Seeded initial parameters of the warm-start network, packed per layer as W [fan_out,
    fan_in] row-major then b: He-normal weights (std sqrt(2 / fan_in)), the last layer's scaled
    by last_scale, zero biases. FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l, (fi, fo) in enumerate(MLP_LAYERS):
        W = rng.standard_normal((fo, fi)) * math.sqrt(2.0 / fi)
        if l == len(MLP_LAYERS) - 1:
            W *= last_scale
        parts += [W.reshape(-1), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)


def camera_rays(width: int, height: int, eye, target, up=(0.0, 0.0, 1.0), fov_deg: float = 50.0):
    """Pinhole camera rays through pixel centres: origins [n, 3] (all at eye) and unit
    directions [n, 3], row-major with the first row at the top of the image."""
    eye, target, up = (np.asarray(a, dtype=np.float64) for a in (eye, target, up))
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    half = math.tan(math.radians(fov_deg) / 2.0)
    aspect = width / height
    px = ((np.arange(width) + 0.5) / width * 2.0 - 1.0) * half * aspect
    py = (1.0 - (np.arange(height) + 0.5) / height * 2.0) * half
    PY, PX = np.meshgrid(py, px, indexing="ij")
    d = fwd[None, :] + PX.reshape(-1, 1) * right[None, :] + PY.reshape(-1, 1) * upv[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(eye, d.shape).copy()
    return o, d


def ray_scenes():
    """Static ray-intersection scenes, name -> (grid, q [n_nodes, 12], eye, target):
    a flat 10 x 10 sheet, a 10 x 10 cylinder (r 0.3 m, 1 m high) and a 30 x 30 sheet draped by the
    sinusoid field (5 cm), each seen from a camera above and to the side."""
    g1, q1 = flat_sheet(10, 10)
    g2, q2 = cylinder(10, 10)
    g3, _, q3 = sheet_sinusoid(30, 3, 0.05)
    return {
        "plane": (g1, q1, (0.3, -0.6, 0.8), (0.5, 0.5, 0.0)),
        "cylinder": (g2, q2, (1.2, 0.4, 0.9), (0.0, 0.0, 0.5)),
        "drape": (g3, q3, (0.5, -0.35, 0.55), (0.5, 0.5, 0.0)),
    }


def ccd_scene(name: str, n_points: int = 4096, seed: int = 11):
    """Continuous-collision scenes: (grid, q [n_nodes, 12] at the start of the step, dq [n_nodes,
    12] displacement over the step, x0 [n, 3] point positions, dx [n, 3] point displacements).

    plane: flat 10 x 10-patch 1 m sheet translated 2 cm up over the step; points in a slab
           around it moving up or down by up to 6 cm.
    drape: the 30 x 30-patch sinusoid sheet (5 cm, seed 3) moving to another sinusoid state
           (5 cm, seed 7) 2 cm lower; points over the sheet within 8 cm of z = 0 moving by
           N(0, 4 cm) vertically and N(0, 1 cm) in plane.
    static: the drape sheet at rest (dq = 0), the same points.
    cylinder: the periodic 10 x 10-patch cylinder (r 0.3 m) expanding radially by 10%; points at
           radius U[0, 0.5] m moving radially by U[-0.3, 0.3] m.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if name == "plane":
        g, q = flat_sheet(10, 10)
        dq = np.zeros_like(q)
        dq[:, 2] = 0.02
        x0 = np.stack([rng.uniform(-0.05, 1.05, n_points), rng.uniform(-0.05, 1.05, n_points),
                       rng.uniform(-0.04, 0.06, n_points)], axis=1)
        dx = np.stack([rng.normal(0.0, 0.01, n_points), rng.normal(0.0, 0.01, n_points),
                       rng.uniform(-0.06, 0.06, n_points)], axis=1)
        return g, q, dq, x0, dx
    if name == "cylinder":
        g, q = cylinder(10, 10)
        dq = 0.1 * q                      # radial breathing by 10% (the axis coordinate too)
        dq[:, 2] = 0.0
        dq[:, 8] = 0.0
        th = rng.uniform(0.0, 2.0 * math.pi, n_points)
        r0 = rng.uniform(0.0, 0.5, n_points)
        x0 = np.stack([r0 * np.cos(th), r0 * np.sin(th), rng.uniform(0.05, 0.95, n_points)], axis=1)
        dr = rng.uniform(-0.3, 0.3, n_points)
        dx = np.stack([dr * np.cos(th), dr * np.sin(th), rng.normal(0.0, 0.02, n_points)], axis=1)
        return g, q, dq, x0, dx
    g, _, q = sheet_sinusoid(30, 3, 0.05)
    if name == "static":
        dq = np.zeros_like(q)
    else:
        _, _, q1 = sheet_sinusoid(30, 7, 0.05)
        q1 = q1.copy()
        q1[:, 2] -= 0.02
        dq = q1 - q
    x0 = np.stack([rng.uniform(0.02, 0.98, n_points), rng.uniform(0.02, 0.98, n_points),
                   rng.uniform(-0.08, 0.08, n_points)], axis=1)
    dx = np.stack([rng.normal(0.0, 0.01, n_points), rng.normal(0.0, 0.01, n_points),
                   rng.normal(0.0, 0.04, n_points)], axis=1)
    return g, q, dq, x0, dx
