"""Learned Newton warm start: data from the plain solver, training, and warm-started rollouts.

Host-side orchestration of libbhem's kernels (bhem.py). The scene is a flat sheet under gravity
with its four corners held and twisted in plane at seeded rates (scenes.corner_twist_*):
  1. ``generate`` steps many trajectories with the batched zero-guess solver
     (shell_batch_newton_step) and records, per step and node, the features of the state before
     the step (shell_node_features) and the update the solver found beyond the inertial predictor
     (shell_warm_targets). The data stay in device memory.
  2. ``train`` fits the network with the library's forward, backward and Adam kernels
     (shell_mlp_train_step) on minibatches drawn uniformly from all recorded rows.
  3. ``rollout`` steps one shell with shell_newton_step from three starting points: the zero guess
     q^n (the plain method), the inertial predictor q^n + dt v^n, or the network's prediction.
     Convergence is measured against the residual at the zero guess in every case, so a warm start
     changes the work, not the accepted answer. A warm-started step that fails is redone from the
     zero guess (counted as a fallback).
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import bhem
from . import scenes as S


@dataclasses.dataclass
class Scene:
    n: int = 64                 # patches per side of the square sheet
    dt: float = 1e-3
    newton_rtol: float = 1e-8
    pcg_rtol: float = 1e-6
    pcg_max: int = 2000
    newton_max: int = 200       # twisted corners (up to 400 degrees) make some steps hard
    max_twist_deg: float = 2.0

    def params(self):
        return bhem.step_params(dt=self.dt, newton_rtol=self.newton_rtol, newton_max=self.newton_max,
                                pcg_rtol=self.pcg_rtol, pcg_max=self.pcg_max)

    def sheet(self):
        g, rest = S.flat_sheet(self.n, self.n)
        return g, S.SHEET_MATERIAL, rest


@dataclasses.dataclass
class Dataset:
    X: object          # torch float32 [rows, 28] (CUDA)
    T: object          # torch float32 [rows, 12] (CUDA)
    newton_iters: np.ndarray   # [steps, n_traj] zero-guess Newton iterations of the generating runs
    seconds: float
    dropped: int = 0           # trajectories stopped at a step the solver did not converge


def _prescriptions(g, rest, rates, steps):
    """mask [n_dof] (same every step) and q_fixed [steps, n_dof] of one trajectory."""
    mask, _ = S.corner_twist_prescription(g, rest, 1, rates)
    vals = np.stack([S.corner_twist_prescription(g, rest, k, rates)[1] for k in range(1, steps + 1)])
    return mask, vals


def generate(scene: Scene, n_traj: int, steps: int, seed: int) -> Dataset:
    """Runs n_traj trajectories of `steps` steps with the batched zero-guess solver."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    g, mat, rest = scene.sheet()
    n_dof, n_nodes = g.n_dof, g.n_nodes
    rates = S.corner_twist_rates(seed, n_traj, scene.max_twist_deg)
    rows = n_traj * steps * n_nodes
    X = torch.empty(rows, 28, dtype=torch.float32, device=dev)
    T = torch.empty(rows * 12, dtype=torch.float32, device=dev)
    feat_shell = bhem.Shell(g, mat, rest, precision="mixed")
    masks, vals = zip(*[_prescriptions(g, rest, rates[s], steps) for s in range(n_traj)])
    mask = torch.from_numpy(np.concatenate(masks)).to(dev)
    qfix_all = torch.from_numpy(np.concatenate(vals, axis=1)).to(dev)      # [steps, n_traj * n_dof]
    q = torch.from_numpy(np.tile(np.asarray(rest).reshape(-1), n_traj)).to(dev)
    v = torch.zeros_like(q)
    P = scene.params()
    iters = np.zeros((steps, n_traj), dtype=np.int32)
    alive = np.ones(n_traj, dtype=bool)
    keep = torch.ones(steps * n_traj, dtype=torch.bool, device=dev)   # per (step, trajectory) rows
    t0 = time.perf_counter()
    with bhem.Batch([(g, mat, rest)] * n_traj) as batch:
        for k in range(steps):
            q_old, v_old = q.clone(), v.clone()
            base = k * n_traj * n_nodes
            for s in range(n_traj):
                sl = slice(s * n_dof, (s + 1) * n_dof)
                r0 = base + s * n_nodes
                bhem.node_features(feat_shell, q[sl], v[sl], X[r0:r0 + n_nodes])
            torch.cuda.synchronize()
            stats = batch.newton_step(q, v, P, mask=mask, q_fixed=qfix_all[k])
            for s, st in enumerate(stats):
                if st["status"] != 0 and st["status"] not in (6, 7, 8):
                    raise bhem.ShellError(st["status"], f"generating step {k}, trajectory {s}")
                if st["status"] != 0:
                    alive[s] = False          # a step the solver did not finish: stop recording
                if not alive[s]:
                    keep[k * n_traj + s] = False
            iters[k] = [st["newton_iters"] for st in stats]
            bhem.warm_targets(q, q_old, v_old, scene.dt, T[base * 12:(base + n_traj * n_nodes) * 12])
    torch.cuda.synchronize()
    feat_shell.close()
    T = T.view(rows, 12)
    if not bool(keep.all()):
        rows_keep = keep.repeat_interleave(n_nodes)
        X, T = X[rows_keep].contiguous(), T[rows_keep].contiguous()
    return Dataset(X, T, iters, time.perf_counter() - t0, int((~alive).sum()))


def set_normalization(net: "bhem.Mlp", data: Dataset):
    """Per-column mean and standard deviation of the data set's features and targets."""
    in_mean, in_std = net.column_stats(data.X)
    out_mean, out_std = net.column_stats(data.T)
    net.set_normalization(in_mean, in_std, out_mean, out_std)


def train(net: "bhem.Mlp", data: Dataset, iters: int, batch_rows: int, seed: int, lr_max: float = 1e-3,
          lr_min: float = 1e-5, log_every: int = 0):
    """Fits the network to the data set (normalisation from the data; cosine learning rate).
    Returns (losses [(iteration, loss)], seconds)."""
    import torch
    set_normalization(net, data)
    gen = torch.Generator(device=data.X.device)
    gen.manual_seed(seed)
    rows = data.X.shape[0]
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(iters):
        idx = torch.randint(0, rows, (batch_rows,), generator=gen, device=data.X.device, dtype=torch.int32)
        lr = lr_min + 0.5 * (lr_max - lr_min) * (1.0 + math.cos(math.pi * it / max(1, iters - 1)))
        want = bool(log_every) and (it % log_every == 0 or it == iters - 1)
        loss = net.train_step(data.X, data.T, idx, lr, want_loss=want)
        if want:
            losses.append((it, loss))
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def validation_loss(net: "bhem.Mlp", data: Dataset, rows: int = 65536, seed: int = 0) -> float:
    """Loss on `rows` rows drawn uniformly (seeded) from a data set (no update)."""
    import torch
    rows = min(rows, net.max_rows)
    gen = torch.Generator(device=data.X.device)
    gen.manual_seed(seed)
    idx = torch.randint(0, data.X.shape[0], (rows,), generator=gen, device=data.X.device, dtype=torch.int32)
    return net.gradients(data.X, data.T, idx=idx)


def rollout(scene: Scene, rates, steps: int, mode: str, net: "bhem.Mlp" = None, keep_states: bool = False):
    """Steps one shell `steps` times; mode is "zero", "inertial" or "learned".

    Returns a dict with per-step Newton and PCG iterations, the number of fallbacks, the elapsed
    device time (CUDA events on the shell's stream around the whole loop, warm-start inference
    included) and the final q."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    g, mat, rest = scene.sheet()
    mask_np, vals = _prescriptions(g, rest, rates, steps)
    mask = torch.from_numpy(mask_np).to(dev)
    qfix = torch.from_numpy(vals).to(dev)
    P = scene.params()
    out = {"newton": [], "pcg": [], "fallbacks": 0, "res_ratio": [], "mode": mode}
    with bhem.Shell(g, mat, rest, precision="mixed") as shell:
        q = torch.from_numpy(np.asarray(rest).reshape(-1).copy()).to(dev)
        v = torch.zeros_like(q)
        warm = torch.empty_like(q)
        q_old, v_old = torch.empty_like(q), torch.empty_like(q)
        states = []
        stream = shell.stream
        launches0 = shell.kernel_launches() + (net.kernel_launches() if net is not None else 0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(steps):
            w = None
            if mode != "zero":
                q_old.copy_(q)
                v_old.copy_(v)
                if mode == "learned":
                    w = net.warm_start(shell, q, v, scene.dt, warm)
                else:
                    w = bhem.inertial_warm_start(shell, q, v, scene.dt, warm)
            st = shell.newton_step(q, v, P, mask=mask, q_fixed=qfix[k], warm=w)
            if st["status"] != 0 and w is not None:
                out["fallbacks"] += 1
                q.copy_(q_old)
                v.copy_(v_old)
                st2 = shell.newton_step(q, v, P, mask=mask, q_fixed=qfix[k])
                st2["newton_iters"] += st["newton_iters"]
                st2["pcg_iters_total"] += st["pcg_iters_total"]
                st = st2
            if st["status"] != 0:
                raise bhem.ShellError(st["status"], f"{mode} rollout step {k} failed")
            out["newton"].append(st["newton_iters"])
            out["pcg"].append(st["pcg_iters_total"])
            out["res_ratio"].append(st["res_final"] / st["res0"] if st["res0"] > 0 else 0.0)
            if keep_states:
                states.append(q.clone())
        ev1.record(stream)
        ev1.synchronize()
        out["seconds"] = ev0.elapsed_time(ev1) / 1e3
        out["launches"] = shell.kernel_launches() + (net.kernel_launches() if net is not None else 0) - launches0
        out["q"] = q.clone()
        if keep_states:
            out["states"] = states
    out["steps"] = steps
    out["steps_per_s"] = steps / out["seconds"]
    out["mean_newton"] = float(np.mean(out["newton"]))
    out["mean_pcg"] = float(np.mean(out["pcg"]))
    out["max_res_ratio"] = float(np.max(out["res_ratio"]))
    return out


def make_network(max_rows: int, seed: int) -> "bhem.Mlp":
    net = bhem.Mlp(max_rows)
    net.set_params(S.mlp_init_params(seed))
    return net
