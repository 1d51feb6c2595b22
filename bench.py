"""Benchmark of the BHEM hot path on GB300: Newton iterations of the implicit-Euler step on a
256 x 256-patch sheet (66,049 nodes, 792,588 DOF) displaced by the seeded 8-term sinusoid field.

One step = one Newton iteration through shell_newton_step (newton_max = 1): FP64 residual
(energy + gradient kernels, mass product), FP32 element Hessians of every patch assembled into
the 12x12 BSR (+ M / dt^2), the regulariser's diagonal fix, block-Jacobi set-up, PCG solves of 50
iterations (FP32 SpMV, FP64 dots; a solve that meets negative curvature restarts with a larger
shift, and pcg_iterations_per_step counts every iteration), line search with FP64 per-patch
energy differences, update and velocity. The metric is patch-Hessians/s: patches whose E,
48-gradient and exact 48x48 Hessian were evaluated and assembled, per second, with everything
else the Newton iteration needs included in the time. The default run adds, as extra keys, the
280x5 annulus, the 512-sheet batch, the learned warm start and the 200-step twist, and the
oracle on all host cores and on one thread.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "patch-Hessians/s and Newton steps/s at 1e-8 residual; batched/learned vs plain"
UNIT = "patch-Hessians/s"
WORKLOADS = {
    "sheet256": "256x256-patch 1 m sheet, 8-term sinusoid displacement (5 cm), FP32 element eval "
                "+ BSR assembly + block-Jacobi PCG solves of 50 iterations (fewer only when the FP32 "
                "residual is exhausted or negative curvature restarts the solve), FP64 residual/reductions",
    "sheet192": "192x192-patch 1 m sheet (profiling size: FP32 BSR 192 MB > L2), same recipe as sheet256",
    "batch512": "512 independent 1 m sheets, n x n patches with n ~ U{4..40}, log10 E ~ U[4,6], "
                "h ~ U[0.5,2] mm, N(0,1e-3) noise, two corners pinned, gravity; one implicit-Euler "
                "step per sheet (Newton to 1e-8 each) in one batch; plain = the same sheets one by one",
    "learned64": "64x64-patch 1 m sheet under gravity, four corners held and twisted in plane at "
                 "seeded rates U[-2,2] deg/step; warm-start MLP 28-256-256-256-12 (BF16, GELU) trained "
                 "on 10,000 steps of the plain solver (50 trajectories x 200 steps); 200 implicit-Euler "
                 "steps of an unseen trajectory, Newton to 1e-8 of the zero-guess residual, PCG to 1e-6",
    "mlp16384": "warm-start network kernels alone (profiling size): MLP 28-256-256-256-12 (BF16, GELU) on "
                "seeded N(0,1) features and targets; forward and training step of a 16,384-row batch, fused "
                "warm start of the 64x64-patch sheet",
    "twist30": "30x30-patch 1 m sheet, centre node held and its x_,1, x_,2 rotated 2 deg per step about +z, "
               "no gravity, dt = 2 ms, 200 implicit-Euler steps to 1e-8 (PCG to 1e-6), mixed precision; "
               "exact Hessian against the pseudo Hessian (App. B)",
    "rays_drape": "static ray-patch intersection (Sec. 5): 1024x768 pinhole camera (786,432 rays) on the "
                  "30x30-patch 1 m sheet draped by the 8-term sinusoid field (5 cm), FP64, Newton split "
                  "(Fig. subany); midpoint split and the plane / cylinder scenes reported beside it",
    "ccd_drape": "point-patch continuous collision detection (Sec. 5, Eq. ineqccd): 1,048,576 points "
                 "moving over one step against the 30x30-patch sheet deforming from one 5 cm sinusoid "
                 "state to another 2 cm lower, FP64, Newton split; midpoint split and the translating "
                 "plane reported beside it",
    "direct": "direct solver comparator (Sec. 6.1): implicit-Euler steps of the 10x10 noisy sheet "
              "(config 1, 1,452 DOF, 10 steps), of the 30x30 noisy sheet (11,532 DOF, 5 steps) and of the "
              "30x30 sinusoid sheet under gravity (3 steps), FP64, banded Cholesky over the node rows "
              "(hand-written kernels) against block-Jacobi PCG at eta = 1e-6 and 1e-13",
    "annulus280x5": "280x5-patch periodic annular strip, 8-term sinusoid displacement (5 cm), "
                    "FP32 element eval + BSR assembly + 50-iteration block-Jacobi PCG, FP64 "
                    "residual/reductions",
}


def make_workload(name):
    from paper_2312_14839_gb300 import scenes as S
    if name == "sheet256":
        g, rest, q = S.sheet_sinusoid(256, 3)
    elif name == "sheet192":
        g, rest, q = S.sheet_sinusoid(192, 3)
    elif name == "annulus280x5":
        g, rest, q = S.annulus_sinusoid(280, 5, 3)
    else:
        raise SystemExit(f"unknown workload {name}")
    return g, S.SHEET_MATERIAL, rest, q


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def kernel_source_sha(kernel_src: str, kernel: str) -> str:
    """sha256 (16 hex digits) of one kernel's definition in a source file: from the line that
    starts with `kernel(` to the first closing brace at column 0."""
    text = open(kernel_src).read()
    start = text.find("\n" + kernel + "(")
    if start < 0:
        return ""
    end = text.find("\n}\n", start)
    return hashlib.sha256(text[start:end + 3].encode()).hexdigest()[:16]


def recorded_traffic(kernel_src: str, kernel: str, workload: str):
    """DRAM bytes per SpMV launch from the committed ncu summary, when it was taken on the
    current kernel definition (sha256 of its source text recorded in the summary); else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = kernel_source_sha(kernel_src, kernel)
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- `"):
            k, _, v = line.strip()[3:].partition("`:")
            vals[k.strip()] = v.strip().strip("`")
    if not h or vals.get("kernel_source_sha256_16") != h:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout: float = 10.0):
        """Blocks until the sampler has printed its first line (nvidia-smi's start-up, NVML
        initialisation included, is then over), so that it does not overlap a timed region."""
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.02)
        return self

    def mark(self):
        """Start of the timed region: the summary covers the samples taken from here on."""
        self.skip = len(self.lines)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines[getattr(self, "skip", 0):]:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baselines(workload: str, n_steps: int = 4, n: int = 48):
    """The oracle (plain FP64 C) on a bounded sample of the same workload: the same sinusoid
    recipe on an n x n sheet (a 70x5 annulus for the strip), one Newton iteration with 50-iteration
    PCG solves per step, on all host cores (its OpenMP loops over patches and rows) and on one
    thread. Returns (all cores, single thread)."""
    import oracle as O
    from paper_2312_14839_gb300 import scenes as S
    if workload == "annulus280x5":
        g, rest, q = S.annulus_sinusoid(70, 5, 3)
        sample = "70x5-patch periodic annulus, same recipe"
    else:
        g, rest, q = S.sheet_sinusoid(n, 3)
        sample = f"{n}x{n}-patch sheet, same recipe"
    P = O.step_params(dt=1e-3, newton_max=1, pcg_fixed_iters=50)
    out = []
    for threads in (os.cpu_count() or 1, 1):
        used = O.set_threads(threads)
        # warm-up; then the regulariser level is carried from step to step, as on the GPU
        P.tau_carry = O.newton_step(g, S.SHEET_MATERIAL, rest, q.reshape(-1), np.zeros(g.n_dof), P)[2]["tau_final"]
        t0 = time.perf_counter()
        for _ in range(n_steps):
            O.newton_step(g, S.SHEET_MATERIAL, rest, q.reshape(-1), np.zeros(g.n_dof), P)
        dt = (time.perf_counter() - t0) / n_steps
        out.append({"value": g.n_patches / dt, "unit": UNIT, "cores": used, "kind": "oracle",
                    "nproc": os.cpu_count(),
                    "sample": f"{sample}, {n_steps} x one Newton iteration (50-iteration PCG solves), "
                              f"{dt:.2f} s each, {used} thread(s)"})
    O.set_threads(os.cpu_count() or 1)
    return out[0], out[1]


def reduce_over_ranks(dist, seconds, units, device=None):
    """Whole-job aggregate of a weak-scaling run: the slowest rank's timed region (max over ranks)
    and the units of work of all ranks (sum). Every rank calls it with its own figures; with no
    process group (dist None) the figures come back unchanged. The tensors live on `device` (the
    rank's GPU under NCCL, the CPU under gloo)."""
    if dist is None:
        return float(seconds), float(units)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2312_14839_gb300 import scenes as S
    O.build()
    cores = O.set_threads(os.cpu_count() or 1)
    n = 48
    g, rest, q = S.sheet_sinusoid(n, 3) if args.workload == "sheet256" else S.annulus_sinusoid(70, 5, 3)
    P = O.step_params(dt=1e-3, newton_max=1, pcg_fixed_iters=50)
    for _ in range(args.warmup):
        P.tau_carry = O.newton_step(g, S.SHEET_MATERIAL, rest, q.reshape(-1), np.zeros(g.n_dof), P)[2]["tau_final"]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.tau_carry = O.newton_step(g, S.SHEET_MATERIAL, rest, q.reshape(-1), np.zeros(g.n_dof), P)[2]["tau_final"]
    el = time.perf_counter() - t0
    v = g.n_patches * args.steps / el
    sample = (f"{g.nu}x{g.nv}-patch sample of the {args.workload} recipe, one Newton iteration "
              f"(50-iteration PCG solves) per step, {cores} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "nproc": os.cpu_count()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batch_bench(args):
    """Batched vs plain GPU Newton on the 512-sheet workload (one JSON line)."""
    print(json.dumps(batch_line(args, args.steps, args.warmup, max(1, min(args.steps, 2)))), flush=True)


def batch_line(args, steps, warmup, plain_reps):
    """Batched vs plain GPU Newton on the 512-sheet workload: `steps` timed batch steps after
    `warmup`, and `plain_reps` timed passes over the same sheets one by one."""
    import torch
    from paper_2312_14839_gb300 import bhem
    from paper_2312_14839_gb300 import scenes as S
    torch.cuda.set_device(0)
    bhem.load()
    sheets = S.batch_sheets(512, seed=4)
    dev = torch.device("cuda", 0)
    masks, q0s = [], []
    for g, m, r, q in sheets:
        c = S.corner_nodes(g)
        masks.append(S.pinned_mask(g, [c[0], c[3]]))
        q0s.append(q.reshape(-1))
    q0 = torch.as_tensor(np.concatenate(q0s), device=dev)
    mask = torch.as_tensor(np.concatenate(masks), device=dev)
    P = bhem.step_params(dt=1e-3)
    B = bhem.Batch([(g, m, r) for g, m, r, _ in sheets], stream=torch.cuda.current_stream())
    tune = B.autotune(q0)
    q, v, v0 = q0.clone(), torch.zeros_like(q0), torch.zeros_like(q0)
    patches = np.array([g.n_patches for g, _, _, _ in sheets])

    def bstep():
        q.copy_(q0)
        v.copy_(v0)
        return B.newton_step(q, v, P, mask=mask, q_fixed=q0)

    with ClockSampler(0) as clk:
        clk.wait_first()
        for _ in range(warmup):
            st = bstep()
        torch.cuda.synchronize()
        l0 = B.info()["kernel_launches"]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk.mark()
        ev0.record()
        ph, iters = 0.0, []
        for _ in range(steps):
            st = bstep()
            it = np.array([x["newton_iters"] for x in st])
            ph += float((patches * it).sum())
            iters.append(it)
        ev1.record()
        torch.cuda.synchronize()
    sec = ev0.elapsed_time(ev1) / 1e3
    launches = B.info()["kernel_launches"] - l0
    ok = all(x["status"] == 0 and x["res_final"] <= 1e-8 * x["res0"] for x in st)
    # plain: the same sheets stepped one by one through shell_newton_step
    shells = [bhem.Shell(g, m, torch.as_tensor(r.reshape(-1), device=dev), precision="mixed")
              for g, m, r, _ in sheets]
    qs = [torch.as_tensor(x, device=dev) for x in q0s]
    ms_ = [torch.as_tensor(x, device=dev) for x in masks]
    qw = [x.clone() for x in qs]
    vw = [torch.zeros_like(x) for x in qs]

    def pstep():
        tot = 0
        for k, sh in enumerate(shells):
            qw[k].copy_(qs[k])
            vw[k].zero_()
            tot += sh.newton_step(qw[k], vw[k], P, mask=ms_[k], q_fixed=qs[k])["newton_iters"] * sheets[k][0].n_patches
        return tot
    pstep()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    preps = plain_reps
    for _ in range(preps):
        pph = pstep()
    torch.cuda.synchronize()
    psec = (time.perf_counter() - t0) / preps
    for sh in shells:
        sh.close()
    it_all = np.concatenate(iters)
    B.close()
    return {
        "metric": METRIC, "value": ph / sec, "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": sec / steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded sheets)",
        "config": {"workload": WORKLOADS["batch512"], "sheets": len(sheets), "patches": int(patches.sum()),
                   "dof": B.n_dof, "autotuned": {"patches_per_item": tune["patches_per_item"],
                                                 "assembly": ["atomic", "color"][tune["assembly"]]}},
        "sheet_steps_per_s": len(sheets) * steps / sec,
        "plain_sheet_steps_per_s": len(sheets) / psec,
        "batched_vs_plain": (len(sheets) * steps / sec) / (len(sheets) / psec),
        "plain_value": pph / psec,
        "newton_iters_per_sheet": {"mean": float(it_all.mean()), "max": int(it_all.max())},
        "all_sheets_converged_1e-8": bool(ok), "gpu_launches": launches, "clocks": clk.summary(),
    }


def run_mlp_bench(args):
    """The warm-start network's kernels alone on seeded synthetic rows (no solver data): the JSON
    line of network_timing, value = training-step GEMM TFLOP/s."""
    import torch
    from paper_2312_14839_gb300 import learned as L
    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    X = torch.as_tensor(rng.normal(size=(65536, 28)), dtype=torch.float32, device="cuda")
    T = torch.as_tensor(rng.normal(size=(65536, 12)), dtype=torch.float32, device="cuda")
    net = L.make_network(16384, 5)
    with ClockSampler(0) as clk:
        clk.wait_first()
        clk.mark()
        nk = network_timing(net, X, T, reps=max(1, args.steps))
    net.close()
    tr = nk["train_step_16384_rows"]
    line = {"metric": "warm-start network GEMM throughput (training step)", "value": tr["tflops"],
            "unit": "TFLOP/s", "n_gpus": 1, "steps": max(1, args.steps), "warmup": 3,
            "ms_per_step": tr["us"] / 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (FP32 accumulation)", "data": "synthetic (seeded N(0,1) rows)",
            "config": {"workload": WORKLOADS["mlp16384"], "batch_rows": 16384},
            "network_kernels": nk, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_learned_bench(args):
    """Learned warm start vs the plain zero-guess Newton (and the inertial predictor) on the
    64x64 corner-twist sheet (one JSON line)."""
    print(json.dumps(learned_line(args)), flush=True)


def learned_line(args):
    """Learned warm start vs the plain zero-guess Newton (and the inertial predictor) on the
    64x64 corner-twist sheet. The timed region of each arm is a 200-step rollout, warm-start
    inference included."""
    import torch
    from paper_2312_14839_gb300 import bhem
    from paper_2312_14839_gb300 import learned as L
    from paper_2312_14839_gb300 import scenes as S
    torch.cuda.set_device(0)
    bhem.load()
    scene = L.Scene(n=64)
    n_traj, gen_steps, roll_steps = 50, 200, 200
    data = L.generate(scene, n_traj=n_traj, steps=gen_steps, seed=4)
    net = L.make_network(16384, 5)
    losses, train_sec = L.train(net, data, iters=args.train_iters, batch_rows=16384, seed=6,
                                log_every=max(1, args.train_iters // 4))
    rates = S.corner_twist_rates(999, 1)[0]
    for mode in ("zero", "inertial", "learned"):        # warm-up: short rollouts of every arm
        L.rollout(scene, rates, args.warmup, mode, net)
    res = {}
    with ClockSampler(0) as clk:
        clk.wait_first()
        clk.mark()
        for mode in ("zero", "inertial", "learned"):
            res[mode] = L.rollout(scene, rates, roll_steps, mode, net)
    z, i, l = res["zero"], res["inertial"], res["learned"]
    g, _, rest = scene.sheet()
    disp = float((z["q"] - torch.as_tensor(rest.reshape(-1), device=z["q"].device)).abs().max())
    diff = float((l["q"] - z["q"]).abs().max())

    def arm(r):
        return {"steps_per_s": r["steps_per_s"], "newton_iters_mean": r["mean_newton"],
                "pcg_iters_per_step": r["mean_pcg"], "newton_hist": np.bincount(r["newton"]).tolist(),
                "fallbacks": r["fallbacks"], "max_final_residual_ratio": r["max_res_ratio"]}
    line = {
        "metric": METRIC, "value": l["steps_per_s"], "unit": "implicit-Euler steps/s", "n_gpus": 1,
        "steps": roll_steps, "warmup": args.warmup, "ms_per_step": l["seconds"] / roll_steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 MLP + f32/f64 solver",
        "data": "synthetic (seeded corner-twist trajectories of the plain solver)",
        "config": {"workload": WORKLOADS["learned64"], "patches": g.n_patches, "nodes": g.n_nodes,
                   "train_rows": int(data.X.shape[0]), "train_iters": args.train_iters, "batch_rows": 16384},
        "learned": arm(l), "plain_zero_guess": arm(z), "inertial_predictor": arm(i),
        "learned_vs_plain": l["steps_per_s"] / z["steps_per_s"],
        "learned_vs_inertial": l["steps_per_s"] / i["steps_per_s"],
        "final_state_max_abs_diff_vs_plain": diff, "final_displacement_max_abs": disp,
        "train": {"loss_first": losses[0][1], "loss_last": losses[-1][1], "seconds": train_sec,
                  "iters_per_s": args.train_iters / train_sec},
        "data_generation": {"steps": n_traj * gen_steps, "seconds": data.seconds,
                            "newton_iters_mean": float(data.newton_iters.mean()),
                            "trajectories_stopped_unconverged": data.dropped},
        "gpu_launches": l["launches"], "clocks": clk.summary(),
        "network_kernels": network_timing(net, data.X, data.T),
    }
    net.close()
    return line


# BF16 multiply-adds per row of one forward pass (padded fan-in x fan-out of the 4 layers)
MLP_MAC_PER_ROW = 32 * 256 + 2 * 256 * 256 + 256 * 16


def network_timing(net, X_all, T_all, n_sheet=64, reps=20):
    """The warm-start network's tensor-core kernels (tcgen05 GEMM, fused warm start) timed with
    CUDA events on the network's stream after 3 warm-up calls: forward of a 16,384-row batch (four
    GEMM launches plus the input and output kernels), one training step of that batch (forward,
    loss, backward, Adam), and the fused warm start of the 64x64 sheet (one launch, 4,225 nodes).
    Rates are GEMM FLOPs over the whole call, against the measured BF16 peak."""
    import torch
    from paper_2312_14839_gb300 import bhem
    from paper_2312_14839_gb300 import scenes as S
    rows = 16384
    X, T = X_all[:rows].contiguous(), T_all[:rows].contiguous()
    idx = torch.arange(rows, dtype=torch.int32, device=X.device)
    Y = torch.empty(rows, 12, dtype=torch.float32, device=X.device)
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops") \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0

    def timed(fn):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e-3

    def entry(sec, flop):
        return {"us": sec * 1e6, "gemm_flop": flop, "tflops": flop / sec / 1e12,
                "frac_of_bf16_peak": flop / sec / 1e12 / peak}

    fwd_flop = 2 * rows * MLP_MAC_PER_ROW
    train_flop = 2 * rows * (3 * MLP_MAC_PER_ROW - 32 * 256)
    out = {"forward_16384_rows": entry(timed(lambda: net.forward(X, Y)), fwd_flop),
           "train_step_16384_rows": entry(timed(lambda: net.train_step(X_all, T_all, idx, 0.0)), train_flop)}
    g, rest = S.flat_sheet(n_sheet, n_sheet)
    with bhem.Shell(g, S.SHEET_MATERIAL, rest.reshape(-1)) as sh:
        q = torch.as_tensor(rest.reshape(-1), dtype=torch.float64, device="cuda")
        v = torch.zeros_like(q)
        w = torch.empty_like(q)
        out["warm_start_64x64"] = entry(timed(lambda: net.warm_start(sh, q, v, 1e-3, w)),
                                        2 * g.n_nodes * MLP_MAC_PER_ROW)
    out["peak_source"] = "measured bf16_tflops (MEASURED_PEAKS.json), cuBLAS 8192^3 burst"
    out["kernels"] = ("k_gemm_tc (tcgen05.mma kind::f16 into TMEM, TMA 128-byte-swizzled operands), "
                      "k_mlp_warm (fused warm start, same MMA sequence)")
    return out


# Algorithmic work per patch of the two arithmetic-bound kernels (the units are stated in DESIGN):
#  - element Hessian: the factored Phi^T M_g Phi contraction with symmetry, 16 x 15 x 48 x 5 (T)
#    + 1,176 x 80 (K) = 151,680 FMA;
#  - FP64 energy + gradient: sum-factorised interpolation 1,536 + gradient transpose 1,536 +
#    about 190 FMA of nonlinear point work at each of the 16 Gauss points = 6,112 FMA.
ELEMENT_FLOP_PER_PATCH = 2 * (16 * 15 * 48 * 5 + 1176 * 80)
ENERGY64_FLOP_PER_PATCH = 2 * (1536 + 1536 + 16 * 190)
# The tensor-core form of the element pass (the default of a mixed-precision shell) issues per patch
# 96 rows (6 component pairs x 16 J) x 16 columns x 96 K values (16 Gauss points x 6 kinds) TF32
# multiply-adds, three times (head and tail products): 442,368 tensor MACs.
ELEMENT_TC_TENSOR_FLOP_PER_PATCH = 2 * 3 * 96 * 16 * 96
# dense TF32 against dense BF16 on the fifth-generation tensor cores (nominal 1.1 / 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def element_form():
    """Which FP32 element pass a mixed-precision shell created now runs (BHEM_ELEMENT)."""
    return "ffma" if os.environ.get("BHEM_ELEMENT") == "ffma" else "tc"


def element_kernel_name():
    if element_form() == "tc":
        return ("k_element_tc (FP32 exact Hessian: Gauss-point matrices and T rows on the FMA pipe, "
                "the contraction K = Psi^T T on tcgen05 kind::tf32 from tensor memory")
    return "k_element_full<float> (FP32 exact Hessian on the FMA pipe"


def alu_rooflines(sh, q_d, P, n_patches, stream, reps=5):
    """Element Hessian pass and FP64 energy/gradient pass timed with CUDA events on the shell's
    stream, against FP32 / FP64 FMA peaks measured in the same run (shell_measure_fma_peak)."""
    import torch
    from paper_2312_14839_gb300 import bhem
    peak32 = bhem.measure_fma_peak(False, 4096, stream)
    peak64 = bhem.measure_fma_peak(True, 256, stream)

    def timed(fn):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    t_el = timed(lambda: sh.energy_grad_hess(q_d, mass_scale=1.0 / P.dt ** 2, want_energy=False,
                                             want_grad=False))
    t_eg = timed(lambda: sh.energy_grad_hess(q_d, want_hessian=False))
    out = []
    for kern, t, flop, pk, what in (
            (element_kernel_name() + " + BSR scatter; the BSR clear is in the time)",
             t_el, ELEMENT_FLOP_PER_PATCH, peak32, "FP32"),
            ("k_energy_grad64 (FP64 energy + assembled gradient; the gradient clear is in the time)",
             t_eg, ENERGY64_FLOP_PER_PATCH, peak64, "FP64")):
        ach = flop * n_patches / t / 1e12
        out.append({"kernel": kern, "bound": "alu", "achieved": ach, "peak": pk / 1e12, "unit": "TFLOP/s",
                    "frac": ach * 1e12 / pk, "flop_per_patch": flop, "avg_launch_us": t * 1e6,
                    "peak_source": f"measured {what} FMA microbenchmark (shell_measure_fma_peak)"})
    if element_form() == "tc":
        # the same pass's tensor-core work against the TF32 peak (measured BF16 x nominal ratio)
        path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        bf16 = json.load(open(path)).get("bf16_tflops") if os.path.exists(path) else None
        tf32 = (bf16 if bf16 else 1900.0) * TF32_PER_BF16
        ach = ELEMENT_TC_TENSOR_FLOP_PER_PATCH * n_patches / t_el / 1e12
        out.append({"kernel": "k_element_tc tensor-core work (TF32 head and tail products)", "bound": "tensor",
                    "achieved": ach, "peak": tf32, "unit": "TFLOP/s", "frac": ach / tf32,
                    "flop_per_patch": ELEMENT_TC_TENSOR_FLOP_PER_PATCH, "avg_launch_us": t_el * 1e6,
                    "peak_source": ("measured bf16_tflops (MEASURED_PEAKS.json) x 1.1/2.25 (nominal dense "
                                    "TF32/BF16)" if bf16 else "fallback 1.9 PFLOP/s bf16 x 1.1/2.25")})
    return out


def element_kernel_only(sh, q_d, n_patches, stream, reps=5):
    """The element kernel without assembly: E-, gradient- and exact-Hessian evaluation of every
    patch with the 48x48 FP32 Hessians written unassembled (no BSR clear or scatter), CUDA events
    on the shell's stream."""
    import torch
    H = torch.empty(n_patches, 48, 48, dtype=torch.float32, device=q_d.device)
    from paper_2312_14839_gb300 import bhem
    lib = bhem.load()

    def run():
        bhem._check(lib.shell_element_egh(sh._h, bhem._ptr(q_d), 1, None, None, bhem._ptr(H)))

    for _ in range(2):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    del H
    return {"patch_hessians_per_s": n_patches / t, "avg_launch_us": t * 1e6,
            "what": element_kernel_name() + ") writing the 48x48 FP32 Hessians unassembled (no BSR clear or scatter)"}


# FP64 operations per step of the ray search (adds, multiplies, compares, min/max, divisions and
# square roots one each), counted from the kernel source: a patch's root box test, one candidate
# box (blossoming of 8 curves per coordinate and the slab test), one Newton iteration, and the
# fixed work of one split (Newton variant: centre evaluation, projection, acceptance, pinwheel).
RAY_OPS_ROOT = 25
RAY_OPS_BOX = 1324
RAY_OPS_NEWTON_ITER = 367
RAY_OPS_SPLIT = {"midpoint": 11, "newton": 311}


def ray_ops(stats, n_patches: int, variant: str) -> float:
    """Algorithmic FP64 operations of one trace from the per-ray counts (stats [n, 4])."""
    st = stats.astype(np.int64)
    return float(RAY_OPS_ROOT * n_patches * len(st) + RAY_OPS_BOX * (st[:, 2] - n_patches).sum()
                 + RAY_OPS_NEWTON_ITER * st[:, 3].sum() + RAY_OPS_SPLIT[variant] * st[:, 0].sum())


def write_depth_pgm(path: str, tau, flags, W: int, H: int):
    """The frame's hit distances as a 16-bit binary PGM (nearest = brightest, misses black)."""
    hit = (flags & 1) == 1
    img = np.zeros(W * H, dtype=np.uint16)
    if hit.any():
        t = tau[hit]
        lo, hi = float(t.min()), float(t.max())
        img[hit] = (65535.0 * (1.0 - (t - lo) / max(hi - lo, 1e-30)) * 0.9 + 6553.5).astype(np.uint16)
    with open(path, "wb") as f:
        f.write(f"P5\n{W} {H}\n65535\n".encode())
        f.write(img.reshape(H, W).astype(">u2").tobytes())


def run_rays_bench(args):
    """Static ray-patch intersection: rays/s on the draped sheet (one JSON line)."""
    import torch
    import oracle as O
    from paper_2312_14839_gb300 import bhem
    from paper_2312_14839_gb300 import scenes as S
    torch.cuda.set_device(0)
    bhem.load()
    dev = torch.device("cuda", 0)
    W, H = (int(x) for x in args.frame.lower().split("x"))
    n = W * H
    scenes = S.ray_scenes()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    def trace_timing(name, variant, steps, warmup, want_e2e=False):
        g, q, eye, tgt = scenes[name]
        o, d = S.camera_rays(W, H, eye, tgt)
        sh = bhem.Shell(g, S.SHEET_MATERIAL, torch.as_tensor(q.reshape(-1), device=dev), precision="fp64")
        stream = sh.stream
        dq = torch.as_tensor(q.reshape(-1), dtype=torch.float64, device=dev)
        do, dd = torch.as_tensor(o, device=dev), torch.as_tensor(d, device=dev)
        out = sh.trace_rays(dq, do, dd, variant=variant, want_stats=True)
        for _ in range(warmup):
            sh.trace_rays(dq, do, dd, variant=variant, out=out)
        torch.cuda.synchronize()
        stats = out["stats"].cpu().numpy()
        flags = out["flags"].cpu().numpy()
        if args.image and name == "drape" and variant == "newton":
            write_depth_pgm(args.image, out["tau"].cpu().numpy(), flags, W, H)
        res = {"hit_fraction": float((flags & 1).mean()), "flagged": int((flags & 6).astype(bool).sum()),
               "splits_mean": float(stats[:, 0].mean()), "splits_max": int(stats[:, 0].max()),
               "heap_peak_max": int(stats[:, 1].max()), "newton_iters_mean": float(stats[:, 3].mean()),
               "fp64_ops_per_trace": ray_ops(stats, g.n_patches, variant)}
        l0 = sh.kernel_launches()
        ms = []
        clk = None
        with ClockSampler(0) as c:
            for _ in range(steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sh.trace_rays(dq, do, dd, variant=variant, out=out)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
        clk = c.summary()
        res["gpu_launches_per_trace"] = (sh.kernel_launches() - l0) / max(steps, 1)
        res["ms_per_trace"] = float(np.mean(ms))
        res["rays_per_s"] = n / (res["ms_per_trace"] / 1e3)
        if want_e2e:
            # the public call with host data: pinned host rays in, host hits out, every step
            ho, hd = torch.as_tensor(o).pin_memory(), torch.as_tensor(d).pin_memory()
            host = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items() if k != "stats"}
            dev_out = {k: v for k, v in out.items() if k != "stats"}
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(steps):
                    do.copy_(ho, non_blocking=True)
                    dd.copy_(hd, non_blocking=True)
                    sh.trace_rays(dq, do, dd, variant=variant, out=dev_out)
                    for k in host:
                        host[k].copy_(dev_out[k], non_blocking=True)
                e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            res["e2e"] = {"value": n * steps / sec, "unit": "rays/s",
                          "h2d_bytes_per_step": int(ho.numel() * 8 + hd.numel() * 8),
                          "d2h_bytes_per_step": int(sum(v.numel() * v.element_size() for v in host.values()))}
        sh.close()
        return res, clk

    main_res, clk = trace_timing("drape", "newton", args.steps, args.warmup, want_e2e=True)
    others = {}
    for name in ("drape", "cylinder", "plane"):
        for variant in ("newton", "midpoint"):
            if (name, variant) == ("drape", "newton"):
                continue
            r, _ = trace_timing(name, variant, 1, 1)
            others[f"{name}_{variant}"] = {k: r[k] for k in ("rays_per_s", "ms_per_trace", "hit_fraction",
                                                             "splits_mean", "splits_max", "flagged")}
    peak64 = bhem.measure_fma_peak(True, 256, torch.cuda.current_stream())
    peak_ops = peak64 / 2.0     # one FP64 pipe instruction per add, multiply or compare
    ach = main_res["fp64_ops_per_trace"] / (main_res["ms_per_trace"] / 1e3)
    # the oracle on a seeded sample of the same frame, all host cores
    cpu = None
    if not args.no_cpu_baseline:
        g, q, eye, tgt = scenes["drape"]
        o, d = S.camera_rays(W, H, eye, tgt)
        idx = np.sort(np.random.default_rng(5).choice(n, min(n, 65536), replace=False))
        O.build()
        cores = O.set_threads(os.cpu_count() or 1)
        t0 = time.perf_counter()
        O.trace_rays(g, q, o[idx], d[idx], True)
        sec = time.perf_counter() - t0
        cpu = {"value": len(idx) / sec, "unit": "rays/s", "cores": cores, "kind": "oracle", "nproc": os.cpu_count(),
               "sample": f"{len(idx):,} seeded rays of the same {W}x{H} frame, Newton split, {sec:.1f} s on "
                         f"{cores} host threads"}
    print(json.dumps({
        "metric": "rays/s, static ray-patch intersection (Sec. 5)", "value": main_res["rays_per_s"],
        "unit": "rays/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": main_res["ms_per_trace"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (pinhole camera rays)",
        "config": {"workload": WORKLOADS["rays_drape"], "frame": f"{W}x{H}", "rays": n, "patches": 900,
                   "l2": "flushed (256 MB write) before every timed trace"},
        "e2e": main_res["e2e"], "gpu_launches": main_res["gpu_launches_per_trace"] * args.steps,
        "roofline": {"bound": "alu", "achieved": ach / 1e12, "peak": peak_ops / 1e12, "unit": "TFLOP/s",
                     "frac": ach / peak_ops, "traffic": None,
                     "kernel": "k_trace_rays (+ k_ray_nets, k_trace_rays_redo in the same events)",
                     "work": "FP64 operations counted per ray from its splits, boxes and Newton iterations",
                     "peak_source": "measured FP64 FMA rate (shell_measure_fma_peak) as instructions/s"},
        "cpu_baseline": cpu, "search": {k: main_res[k] for k in ("hit_fraction", "flagged", "splits_mean",
                                                              "splits_max", "heap_peak_max", "newton_iters_mean",
                                                              "fp64_ops_per_trace")},
        "other_scenes": others, "clocks": clk,
    }), flush=True)


# FP64 operations per step of the collision search, counted from the kernel source like the ray
# search's: a patch's swept-box test, one feasibility test (two nets cut per axis, half-line
# classification, extents, interval subtraction), one Newton iteration in (u, v, s), and the fixed
# work of one split.
CCD_OPS_ROOT = 6
CCD_OPS_FEASIBLE = 2950
CCD_OPS_NEWTON_ITER = 660
CCD_OPS_SPLIT = {"midpoint": 11, "newton": 30}


def ccd_ops(stats, n_patches: int, variant: str) -> float:
    st = stats.astype(np.int64)
    return float(CCD_OPS_ROOT * n_patches * len(st) + CCD_OPS_FEASIBLE * st[:, 2].sum()
                 + CCD_OPS_NEWTON_ITER * st[:, 3].sum() + CCD_OPS_SPLIT[variant] * st[:, 0].sum())


def run_ccd_bench(args):
    """Point-patch continuous collision detection: contact queries/s (one JSON line)."""
    import torch
    import oracle as O
    from paper_2312_14839_gb300 import bhem
    from paper_2312_14839_gb300 import scenes as S
    torch.cuda.set_device(0)
    bhem.load()
    dev = torch.device("cuda", 0)
    n = args.points
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    def timing(scene, variant, steps, warmup, want_e2e=False):
        g, q, dq, x0, dx = S.ccd_scene(scene, n)
        sh = bhem.Shell(g, S.SHEET_MATERIAL, torch.as_tensor(q.reshape(-1), device=dev), precision="fp64")
        stream = sh.stream
        dq_, ddq = (torch.as_tensor(a.reshape(-1), dtype=torch.float64, device=dev) for a in (q, dq))
        dx0, ddx = torch.as_tensor(x0, device=dev), torch.as_tensor(dx, device=dev)
        out = sh.ccd_points(dq_, ddq, dx0, ddx, variant=variant, want_stats=True)
        for _ in range(warmup):
            sh.ccd_points(dq_, ddq, dx0, ddx, variant=variant, out=out)
        torch.cuda.synchronize()
        stats, flags = out["stats"].cpu().numpy(), out["flags"].cpu().numpy()
        res = {"contact_fraction": float((flags & 1).mean()), "flagged": int((flags & 6).astype(bool).sum()),
               "splits_mean": float(stats[:, 0].mean()), "splits_max": int(stats[:, 0].max()),
               "heap_peak_max": int(stats[:, 1].max()), "feasibility_tests_mean": float(stats[:, 2].mean()),
               "newton_iters_mean": float(stats[:, 3].mean()), "fp64_ops_per_call": ccd_ops(stats, g.n_patches, variant)}
        l0 = sh.kernel_launches()
        ms = []
        with ClockSampler(0) as c:
            for _ in range(steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sh.ccd_points(dq_, ddq, dx0, ddx, variant=variant, out=out)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
        clk = c.summary()
        res["gpu_launches_per_call"] = (sh.kernel_launches() - l0) / max(steps, 1)
        res["ms_per_call"] = float(np.mean(ms))
        res["queries_per_s"] = n / (res["ms_per_call"] / 1e3)
        if want_e2e:
            hx0, hdx = torch.as_tensor(x0).pin_memory(), torch.as_tensor(dx).pin_memory()
            host = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items() if k != "stats"}
            dev_out = {k: v for k, v in out.items() if k != "stats"}
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(steps):
                    dx0.copy_(hx0, non_blocking=True)
                    ddx.copy_(hdx, non_blocking=True)
                    sh.ccd_points(dq_, ddq, dx0, ddx, variant=variant, out=dev_out)
                    for k in host:
                        host[k].copy_(dev_out[k], non_blocking=True)
                e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            res["e2e"] = {"value": n * steps / sec, "unit": "contact queries/s",
                          "h2d_bytes_per_step": int((hx0.numel() + hdx.numel()) * 8),
                          "d2h_bytes_per_step": int(sum(v.numel() * v.element_size() for v in host.values()))}
        sh.close()
        return res, clk

    main_res, clk = timing("drape", "newton", args.steps, args.warmup, want_e2e=True)
    others = {}
    for scene, variant in (("drape", "midpoint"), ("plane", "newton"), ("plane", "midpoint")):
        r, _ = timing(scene, variant, 1, 1)
        others[f"{scene}_{variant}"] = {k: r[k] for k in ("queries_per_s", "ms_per_call", "contact_fraction",
                                                          "splits_mean", "splits_max", "flagged")}
    peak_ops = bhem.measure_fma_peak(True, 256, torch.cuda.current_stream()) / 2.0
    ach = main_res["fp64_ops_per_call"] / (main_res["ms_per_call"] / 1e3)
    cpu = None
    if not args.no_cpu_baseline:
        g, q, dq, x0, dx = S.ccd_scene("drape", n)
        idx = np.sort(np.random.default_rng(5).choice(n, min(n, 1048576), replace=False))
        O.build()
        cores = O.set_threads(os.cpu_count() or 1)
        t0 = time.perf_counter()
        O.ccd_points(g, q, dq, x0[idx], dx[idx], True)
        sec = time.perf_counter() - t0
        cpu = {"value": len(idx) / sec, "unit": "contact queries/s", "cores": cores, "kind": "oracle",
               "nproc": os.cpu_count(),
               "sample": f"{len(idx):,} seeded points of the same batch, Newton split, {sec:.1f} s on "
                         f"{cores} host threads"}
    print(json.dumps({
        "metric": "contact queries/s, point-patch continuous collision detection (Sec. 5)",
        "value": main_res["queries_per_s"], "unit": "contact queries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_res["ms_per_call"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded moving points)",
        "config": {"workload": WORKLOADS["ccd_drape"], "points": n, "patches": 900,
                   "l2": "flushed (256 MB write) before every timed call"},
        "e2e": main_res["e2e"], "gpu_launches": main_res["gpu_launches_per_call"] * args.steps,
        "roofline": {"bound": "alu", "achieved": ach / 1e12, "peak": peak_ops / 1e12, "unit": "TFLOP/s",
                     "frac": ach / peak_ops, "traffic": None,
                     "kernel": "k_ccd_points (+ k_ccd_nets, k_ccd_points_redo in the same events)",
                     "work": "FP64 operations counted per point from its splits, feasibility tests and Newton iterations",
                     "peak_source": "measured FP64 FMA rate (shell_measure_fma_peak) as instructions/s"},
        "cpu_baseline": cpu, "search": {k: main_res[k] for k in ("contact_fraction", "flagged", "splits_mean",
                                                              "splits_max", "heap_peak_max", "feasibility_tests_mean",
                                                              "newton_iters_mean", "fp64_ops_per_call")},
        "other_scenes": others, "clocks": clk,
    }), flush=True)


def run_direct_bench(args):
    """Direct (banded Cholesky) against PCG Newton solves: steps/s and Newton iterations."""
    import torch
    from paper_2312_14839_gb300 import bhem
    from paper_2312_14839_gb300 import scenes as S
    torch.cuda.set_device(0)
    bhem.load()
    dev = torch.device("cuda", 0)
    cases = {}
    for name, (g, rest, q0), steps in (("sheet10_noise", S.sheet_noisy(10, 1e-3, 1), 10),
                                       ("sheet30_noise", S.sheet_noisy(30, 1e-3, 1), 5),
                                       ("sheet30_sinusoid", S.sheet_sinusoid(30, 3), 3)):
        mask = torch.as_tensor(S.pinned_mask(g, [0, g.n_nodes - 1]), device=dev)
        res = {}
        for label, solver, eta in (("direct", "direct", 1e-6), ("pcg_eta1e-6", "pcg", 1e-6),
                                   ("pcg_eta1e-13", "pcg", 1e-13)):
            P = bhem.step_params(dt=1e-3, pcg_rtol=eta, pcg_max=20000)
            sh = bhem.Shell(g, S.SHEET_MATERIAL, torch.as_tensor(rest.reshape(-1), device=dev), precision="fp64",
                            solver=solver)

            def rollout(n):
                q = torch.as_tensor(q0.reshape(-1).copy(), device=dev)
                v = torch.zeros_like(q)
                qf = q.clone()
                out = []
                for _ in range(n):
                    st = sh.newton_step(q, v, P, mask=mask, q_fixed=qf)
                    out.append((st["newton_iters"], st["pcg_iters_total"], st["status"]))
                return out
            rollout(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(sh.stream)
            it = rollout(steps)
            e1.record(sh.stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            res[label] = {"steps_per_s": steps / sec, "ms_per_step": sec / steps * 1e3,
                          "newton_iters": [a for a, _, _ in it], "pcg_iters_per_step": float(np.mean([b for _, b, _ in it])),
                          "status": sorted({c for _, _, c in it})}
            sh.close()
        res["newton_iters_equal_direct_vs_pcg_eta1e-13"] = res["direct"]["newton_iters"] == res["pcg_eta1e-13"]["newton_iters"]
        cases[name] = {"dof": g.n_dof, "steps": steps, **res}
    main = cases["sheet30_noise"]["direct"]
    print(json.dumps({
        "metric": "implicit-Euler steps/s with the direct (banded Cholesky) Newton solve",
        "value": main["steps_per_s"], "unit": "implicit-Euler steps/s", "n_gpus": 1, "steps": 5,
        "warmup": 1, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOADS["direct"]},
        "cases": cases,
    }), flush=True)


def run_twist_bench(args):
    """Exact against pseudo Hessian on the twist scene (one JSON line)."""
    print(json.dumps(twist_line(args)), flush=True)


def twist_line(args):
    """Exact against pseudo Hessian on the twist scene: implicit-Euler steps/s and Newton
    iterations at 1e-8, plus the element pass time of each Hessian."""
    import torch
    from paper_2312_14839_gb300 import bhem
    from paper_2312_14839_gb300 import scenes as S
    torch.cuda.set_device(0)
    bhem.load()
    dev = torch.device("cuda", 0)
    g, rest = S.flat_sheet(30, 30)
    mat = S.SHEET_MATERIAL
    steps = 200
    pres = [S.twist_prescription(g, rest, k) for k in range(1, steps + 1)]
    mask = torch.as_tensor(pres[0][0], device=dev)
    qfix = torch.as_tensor(np.stack([v for _, v in pres]), device=dev)
    # the Newton cap is generous; steps that still end unconverged are counted (q then holds the
    # last iterate)
    P = bhem.step_params(dt=2e-3, gravity=(0.0, 0.0, 0.0), newton_max=200)
    res = {}
    clk_all = []
    for hess in ("exact", "pseudo"):
        sh = bhem.Shell(g, mat, torch.as_tensor(rest.reshape(-1), device=dev), precision="mixed", hessian=hess)
        stream = sh.stream
        rest_d = torch.as_tensor(rest.reshape(-1), device=dev)

        def rollout(n):
            q, v = rest_d.clone(), torch.zeros_like(rest_d)
            it = []
            for k in range(n):
                st = sh.newton_step(q, v, P, mask=mask, q_fixed=qfix[k])
                if st["status"] not in (0, 6, 7, 8):
                    raise bhem.ShellError(st["status"], f"twist step {k} ({hess})")
                it.append((st["newton_iters"], st["pcg_iters_total"], st["status"], st["regularizations"]))
            return it
        rollout(args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = sh.kernel_launches()
        torch.cuda.synchronize()
        with ClockSampler(0) as clk:
            clk.wait_first()
            clk.mark()
            e0.record(stream)
            it = rollout(steps)
            e1.record(stream)
            torch.cuda.synchronize()
        clk_all.append(clk.summary())
        sec = e0.elapsed_time(e1) / 1e3
        # element pass of this Hessian (BSR clear + element kernel); its cost does not depend on q
        q_end = rest_d.clone()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            sh.energy_grad_hess(q_end, mass_scale=1.0 / P.dt ** 2, want_energy=False, want_grad=False)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(10):
            sh.energy_grad_hess(q_end, mass_scale=1.0 / P.dt ** 2, want_energy=False, want_grad=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        newton = np.array([a for a, _, _, _ in it])
        res[hess] = {"steps_per_s": steps / sec, "ms_per_step": sec / steps * 1e3,
                     "newton_iters_mean": float(newton.mean()), "newton_iters_max": int(newton.max()),
                     "pcg_iters_per_step": float(np.mean([b for _, b, _, _ in it])),
                     "unconverged_steps": int(sum(1 for *_, st_, _ in it if st_ != 0)),
                     "regularized_solves_per_step": float(np.mean([r for *_, r in it])),
                     "element_pass_us": ev0.elapsed_time(ev1) / 10 * 1e3,
                     "gpu_launches": sh.kernel_launches() - l0}
        sh.close()
    ex, ps = res["exact"], res["pseudo"]
    return {
        "metric": METRIC, "value": ex["steps_per_s"], "unit": "implicit-Euler steps/s", "n_gpus": 1,
        "steps": steps, "warmup": args.warmup, "ms_per_step": ex["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (twist prescription)",
        "config": {"workload": WORKLOADS["twist30"], "patches": g.n_patches, "dof": g.n_dof},
        "exact_hessian": ex, "pseudo_hessian": ps,
        "pseudo_vs_exact_steps_per_s": ps["steps_per_s"] / ex["steps_per_s"],
        "gpu_launches": ex["gpu_launches"], "clocks": clk_all[0],
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sheet256", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="sheet256: leave out the annulus, batch, learned and twist measurements")
    ap.add_argument("--spmv-reps", type=int, default=50)
    ap.add_argument("--train-iters", type=int, default=4000)
    ap.add_argument("--spmv", default="auto", choices=["auto", "plain", "tma"])
    ap.add_argument("--frame", default="1024x768", help="rays_drape: camera frame WxH")
    ap.add_argument("--points", type=int, default=1 << 20, help="ccd_drape: query points")
    ap.add_argument("--image", default="", help="rays_drape: write the drape frame's depth buffer (PGM) here")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch512":
        run_batch_bench(args)
        return
    if args.workload == "mlp16384":
        run_mlp_bench(args)
        return
    if args.workload == "learned64":
        run_learned_bench(args)
        return
    if args.workload == "twist30":
        run_twist_bench(args)
        return
    if args.workload == "rays_drape":
        run_rays_bench(args)
        return
    if args.workload == "ccd_drape":
        run_ccd_bench(args)
        return
    if args.workload == "direct":
        run_direct_bench(args)
        return

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2312_14839_gb300 import bhem
    bhem.load()

    line = step_workload_line(args, args.workload, dist, world, rank, full=True)
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "sheet256":
        line["workloads"] = extra_workloads(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        line["cpu_baseline"], line["cpu_baseline_single_thread"] = cpu_baselines(args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def step_workload_line(args, workload, dist, world, rank, full=True):
    """One Newton iteration of the implicit-Euler step per bench step (newton_max = 1, 50 PCG
    iterations) on a sinusoid-displaced shell: device-timed steps, and with full=True the end-to-
    end (host buffers) leg, the SpMV roofline, the arithmetic rooflines and the element-only
    rate."""
    import torch
    from paper_2312_14839_gb300 import bhem
    g, mat, rest, q0 = make_workload(workload)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    rest_d = torch.as_tensor(rest.reshape(-1), device=dev)
    q0_d = torch.as_tensor(q0.reshape(-1), device=dev)
    sh = bhem.Shell(g, mat, rest_d, precision="mixed", stream=stream, spmv=args.spmv)
    P = bhem.step_params(dt=1e-3, newton_max=1, pcg_fixed_iters=50)
    q = q0_d.clone()
    v = torch.zeros_like(q)
    v0 = torch.zeros_like(q)

    def step():
        # every step restarts from the same state; the regulariser level of the previous step is
        # carried in (tau_carry), as a simulation carries it from step to step
        q.copy_(q0_d)
        v.copy_(v0)
        st = sh.newton_step(q, v, P)
        P.tau_carry = st["tau_final"]
        return st

    stats = None
    # the clock sampler starts before the warm-up, and its start-up (NVML) is over before the
    # timed region opens
    with ClockSampler(torch.cuda.current_device()) as clk:
        clk.wait_first()
        for _ in range(args.warmup):
            stats = step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        launches0 = sh.kernel_launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk.mark()
        torch.cuda.synchronize()
        ev0.record(stream)
        newton_iters, spmvs = 0, 0
        for _ in range(args.steps):
            stats = step()
            newton_iters += stats["newton_iters"]
            spmvs += stats["pcg_iters_total"]
        ev1.record(stream)
        torch.cuda.synchronize()
        launches = sh.kernel_launches() - launches0
        ms, total_iters = reduce_over_ranks(dist, ev0.elapsed_time(ev1), newton_iters, dev)
        sec = ms / 1e3
        value = g.n_patches * total_iters / sec
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded sinusoid displacement, no external data)",
            "config": {"workload": WORKLOADS[workload], "patches": g.n_patches, "nodes": g.n_nodes,
                       "dof": g.n_dof, "bsr_blocks": sh.n_blocks, "newton_iterations_per_step": 1,
                       "pcg_iterations_per_solve": 50, "precision": "mixed",
                       "l2": "inputs larger than L2 (FP32 BSR 340 MB)" if workload == "sheet256"
                             else "working set smaller than L2 (not flushed)",
                       "parallelism": f"replicas{world}" if world > 1 else "single GPU"},
            "newton_steps_per_s": total_iters / sec,
            "pcg_iterations_per_step": spmvs / args.steps,
            "gpu_launches": launches,
            "last_step_stats": stats,
        }
        if not full:
            line["clocks"] = clk.summary()
            sh.close()
            return line

        # e2e: the same Newton iteration through the C ABI with pinned host buffers (H2D of q, v
        # and D2H of q, v inside the timed region). Every step starts from the same host state as
        # the device-timed steps; the host-side reset of the pinned buffers is outside the timed
        # calls.
        qh = torch.empty(g.n_dof, dtype=torch.float64, pin_memory=True)
        vh = torch.empty(g.n_dof, dtype=torch.float64, pin_memory=True)
        qh_np, vh_np = qh.numpy(), vh.numpy()
        q0_flat = np.ascontiguousarray(q0.reshape(-1))

        def e2e_step():
            np.copyto(qh_np, q0_flat)
            vh_np.fill(0.0)
            t = time.perf_counter()
            st = sh.newton_step(qh_np, vh_np, P)   # synchronous: returns host stats
            el = time.perf_counter() - t
            P.tau_carry = st["tau_final"]
            return st["newton_iters"], el

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        e2e_iters, e2e_sec = 0, 0.0
        for _ in range(args.steps):
            it, dt_ = e2e_step()
            e2e_iters += it
            e2e_sec += dt_
        line["clocks"] = clk.summary()
    e2e_sec, e2e_iters = reduce_over_ranks(dist, e2e_sec, e2e_iters, dev)
    m = g.n_dof
    line["e2e"] = {"value": g.n_patches * e2e_iters / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": 2 * m * 8,
                   "d2h_bytes_per_step": 2 * m * 8}

    # roofline of the dominant kernel (the FP32 BSR SpMV, one launch per PCG iteration), timed
    # live with CUDA events on the shell's stream over back-to-back launches on the assembled
    # matrix
    sh.energy_grad_hess(q0_d, mass_scale=1.0 / P.dt ** 2, want_energy=False, want_grad=False)
    x = torch.randn(g.n_dof, dtype=torch.float32, device=dev)
    y = torch.empty(g.n_dof, dtype=torch.float32, device=dev)
    for _ in range(5):
        sh.spmv(x, y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("spmv_roofline")
    e0.record(stream)
    for _ in range(args.spmv_reps):
        sh.spmv(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    spmv_s = e0.elapsed_time(e1) / 1e3 / args.spmv_reps
    nb, n = sh.n_blocks, sh.n_nodes
    sym = args.spmv != "tma" and os.environ.get("BHEM_SPMV_SYM") == "1"
    if sym:
        # diagonal and upper blocks once, column indices, the transpose map of the lower blocks,
        # row pointers, diagonal positions, x and y
        spmv_bytes = ((nb + n) // 2) * 144 * 4 + nb * 4 + ((nb - n) // 2) * 4 + (n + 1) * 4 + n * 4 + m * 4 + m * 4
    else:
        spmv_bytes = nb * 144 * 4 + nb * 4 + (n + 1) * 4 + m * 4 + m * 4
    peak, peak_kind = measured_peaks()
    achieved = spmv_bytes / spmv_s / 1e9
    traffic = recorded_traffic(os.path.join(ROOT, "paper_2312_14839_gb300", "csrc", "solver.cu"),
                               "k_spmv32_tma" if args.spmv == "tma" else "k_spmv32_sym" if sym else "k_spmv32",
                               workload)
    line["roofline"] = {
        "kernel": ("k_spmv32_tma (FP32 12x12 BSR SpMV of the PCG, bulk-copy pipelined)" if args.spmv == "tma" else
                   "k_spmv32_sym (FP32 12x12 BSR SpMV of the PCG: diagonal and upper blocks streamed, lower "
                   "blocks read as their transposes through L2)" if sym else
                   "k_spmv32 (FP32 12x12 BSR SpMV of the PCG, both triangles streamed)"),
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.8 TB/s",
        "traffic": traffic, "algorithmic_bytes_per_launch": spmv_bytes, "avg_launch_us": spmv_s * 1e6}
    line["alu_rooflines"] = alu_rooflines(sh, q0_d, P, g.n_patches, stream)
    # the warp-level tensor-core rates beside the FP32 FMA peak: what a TF32 split of the element
    # contraction could run at (three TF32 products per FP32-accurate product)
    line["warp_mma_peaks_tflops"] = {"tf32_m16n8k8": bhem.measure_mma_peak(0, 2048, stream) / 1e12,
                                     "bf16_m16n8k16": bhem.measure_mma_peak(1, 2048, stream) / 1e12}
    line["element_kernel_only"] = element_kernel_only(sh, q0_d, g.n_patches, stream)
    sh.close()
    return line


def extra_workloads(args):
    """The other configurations of the metric, measured in the same run: the 280x5 annulus step,
    the 512-sheet batch (batched against plain), the learned warm start (against the zero guess
    and the inertial predictor) and the 200-step twist (exact and pseudo Hessian)."""
    out = {}
    t0 = time.perf_counter()
    ann = step_workload_line(args, "annulus280x5", None, 1, 0, full=False)
    out["annulus280x5"] = {k: ann[k] for k in ("value", "unit", "ms_per_step", "newton_steps_per_s",
                                               "pcg_iterations_per_step", "gpu_launches", "clocks")}
    out["annulus280x5"]["patches"] = ann["config"]["patches"]
    b = batch_line(args, steps=min(args.steps, 5), warmup=2, plain_reps=1)
    out["batch512"] = {k: b[k] for k in ("sheet_steps_per_s", "plain_sheet_steps_per_s", "batched_vs_plain",
                                         "value", "plain_value", "unit", "newton_iters_per_sheet",
                                         "all_sheets_converged_1e-8", "steps", "clocks")}
    out["batch512"]["autotuned"] = b["config"]["autotuned"]
    lr = learned_line(args)
    out["learned64"] = {k: lr[k] for k in ("learned", "plain_zero_guess", "inertial_predictor",
                                           "learned_vs_plain", "learned_vs_inertial", "train",
                                           "data_generation", "clocks")}
    tw = twist_line(args)
    out["twist30"] = {k: tw[k] for k in ("exact_hessian", "pseudo_hessian", "pseudo_vs_exact_steps_per_s",
                                         "clocks")}
    out["seconds"] = time.perf_counter() - t0
    return out


if __name__ == "__main__":
    main()
