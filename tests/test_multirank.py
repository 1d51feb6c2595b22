"""Host logic of the multi-process bench path, run as world-size-2 gloo ranks on the CPU.

Under torchrun each rank runs an independent replica of the workload (weak scaling, no data-path
collective); the only cross-rank step is the reduction of the timed region (max over ranks) and
of the work done (sum over ranks), and the reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, figures):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sec, units = figures[rank]
        got = bench.reduce_over_ranks(dist, sec, units)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(list(got), f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_without_process_group_is_identity():
    assert bench.reduce_over_ranks(None, 0.25, 7) == (0.25, 7.0)


def test_reduce_over_two_gloo_ranks(tmp_path):
    # rank 1 is the slower one: the job time is its time, the work is both ranks' work
    figures = [(0.125, 3), (0.5, 4)]
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path), figures), nprocs=2,
                       join=True, start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"rank{r}.json") as f:
            sec, units = json.load(f)
        assert sec == 0.5
        assert units == 7.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(workload="sheet256", steps=1, warmup=3, gpus=2, impl="reference")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""


@pytest.mark.timeout(300)
def test_reference_arm_under_torchrun_two_ranks():
    """The launch the scaling run uses: torchrun, two ranks; rank 0 prints one JSON line and both
    ranks exit 0 (the reference arm is CPU-only, so this runs without a GPU)."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=280)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["n_gpus"] == 2
    assert line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
