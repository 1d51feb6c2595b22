"""Ray-patch intersection (Sec. 5) on the GPU against the FP64 oracle, through the C ABI.

Both sides run the same sequence of IEEE FP64 operations (the CUDA file is compiled without
mul-add contraction, the oracle as plain ISO C), so hits, patches, tau, (u, v), flags and the
search statistics must agree bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _shell(g, q):
    from paper_2312_14839_gb300.bhem import Shell
    rest = torch.as_tensor(np.ascontiguousarray(q).reshape(-1), dtype=torch.float64, device="cuda")
    return Shell(g, S.SHEET_MATERIAL, rest, precision="fp64")


def _gpu_trace(sh, q, o, d, variant):
    dq = torch.as_tensor(np.ascontiguousarray(q).reshape(-1), dtype=torch.float64, device="cuda")
    do = torch.as_tensor(o, dtype=torch.float64, device="cuda")
    dd = torch.as_tensor(d, dtype=torch.float64, device="cuda")
    out = sh.trace_rays(dq, do, dd, variant=variant, want_stats=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _assert_identical(gpu, ref, what):
    tau, patch, uv, flags, stats = ref
    np.testing.assert_array_equal(gpu["flags"], flags, err_msg=what)
    np.testing.assert_array_equal(gpu["patch"], patch, err_msg=what)
    np.testing.assert_array_equal(gpu["tau"], tau, err_msg=what)
    np.testing.assert_array_equal(gpu["uv"], uv, err_msg=what)
    np.testing.assert_array_equal(gpu["stats"], stats, err_msg=what)


@pytest.mark.parametrize("scene", ["plane", "cylinder", "drape"])
@pytest.mark.parametrize("variant", ["newton", "midpoint"])
def test_camera_rays_bit_identical(scene, variant):
    """A 40 x 30 camera (1200 rays over several CTAs and a ragged last one) on each scene."""
    g, q, eye, tgt = S.ray_scenes()[scene]
    o, d = S.camera_rays(40, 30, eye, tgt)
    ref = O.trace_rays(g, q, o, d, variant == "newton", want_stats=True)
    with _shell(g, q) as sh:
        gpu = _gpu_trace(sh, q, o, d, variant)
    _assert_identical(gpu, ref, f"{scene} {variant}")
    hits = int((ref[3] & 1).sum())
    assert 100 < hits < len(o)


def test_camera_inside_cylinder_and_axis_parallel_rays():
    """Origins inside the root boxes (a camera on the cylinder's axis looking at the wall, so
    tau_min = 0) and rays with zero direction components."""
    g, q = S.cylinder(10, 10)
    o1, d1 = S.camera_rays(17, 13, (0.0, 0.0, 0.5), (1.0, 0.2, 0.6))
    o2 = np.array([[0.0, 0.0, 0.5], [0.0, 0.0, 0.5], [0.0, 0.0, -1.0], [0.5, 0.5, 0.5], [0.0, 0.0, 0.5]])
    d2 = np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, 1.0], [0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])
    o, d = np.concatenate([o1, o2]), np.concatenate([d1, d2])
    for variant in ("newton", "midpoint"):
        ref = O.trace_rays(g, q, o, d, variant == "newton", want_stats=True)
        with _shell(g, q) as sh:
            gpu = _gpu_trace(sh, q, o, d, variant)
        _assert_identical(gpu, ref, variant)
        assert (ref[3][: len(o1)] & 1).all()


def test_first_pass_overflow_is_traced_again():
    """Rays lying in a flat 110 x 110 sheet keep up to ~270 candidates in the oracle's unbounded
    heap. Rays that outgrow the first pass's SHELL_RAY_HEAP = 256 entries are traced again with
    the larger heap: every ray, including more such rays than the second pass has threads, is
    bit-identical to the oracle and none is flagged."""
    from paper_2312_14839_gb300.bhem import RAY_HEAP
    g, q = S.flat_sheet(110, 110)
    angs = np.concatenate([np.array([0.3, 0.5]), np.linspace(0.70, 0.87, 298)])
    o = np.stack([-0.05 * np.ones_like(angs), -0.05 * np.tan(angs), np.zeros_like(angs)], axis=1)
    d = np.stack([np.cos(angs), np.sin(angs), np.zeros_like(angs)], axis=1)
    for variant in ("newton", "midpoint"):
        ref = O.trace_rays(g, q, o, d, variant == "newton", want_stats=True)
        over = int((ref[4][:, 1] > RAY_HEAP).sum())
        assert 128 < over < len(o), over
        with _shell(g, q) as sh:
            gpu = _gpu_trace(sh, q, o, d, variant)
        _assert_identical(gpu, ref, variant)


def test_empty_and_all_miss():
    g, q, eye, tgt = S.ray_scenes()["drape"]
    with _shell(g, q) as sh:
        e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
        dq = torch.as_tensor(q.reshape(-1), dtype=torch.float64, device="cuda")
        out = sh.trace_rays(dq, e, e)
        assert out["tau"].numel() == 0
        o = np.tile([0.5, 0.5, 1.0], (300, 1))
        d = np.tile([0.0, 0.0, 1.0], (300, 1))
        gpu = _gpu_trace(sh, q, o, d, "newton")
    assert np.isinf(gpu["tau"]).all() and (gpu["patch"] == -1).all() and (gpu["flags"] == 0).all()


def test_full_size_camera_sampled():
    """The benchmark's workload (1024 x 768 camera on the 30 x 30 draped sheet): no ray flagged,
    and a seeded sample of 600 rays identical to the oracle."""
    g, q, eye, tgt = S.ray_scenes()["drape"]
    o, d = S.camera_rays(1024, 768, eye, tgt)
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(len(o), 600, replace=False))
    with _shell(g, q) as sh:
        for variant in ("newton", "midpoint"):
            gpu = _gpu_trace(sh, q, o, d, variant)
            assert not (gpu["flags"] & 6).any()
            ref = O.trace_rays(g, q, o[idx], d[idx], variant == "newton", want_stats=True)
            _assert_identical({k: v[idx] for k, v in gpu.items()}, ref, variant)
            assert 0.4 < (gpu["flags"] & 1).mean() < 0.8
