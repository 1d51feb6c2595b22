"""Point-patch continuous collision detection (Sec. 5, Eq. ineqccd) on the GPU against the FP64
oracle, through the C ABI. As for the ray search, both sides run the same IEEE FP64 operations
in the same order, so every output must agree bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2312_14839_gb300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _gpu_ccd(g, q, dq, x0, dx, variant):
    from paper_2312_14839_gb300.bhem import Shell
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    with Shell(g, S.SHEET_MATERIAL, t(q).reshape(-1), precision="fp64") as sh:
        out = sh.ccd_points(t(q).reshape(-1), t(dq).reshape(-1), t(x0).reshape(-1, 3), t(dx).reshape(-1, 3),
                            variant=variant, want_stats=True)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}


def _assert_identical(gpu, ref, what):
    s, patch, uv, flags, stats = ref
    np.testing.assert_array_equal(gpu["flags"], flags, err_msg=what)
    np.testing.assert_array_equal(gpu["patch"], patch, err_msg=what)
    np.testing.assert_array_equal(gpu["s"], s, err_msg=what)
    np.testing.assert_array_equal(gpu["uv"], uv, err_msg=what)
    np.testing.assert_array_equal(gpu["stats"], stats, err_msg=what)


@pytest.mark.parametrize("scene", ["plane", "drape", "static", "cylinder"])
@pytest.mark.parametrize("variant", ["newton", "midpoint"])
def test_scenes_bit_identical(scene, variant):
    """1,500 points (several CTAs and a ragged last one) per scene and split; the cylinder is
    periodic in u, so its patches wrap around the seam."""
    g, q, dq, x0, dx = S.ccd_scene(scene, 1500)
    ref = O.ccd_points(g, q, dq, x0, dx, variant == "newton", want_stats=True)
    gpu = _gpu_ccd(g, q, dq, x0, dx, variant)
    _assert_identical(gpu, ref, f"{scene} {variant}")
    hits = int((ref[3] & 1).sum())
    assert 100 < hits < 1400


def test_edge_cases():
    """Points that start on the surface (contact at s = 0), points that do not move, points far
    from the shell, and an empty batch."""
    g, q, dq, x0, dx = S.ccd_scene("drape", 64)
    import ray_brute as RB
    on = []
    for p, (u, v) in ((0, (0.3, 0.7)), (457, (0.5, 0.5)), (899, (0.9, 0.1))):
        X, _, _ = RB.evaluate(RB.patch_coeffs(g, q, p), np.array([u]), np.array([v]))
        on.append(X[0])
    x0 = np.concatenate([x0, np.array(on), x0[:8], np.array([[5.0, 5.0, 5.0], [-3.0, 0.5, 0.0]])])
    dx = np.concatenate([dx, np.tile([0.0, 0.0, 0.01], (3, 1)), np.zeros((8, 3)),
                         np.array([[0.1, 0.0, 0.0], [0.0, 0.0, 0.5]])])
    for variant in ("newton", "midpoint"):
        ref = O.ccd_points(g, q, dq, x0, dx, variant == "newton", want_stats=True)
        gpu = _gpu_ccd(g, q, dq, x0, dx, variant)
        _assert_identical(gpu, ref, variant)
        assert (ref[3][64:67] & 1).all() and (ref[0][64:67] <= 1e-8).all()
        assert not (ref[3][-2:] & 1).any()
    from paper_2312_14839_gb300.bhem import Shell
    with Shell(g, S.SHEET_MATERIAL, torch.as_tensor(q.reshape(-1), device="cuda"), precision="fp64") as sh:
        e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
        dq_d = torch.as_tensor(dq.reshape(-1), device="cuda")
        assert sh.ccd_points(dq_d, dq_d, e, e)["s"].numel() == 0


def test_full_size_batch_sampled():
    """The benchmark's batch (262,144 points against the deforming 30 x 30 drape): nothing
    flagged, and a seeded sample of 600 points identical to the oracle."""
    g, q, dq, x0, dx = S.ccd_scene("drape", 262144)
    rng = np.random.default_rng(13)
    idx = np.sort(rng.choice(len(x0), 600, replace=False))
    for variant in ("newton", "midpoint"):
        gpu = _gpu_ccd(g, q, dq, x0, dx, variant)
        assert not (gpu["flags"] & 6).any()
        ref = O.ccd_points(g, q, dq, x0[idx], dx[idx], variant == "newton", want_stats=True)
        _assert_identical({k: v[idx] for k, v in gpu.items()}, ref, variant)


def test_heap_spill_and_second_pass():
    """Points sliding inside a flat, static 110 x 110 sheet keep up to 267 candidates (the oracle's
    unbounded heap): 184 of the 300 outgrow the first pass's 256 entries, more than the 128 global
    heaps, so both the in-place spill and the second pass run. Every point is bit-identical to
    the oracle and none is flagged."""
    from paper_2312_14839_gb300.bhem import RAY_HEAP
    g, q = S.flat_sheet(110, 110)
    dq = np.zeros_like(q)
    angs = np.concatenate([np.array([0.3, 0.5]), np.linspace(0.70, 0.87, 298)])
    x0 = np.stack([-0.05 * np.ones_like(angs), -0.05 * np.tan(angs), np.zeros_like(angs)], axis=1)
    dx = 2.0 * np.stack([np.cos(angs), np.sin(angs), np.zeros_like(angs)], axis=1)
    for variant in ("newton", "midpoint"):
        ref = O.ccd_points(g, q, dq, x0, dx, variant == "newton", want_stats=True)
        assert 128 < int((ref[4][:, 1] > RAY_HEAP).sum()) < len(x0)
        gpu = _gpu_ccd(g, q, dq, x0, dx, variant)
        _assert_identical(gpu, ref, variant)
