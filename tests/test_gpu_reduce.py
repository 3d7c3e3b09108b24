"""Float64 verification reductions on the GPU against numpy float64, and a full-size property of
the engine that needs them: with symmetric coefficients summing to one, the grid sum of a
Diffusion 2D run is conserved (Sec. 5.1 clamped boundary; the boundary flux cancels)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_00438_gb300 as st
    return st


@pytest.mark.parametrize("n", [1, 7, 1000, 262145, 5_000_003])
def test_reduce_matches_numpy(eng, n):
    import torch
    a = synth.uniform_f32(77, n, -3.0, 5.0)
    b64 = synth.uniform01(78, n) * 2.0
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b64).cuda()
    r = eng.stencil_reduce(ta, tb)
    a64 = a.astype(np.float64)
    assert r["sum_a"] == pytest.approx(a64.sum(), rel=1e-12, abs=1e-9)
    assert r["sumsq_a"] == pytest.approx((a64 * a64).sum(), rel=1e-12)
    assert r["maxabs_a"] == np.abs(a64).max()
    assert r["sum_b"] == pytest.approx(b64.sum(), rel=1e-12)
    assert r["sumsq_diff"] == pytest.approx(((a64 - b64) ** 2).sum(), rel=1e-12)
    assert r["maxabs_diff"] == np.abs(a64 - b64).max()
    r1 = eng.stencil_reduce(ta)
    assert r1["sum_a"] == r["sum_a"] and r1["sumsq_diff"] == 0.0
    r2 = eng.stencil_reduce(ta, tb)
    assert r2 == r   # deterministic


@pytest.mark.slow
def test_sum_conserved_full_size(eng):
    """16384^2, 1000 steps, cw = ce, cn = cs: the float64 grid sum moves only by float32
    rounding of the updates (random-walk bound), never by a boundary or tiling error."""
    import torch
    nx = ny = 16384
    u0 = synth.uniform_f32(41, nx * ny, 0.0, 1.0).reshape(ny, nx)
    k = np.array([0.36, 0.12, 0.12, 0.2, 0.2], np.float32)
    u = torch.from_numpy(u0).cuda()
    out = torch.empty_like(u)
    plan = eng.Plan(0, 2, nx, ny)
    plan.run(u, out, k, 1000)
    plan.sync()
    s0 = eng.stencil_reduce(u)["sum_a"]
    r = eng.stencil_reduce(out)
    # coefficient rounding: sum(k) in float32 differs from 1 by at most a few ulp per step
    drift = abs(float(np.sum(k.astype(np.float64))) - 1.0) * 1000 * s0
    assert abs(r["sum_a"] - s0) <= 1e-6 * s0 + drift
    assert r["sumsq_a"] <= eng.stencil_reduce(u)["sumsq_a"]   # energy does not grow
    assert 0.0 <= u0.min() and r["maxabs_a"] <= float(u0.max())  # maximum principle
