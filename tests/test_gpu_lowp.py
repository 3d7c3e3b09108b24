"""16-bit grid storage (bf16 / fp16 with a float32 code per block, float32 arithmetic) against
the float64 oracle: relative L2 and L-infinity errors after the full step count.  The bar is
relative L2 <= 1e-2; the float32 engine's own error is the control."""
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


def run(st, w, steps, storage, T=0, vec=0, by=0):
    import torch
    u = torch.from_numpy(w.u0).cuda()
    p = None if w.power is None else torch.from_numpy(w.power).cuda()
    out = torch.full_like(u, float("nan"))
    plan = st.Plan(w.kind, 2, w.nx, w.ny, storage=storage, force_T=T, force_vec=vec, partial_rows=by)
    plan.run(u, out, w.coef, steps, power=p)
    plan.sync()
    plan.close()
    return out.cpu().numpy().astype(np.float64)


def errs(g, o):
    d = g - o
    return (float(np.linalg.norm(d) / np.linalg.norm(o)),
            float(np.max(np.abs(d)) / np.max(np.abs(o))))


@pytest.mark.parametrize("storage,bound", [(1, 1e-2), (2, 1e-3)])
def test_lowp_configs(eng, orc, storage, bound):
    cases = [synth.c1_diffusion2d(), synth.c2_thermal2d(nx=2048, ny=2048, steps=1000)]
    for w in cases:
        ref = orc.run(w.kind, w.u0, w.coef, w.steps, w.power, dtype=np.float64)
        l2, linf = errs(run(eng, w, w.steps, storage), ref)
        f32_l2, _ = errs(run(eng, w, w.steps, 0), ref)
        assert l2 <= bound, (w.name, storage, l2, linf)
        assert np.isfinite(linf)
        # 16-bit storage never beats float32 storage (sanity of the control)
        assert l2 >= f32_l2 * 0.5


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("shape", [(0, 0, 0), (8, 4, 0), (2, 4, 0), (1, 4, 0)])
def test_lowp_edges(eng, orc, storage, kind, shape):
    # ragged sizes, one-row and one-column grids, step counts not divisible by T; the default
    # shape (T = 8, 8 cells per lane, partial rows in place) and the two-row variants
    # Bound: the input is coded as (x - mid) / half with mid and half the block's mid-range and
    # half-range, every pass's output as x - offset with the offset one cell of the block; each
    # is rounded to 16 bits, an error of at most u times the coded magnitude (u = 2^-9 bf16,
    # 2^-12 fp16: half an ulp), so at most u * range per cell, range the field's range; the
    # update is a convex combination (plus a source), so the P + 1 roundings of P passes add up
    # to at most (P + 1) u range, range the larger of the input's and the result's (diffusion
    # never widens it, the Hotspot source can).  Relative L2 <= max error / rms of the result;
    # the test takes the tighter of that bound (x 1.5) and the configs' 1e-2.
    T, vec, by = shape
    u = 2.0 ** -9 if storage == 1 else 2.0 ** -12
    for t, (nx, ny, steps) in enumerate([(301, 77, 17), (1, 40, 9), (57, 1, 12), (250, 250, 8),
                                         (1000, 3, 5)]):
        w = synth.make(kind, 2, nx, ny, seed=6000 + 13 * t + kind)
        ref = orc.run(kind, w.u0, w.coef, steps, w.power, dtype=np.float64)
        g = run(eng, w, steps, storage, T, vec, by)
        l2, _ = errs(g, ref)
        passes = -(-steps // (T or 8))
        rng = max(float(w.u0.max() - w.u0.min()), float(ref.max() - ref.min()))
        rms = float(np.sqrt(np.mean(ref ** 2)))
        bound = min(1e-2, 1.5 * (passes + 1) * u * rng / rms)
        assert l2 <= bound, (nx, ny, steps, storage, l2, bound)
    # zero steps copies the input exactly
    w = synth.make(kind, 2, 33, 21, seed=6100 + kind)
    assert np.array_equal(run(eng, w, 0, storage), w.u0.astype(np.float64))
