"""GPU parity of the star diffusion of radius R (Eqs. 1-2 with rad > 1) against the oracle.

Exact plans evaluate each cell in the oracle's order with one rounding per operation: the result
must be bit-identical to the float32 oracle.  Contracted plans use fused multiply-adds in the
same order: max relative error <= 1e-5 after the full step count.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_00438_gb300 as st
    return st


def max_rel(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    floor = 1e-6 * max(np.max(np.abs(o)), 1e-300)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), floor)))


def run(st, w, R, steps, exact, T=0, inplace=False):
    import torch
    u = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda()
    out = u if inplace else torch.full_like(u, float("nan"))
    plan = st.Plan(0, 2, w.nx, w.ny, rad=R, exact=exact, force_T=T)
    info = plan.info()
    plan.run(u, out, w.coef, steps)
    plan.sync()
    plan.close()
    return out.cpu().numpy(), info


# ragged sizes around the 112..120-cell compute blocks, one-cell and thin grids, an odd width
# (plain-load staging) and widths of a multiple of 4 (tensor-map staging)
SIZES = [(1, 1), (3, 2), (2, 9), (13, 11), (117, 5), (128, 128), (241, 130), (300, 257), (333, 201)]


@pytest.mark.parametrize("R,T", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2), (3, 4), (4, 1), (4, 2)])
def test_star_exact_bitwise(eng, orc, R, T):
    for t, (nx, ny) in enumerate(SIZES):
        w = synth.make_star(2, R, nx, ny, seed=9000 + 17 * t + R)
        for steps in sorted({1, T, T + 1, 3 * T + 2}):
            g, info = run(eng, w, R, steps, True, T)
            assert info["T"] == T and info["kernel_id"] == 5
            o = orc.run_star(R, w.u0, w.coef, steps)
            assert np.array_equal(g, o), (R, T, nx, ny, steps, max_rel(g, o))


@pytest.mark.parametrize("R", [2, 3, 4])
def test_star_contracted(eng, orc, R):
    for t, (nx, ny) in enumerate(SIZES[3:] + [(1000, 600)]):
        w = synth.make_star(2, R, nx, ny, seed=9100 + 13 * t + R)
        for steps in (1, 7, 60):
            g, info = run(eng, w, R, steps, False)
            o = orc.run_star(R, w.u0, w.coef, steps)
            assert max_rel(g, o) <= TOL, (R, nx, ny, steps, info["T"], max_rel(g, o))


@pytest.mark.parametrize("R", [2, 4])
def test_star_in_place_and_errors(eng, orc, R):
    w = synth.make_star(2, R, 260, 140, seed=9200 + R)
    for steps in (5, 8):   # odd and even pass counts with the default T
        g, _ = run(eng, w, R, steps, True, inplace=True)
        o = orc.run_star(R, w.u0, w.coef, steps)
        assert np.array_equal(g, o), (R, steps)
    with pytest.raises(eng.StencilError):      # radius above the compiled range
        eng.Plan(0, 2, 64, 64, rad=5)
    with pytest.raises(eng.StencilError):      # star Hotspot is not defined
        eng.Plan(1, 2, 64, 64, rad=2)
    with pytest.raises(eng.StencilError):      # 2D star tiles are 128 wide
        eng.Plan(0, 2, 64, 64, rad=2, force_bx=64)
