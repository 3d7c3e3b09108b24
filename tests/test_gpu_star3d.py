"""GPU parity of the 3D star diffusion of radius R (Eqs. 1-2 with rad > 1; R = 2 is the
13-point stencil) against the oracle, through the C ABI.

Exact plans evaluate each cell in the oracle's order with one rounding per operation: the result
must be bit-identical to the float32 oracle.  Contracted plans use fused multiply-adds in the
same order: max relative error <= 1e-5 after the full step count (every cell is a convex
combination of its neighbours, so nothing amplifies the per-step rounding).
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
    plan = st.Plan(0, 3, w.nx, w.ny, w.nz, rad=R, exact=exact, force_T=T)
    info = plan.info()
    plan.run(u, out, w.coef, steps)
    plan.sync()
    plan.close()
    return out.cpu().numpy(), info


# (nx, ny, nz): one cell, thin and ragged grids around the 56..60-cell compute blocks, odd widths
# (plain-load staging) and widths of a multiple of 4 (tensor-map staging), z long enough for
# several z-segments
SIZES = [(1, 1, 1), (3, 2, 5), (2, 9, 1), (13, 11, 7), (61, 5, 9), (64, 64, 20), (121, 67, 33),
         (117, 130, 18), (200, 61, 70)]


@pytest.mark.parametrize("R,T", [(2, 1), (2, 2), (3, 1), (4, 1)])
def test_star3d_exact_bitwise(eng, orc, R, T):
    for t, (nx, ny, nz) in enumerate(SIZES):
        w = synth.make_star(3, R, nx, ny, nz, seed=9700 + 17 * t + R)
        for steps in sorted({1, T, T + 1, 2 * T + 1}):
            g, info = run(eng, w, R, steps, True, T)
            assert info["T"] == T and info["kernel_id"] == 6
            o = orc.run_star(R, w.u0, w.coef, steps)
            assert np.array_equal(g, o), (R, T, nx, ny, nz, steps, max_rel(g, o))


@pytest.mark.parametrize("R,T", [(2, 1), (2, 2), (3, 1), (4, 1)])
def test_star3d_contracted(eng, orc, R, T):
    for t, (nx, ny, nz) in enumerate(SIZES[::2] + [(260, 130, 40)]):
        w = synth.make_star(3, R, nx, ny, nz, seed=9800 + 13 * t + R)
        for steps in sorted({1, 2 * T + 1, 12}):
            g, _ = run(eng, w, R, steps, False, T)
            o = orc.run_star(R, w.u0, w.coef, steps)
            assert max_rel(g, o) <= TOL, (R, T, nx, ny, nz, steps, max_rel(g, o))


@pytest.mark.parametrize("exact", [True, False])
def test_star3d_in_place_and_default(eng, orc, exact):
    for nx, ny, nz in [(99, 70, 23), (128, 60, 31)]:
        w = synth.make_star(3, 2, nx, ny, nz, seed=9900 + nx)
        for steps in (3, 4):        # odd and even pass counts in place
            g, info = run(eng, w, 2, steps, exact, inplace=True)
            assert info["T"] == 1 and info["bx"] == 64
            o = orc.run_star(2, w.u0, w.coef, steps)
            if exact:
                assert np.array_equal(g, o), (nx, ny, nz, steps)
            else:
                assert max_rel(g, o) <= TOL, (nx, ny, nz, steps)
            g, info = run(eng, w, 2, steps, exact, T=2, inplace=True)
            assert info["T"] == 2
            o = orc.run_star(2, w.u0, w.coef, steps)
            if exact:
                assert np.array_equal(g, o), (nx, ny, nz, steps)
            else:
                assert max_rel(g, o) <= TOL, (nx, ny, nz, steps)


def test_star3d_unsupported(eng):
    st = eng
    for kw in (dict(force_T=4), dict(force_bx=128), dict(kind=1), dict(rad=5),
               dict(storage=st.ST_BF16)):
        args = dict(kind=0, rad=2)
        args.update(kw)
        kind = args.pop("kind")
        with pytest.raises(st.StencilError) as e:
            st.Plan(kind, 3, 40, 30, 20, **args)
        assert e.value.code == st.ST_ERR_UNSUPPORTED, kw
