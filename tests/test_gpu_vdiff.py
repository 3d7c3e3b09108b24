"""GPU parity of diffusion 2D with per-cell coefficients (Table 2 row 1 with its coefficients as
arrays, Sec. 5.1), through the C ABI, against the CPU oracle on the same seeded inputs.

Bars: exact plans (Table 2 order, one rounding per operation) bit-identical to the float32
oracle; contracted plans (fused multiply-adds) within max relative error 1e-5 (the same bound
as the constant-coefficient kernels: every cell is a convex combination of its neighbours, so
contraction changes each step by a few ulp and nothing amplifies it)."""
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


def gpu_run(st, w, steps, exact=False, T=0, bx=0, inplace=False):
    import torch
    u = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda()
    k = torch.from_numpy(np.ascontiguousarray(w.coef)).cuda()
    out = u if inplace else torch.full_like(u, float("nan"))
    plan = st.Plan(st.ST_DIFFUSION_VAR, 2, w.nx, w.ny, exact=exact, force_T=T, force_bx=bx)
    plan.run(u, out, None, steps, power=k)
    plan.sync()
    info = plan.info()
    plan.close()
    return out.cpu().numpy(), info


SIZES = [(1, 1), (1, 7), (7, 1), (2, 2), (5, 3), (13, 11), (31, 17), (97, 61), (130, 67),
         (257, 129), (509, 263), (1031, 45)]


@pytest.mark.parametrize("T,bx", [(1, 128), (2, 512), (4, 128), (4, 512), (8, 128), (8, 512)])
def test_exact_bitwise(eng, orc, T, bx):
    for t, (nx, ny) in enumerate(SIZES):
        w = synth.make_vdiff(nx, ny, seed=9300 + 17 * t)
        for steps in sorted({0, 1, max(T - 1, 1), T, T + 1, 2 * T + 3}):
            g, info = gpu_run(eng, w, steps, exact=True, T=T, bx=bx)
            assert info["T"] == T and info["bx"] == bx
            o = orc.run_vdiff2d(w.u0, w.coef, steps)
            assert np.array_equal(g, o), (nx, ny, steps, max_rel(g, o))


@pytest.mark.parametrize("T,bx", [(1, 0), (2, 0), (4, 128), (4, 512), (8, 0)])
def test_contracted(eng, orc, T, bx):
    for t, (nx, ny) in enumerate(SIZES[::2] + [(700, 300)]):
        w = synth.make_vdiff(nx, ny, seed=9400 + 13 * t)
        for steps in sorted({1, T, 2 * T + 1, 37}):
            g, _ = gpu_run(eng, w, steps, T=T, bx=bx)
            o = orc.run_vdiff2d(w.u0, w.coef, steps)
            assert max_rel(g, o) <= TOL, (nx, ny, steps, max_rel(g, o))


@pytest.mark.parametrize("exact", [True, False])
def test_in_place_and_unaligned_rows(eng, orc, exact):
    for nx, ny in [(203, 91), (516, 77)]:   # odd pitch (plain copies) and a 16-byte multiple
        w = synth.make_vdiff(nx, ny, seed=9500 + nx)
        for steps in (7, 8):                # odd and even pass counts in place
            g, _ = gpu_run(eng, w, steps, exact=exact, T=4, inplace=True)
            o = orc.run_vdiff2d(w.u0, w.coef, steps)
            if exact:
                assert np.array_equal(g, o), (nx, ny, steps)
            else:
                assert max_rel(g, o) <= TOL, (nx, ny, steps)


def test_default_plan_and_errors(eng, orc):
    import torch
    w = synth.make_vdiff(1024, 300, seed=9600)
    g, info = gpu_run(eng, w, 50)
    assert info["vec"] == 4 and info["bx"] == 128 and info["T"] == 4
    assert max_rel(g, orc.run_vdiff2d(w.u0, w.coef, 50)) <= TOL
    st = eng
    for bad in (dict(ndim=3, nz=4), dict(storage=st.ST_BF16), dict(strict=True),
                dict(force_vec=8), dict(force_bx=256)):
        kw = dict(ndim=2, nz=1)
        kw.update(bad)
        with pytest.raises(st.StencilError) as e:
            st.Plan(st.ST_DIFFUSION_VAR, kw.pop("ndim"), 64, 32, kw.pop("nz"), **kw)
        assert e.value.code == st.ST_ERR_UNSUPPORTED, bad
    plan = st.Plan(st.ST_DIFFUSION_VAR, 2, 64, 32)
    u = torch.zeros((32, 64), device="cuda")
    out = torch.zeros_like(u)
    k = torch.zeros((5, 32, 64), device="cuda")
    with pytest.raises(st.StencilError):      # the planes are required
        plan.run(u, out, None, 3)
    with pytest.raises(st.StencilError):      # planes overlapping the output
        plan.run(u, k[1], None, 3, power=k)
    plan.close()
