"""Trajectory runs (every intermediate state of a run, written by the temporally-blocked passes
themselves) against the oracle: state t must equal the oracle's t-step run within the
contracted bar (max relative error 1e-5), for every t, both Table 2 2D stencils, ragged sizes,
step counts that are and are not multiples of the 8 fused steps, and a padded state stride."""
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


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("nx,ny,steps,pad", [(1, 1, 3, 0), (13, 11, 8, 0), (257, 130, 19, 0),
                                             (700, 300, 17, 12), (203, 91, 9, 5)])
def test_trajectory_states(eng, orc, kind, nx, ny, steps, pad):
    import torch
    w = synth.make(kind, 2, nx, ny, seed=9950 + nx + kind)
    u = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda()
    p = None if w.power is None else torch.from_numpy(np.ascontiguousarray(w.power)).cuda()
    stride = nx * ny + pad
    buf = torch.full((steps * stride,), float("nan"), device="cuda")
    plan = eng.Plan(kind, 2, nx, ny)
    eng.stencil_run_trajectory(plan.h, u, buf, stride, p, w.coef, steps)
    plan.sync()
    plan.close()
    got = buf.cpu().numpy()
    ref = w.u0
    for t in range(steps):
        ref = orc.run(kind, ref, w.coef, 1, w.power)
        g = got[t * stride:t * stride + nx * ny].reshape(ny, nx)
        assert max_rel(g, ref) <= TOL, (t, max_rel(g, ref))
        if pad:
            assert np.all(np.isnan(got[t * stride + nx * ny:(t + 1) * stride]))   # gaps untouched


def test_trajectory_errors(eng):
    import torch
    st = eng
    u = torch.zeros((32, 64), device="cuda")
    buf = torch.zeros((4, 32, 64), device="cuda")
    k = [0.5, 0.1, 0.1, 0.15, 0.15]
    exact = st.Plan(0, 2, 64, 32, exact=True)
    with pytest.raises(st.StencilError) as e:
        st.stencil_run_trajectory(exact.h, u, buf, 64 * 32, None, k, 4)
    assert e.value.code == st.ST_ERR_UNSUPPORTED
    exact.close()
    plan = st.Plan(0, 2, 64, 32)
    for args, code in (((u, buf, 64 * 32 - 1, None, k, 4), st.ST_ERR_INVALID_ARG),   # stride too small
                       ((buf[1], buf, 64 * 32, None, k, 4), st.ST_ERR_INVALID_ARG),   # input overlaps
                       ((u, buf, 64 * 32, None, k, 0), st.ST_ERR_INVALID_ARG),        # no steps
                       ((u, buf, 64 * 32, u, k, 4), st.ST_ERR_INVALID_ARG)):          # power for diffusion
        with pytest.raises(st.StencilError) as e:
            st.stencil_run_trajectory(plan.h, *args)
        assert e.value.code == code, args[2:]
    plan.close()
