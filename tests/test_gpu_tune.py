"""The measured parameter choice (Sec. 5.3 / 5.4.2: the model narrows the configurations, the
few it rates best are run and the fastest kept) on the GPU: the tuner times what it says it
timed, a later plan of the same problem takes the cached configuration, and that plan still
meets the parity bars (exact plans bit-identical to the oracle, contracted within 1e-5)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture()
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_00438_gb300 as st
    st.stencil_tune_cache_clear()
    yield st
    st.stencil_tune_cache_clear()   # other tests rely on the model's own choice


def max_rel(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    floor = 1e-6 * max(np.max(np.abs(o)), 1e-300)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), floor)))


def _tensors(w):
    import torch
    u = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda()
    p = None if w.power is None else torch.from_numpy(np.ascontiguousarray(w.power)).cuda()
    return u, p, torch.empty_like(u)


def _tune_then_run(st, orc, w, tune_steps, run_steps, top_k, exact=False, rad=0):
    u, p, out = _tensors(w)
    r = st.stencil_tune(w.kind, w.ndim, w.nx, w.ny, w.nz, u, out, w.coef, tune_steps, p,
                        top_k=top_k, exact=exact, rad=rad)
    assert r["candidates"] >= 1 and r["gcells"] > 0
    assert r["timed"] == (min(top_k, r["candidates"]) if top_k else r["candidates"])
    assert st.stencil_tune_cache_size() == 1
    plan = st.Plan(w.kind, w.ndim, w.nx, w.ny, w.nz, exact=exact, rad=rad)
    info = plan.info()
    assert info["tuned"]
    assert info["T"] == r["force_T"]
    out.fill_(float("nan"))
    plan.run(u, out, w.coef, run_steps, power=p)
    plan.sync()
    plan.close()
    g = out.cpu().numpy()
    o = orc.run_star(w.rad, w.u0, w.coef, run_steps) if rad > 1 else \
        orc.run(w.kind, w.u0, w.coef, run_steps, w.power)
    return r, info, g, o


@pytest.mark.parametrize("kind", [0, 1])
def test_contracted_2d(eng, orc, kind):
    w = synth.make(kind, 2, 1030, 771, seed=9100 + kind)
    r, info, g, o = _tune_then_run(eng, orc, w, 24, 37, top_k=3)
    assert info["vec"] == r["force_vec"]
    assert r["timed"] == 3 and r["model_gcells"] > 0
    assert max_rel(g, o) <= TOL


def test_exact_2d_bitwise(eng, orc):
    w = synth.make(1, 2, 613, 300, seed=9110)
    r, info, g, o = _tune_then_run(eng, orc, w, 16, 21, top_k=0, exact=True)
    # the winner is a streaming tile width or resident tiles (whose width follows from vec)
    assert info["resident"] == (1 if r["resident"] == 1 else 0)
    if not info["resident"]:
        assert info["bx"] == r["force_bx"]
    assert np.array_equal(g, o)


@pytest.mark.parametrize("kind", [0, 1])
def test_contracted_3d(eng, orc, kind):
    w = synth.make(kind, 3, 132, 70, 21, seed=9120 + kind)
    r, info, g, o = _tune_then_run(eng, orc, w, 12, 11, top_k=0)
    assert (info["bx"], info["by"], info["vec"]) == (r["force_bx"], r["force_by"], r["force_vec"])
    assert max_rel(g, o) <= TOL


def test_star(eng, orc):
    w = synth.make_star(2, 2, 300, 260, steps=9, seed=9130)
    r, info, g, o = _tune_then_run(eng, orc, w, 8, 9, top_k=0, rad=2)
    assert max_rel(g, o) <= TOL


def test_cache_is_per_problem_and_clearable(eng, orc):
    w = synth.make(0, 2, 517, 260, seed=9140)
    u, p, out = _tensors(w)
    eng.stencil_tune(0, 2, w.nx, w.ny, 1, u, out, w.coef, 8, None, top_k=2)
    other = eng.Plan(0, 2, w.nx + 1, w.ny)          # another size: the model's own choice
    assert not other.info()["tuned"]
    other.close()
    exact = eng.Plan(0, 2, w.nx, w.ny, exact=True)  # another key (exact)
    assert not exact.info()["tuned"]
    exact.close()
    forced = eng.Plan(0, 2, w.nx, w.ny, force_T=2)  # forced parameters bypass the cache
    assert not forced.info()["tuned"] and forced.info()["T"] == 2
    forced.close()
    eng.stencil_tune_cache_clear()
    again = eng.Plan(0, 2, w.nx, w.ny)
    assert not again.info()["tuned"]
    again.close()


def test_saved_cache_reloads(eng, orc, tmp_path):
    w = synth.make(1, 2, 700, 300, seed=9150)
    u, p, out = _tensors(w)
    r = eng.stencil_tune(1, 2, w.nx, w.ny, 1, u, out, w.coef, 16, p, top_k=2)
    f = tmp_path / "tune.txt"
    eng.stencil_tune_cache_save(str(f))
    eng.stencil_tune_cache_clear()
    eng.stencil_tune_cache_load(str(f))
    plan = eng.Plan(1, 2, w.nx, w.ny)
    info = plan.info()
    plan.close()
    assert info["tuned"] and info["T"] == r["force_T"] and info["vec"] == r["force_vec"]
