"""Resident tiles (one cooperative launch per run, the grid held on chip, halos exchanged every T
steps) against the CPU oracle: exact plans bit-identical to the float32 oracle, contracted plans
within 1e-5 max relative error, on ragged sizes (single rows and columns, edges inside a lane
and on a lane boundary, last blocks narrower than the halo), step counts around T, in place with
one and with several exchanges; the 1024^2 diffusion configuration as the plan chooses it; and
the bounded wait: a block that withholds its cells makes its neighbours give up with
ST_ERR_TIMEOUT, after which the same plan runs correctly again."""
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


def run(st, w, steps, exact, T=0, vec=0, inplace=False, resident=1):
    import torch
    u = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda()
    p = None if w.power is None else torch.from_numpy(np.ascontiguousarray(w.power)).cuda()
    out = u if inplace else torch.full_like(u, float("nan"))
    plan = st.Plan(w.kind, 2, w.nx, w.ny, exact=exact, force_T=T, force_vec=vec, resident=resident)
    info = plan.info()
    plan.run(u, out, w.coef, steps, power=p)
    plan.sync()
    plan.close()
    return out.cpu().numpy(), info


# (nx, ny): one cell, single rows and columns, widths whose east edge falls inside a lane and on
# its last cell for 2 and 4 cells per lane, several blocks each way with narrow last blocks
SIZES = [(1, 1), (1, 40), (57, 1), (33, 21), (64, 9), (301, 77), (250, 250), (517, 263)]


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("vec", [2, 4])
def test_exact_bitwise(eng, orc, kind, vec):
    for t, (nx, ny) in enumerate(SIZES):
        w = synth.make(kind, 2, nx, ny, seed=7200 + 31 * t + kind)
        for T, steps in ((4, 1), (4, 3), (4, 4), (4, 5), (4, 11), (3, 10), (8, 19)):
            g, info = run(eng, w, steps, True, T=T, vec=vec)
            assert info["resident"] == 1 and info["T"] == T and info["vec"] == vec
            o = orc.run(kind, w.u0, w.coef, steps, w.power)
            assert np.array_equal(g, o), (nx, ny, T, steps, max_rel(g, o))


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("vec", [2, 4])
def test_contracted(eng, orc, kind, vec):
    for t, (nx, ny) in enumerate(SIZES + [(1030, 771)]):
        w = synth.make(kind, 2, nx, ny, seed=7300 + 31 * t + kind)
        for T, steps in ((2, 7), (6, 6), (8, 27), (16, 40)):
            try:
                g, info = run(eng, w, steps, False, T=T, vec=vec)
            except eng.StencilError as e:   # too many blocks for one co-resident grid
                assert e.code == eng.ST_ERR_UNSUPPORTED and (nx, ny) == (1030, 771)
                continue
            assert info["resident"] == 1
            o = orc.run(kind, w.u0, w.coef, steps, w.power)
            assert max_rel(g, o) <= TOL, (nx, ny, T, steps, max_rel(g, o))


@pytest.mark.parametrize("kind", [0, 1])
def test_in_place(eng, orc, kind):
    # one epoch (the run reads a copy) and several
    w = synth.make(kind, 2, 301, 277, seed=7400 + kind)
    for exact in (True, False):
        for steps in (3, 8, 21):
            g, _ = run(eng, w, steps, exact, T=8, inplace=True)
            o = orc.run(kind, w.u0, w.coef, steps, w.power)
            if exact:
                assert np.array_equal(g, o), (steps, max_rel(g, o))
            else:
                assert max_rel(g, o) <= TOL, (steps, max_rel(g, o))


def test_small_config_chooses_resident(eng, orc):
    # the 1024^2 diffusion configuration, 100 steps, with nothing forced
    w = synth.c1_diffusion2d()
    g, info = run(eng, w, w.steps, False, resident=0)
    assert info["resident"] == 1 and info["ctas"] <= info["sms"] * 2
    o = orc.run(0, w.u0, w.coef, w.steps)
    assert max_rel(g, o) <= TOL, max_rel(g, o)
    # exact, bit-identical
    g, info = run(eng, w, w.steps, True, resident=0)
    assert info["resident"] == 1
    assert np.array_equal(g, o)


def test_refusals(eng):
    # grids beyond the co-resident blocks, named fields that do not combine, waits of plans
    # that stream
    with pytest.raises(eng.StencilError) as e:
        eng.Plan(0, 2, 8192, 8192, resident=1)
    assert e.value.code == eng.ST_ERR_UNSUPPORTED
    for kw in (dict(resident=1, partial_rows=1), dict(resident=1, storage=eng.ST_BF16),
               dict(resident=1, force_bx=256)):
        with pytest.raises(eng.StencilError) as e:
            eng.Plan(0, 2, 300, 200, **kw)
        assert e.value.code == eng.ST_ERR_UNSUPPORTED, kw
    for kw in (dict(resident=2), dict(partial_rows=3), dict(force_by=1)):
        with pytest.raises(eng.StencilError) as e:
            eng.Plan(0, 2, 300, 200, **kw)
        assert e.value.code == eng.ST_ERR_INVALID_ARG, kw
    p = eng.Plan(0, 2, 4096, 4096, resident=-1)
    assert p.info()["resident"] == 0
    with pytest.raises(eng.StencilError) as e:
        p.set_wait(10 ** 6)
    assert e.value.code == eng.ST_ERR_UNSUPPORTED
    p.close()
    q = eng.Plan(0, 2, 300, 200, resident=1)
    with pytest.raises(eng.StencilError) as e:
        q.set_wait(0)
    assert e.value.code == eng.ST_ERR_INVALID_ARG
    q.close()


def test_bounded_wait_runs_out(eng, orc):
    import torch
    w = synth.make(1, 2, 517, 263, seed=7500)
    u = torch.from_numpy(w.u0).cuda()
    p = torch.from_numpy(w.power).cuda()
    out = torch.empty_like(u)
    plan = eng.Plan(1, 2, w.nx, w.ny, force_T=4, resident=1)
    assert plan.info()["ctas"] > 1
    # block 0 publishes nothing from the first exchange on: its neighbours give up after 20 ms
    plan.set_wait(20 * 10 ** 6, hold_block=0, hold_epoch=0)
    plan.run(u, out, w.coef, 13, power=p)
    with pytest.raises(eng.StencilError) as e:
        plan.sync()
    assert e.value.code == eng.ST_ERR_TIMEOUT
    # the context and the plan stay usable
    plan.set_wait(10 ** 9)
    plan.run(u, out, w.coef, 13, power=p)
    plan.sync()
    plan.close()
    o = orc.run(1, w.u0, w.coef, 13, w.power)
    assert max_rel(out.cpu().numpy(), o) <= TOL
