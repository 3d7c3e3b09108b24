"""Batched runs (many 2D grids of uneven sizes and step counts, one persistent kernel launch fed
by a tile work queue, captured in a graph) against the oracle, grid by grid; graph replay; grids
run in place; a dependency wait that runs out (a pass held back by the test hook, no fault)
reported as ST_ERR_TIMEOUT with the batch and the context still usable."""
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


SPECS = [(0, 300, 200, 37), (1, 257, 129, 100), (0, 1, 50, 9), (1, 64, 1, 12), (0, 700, 500, 8),
         (1, 1000, 37, 23), (0, 130, 67, 0), (1, 509, 263, 57), (0, 2048, 31, 4), (1, 33, 900, 17),
         (0, 97, 61, 1), (1, 400, 400, 80)]


def _make(st, inplace_every=3):
    import torch
    ws, items = [], []
    for i, (kind, nx, ny, steps) in enumerate(SPECS):
        w = synth.make(kind, 2, nx, ny, steps=steps, seed=7000 + i)
        u = torch.from_numpy(w.u0).cuda()
        out = u if (i % inplace_every == 2) else torch.full_like(u, float("nan"))
        p = None if w.power is None else torch.from_numpy(w.power).cuda()
        ws.append(w)
        items.append({"kind": kind, "nx": nx, "ny": ny, "steps": steps, "grid_in": u,
                      "grid_out": out, "power": p, "coeffs": w.coef})
    return ws, items


def test_batch_matches_oracle(eng, orc):
    import torch
    ws, items = _make(eng)
    b = eng.Batch(items)
    b.run()
    b.sync()
    torch.cuda.synchronize()
    for i, (w, it) in enumerate(zip(ws, items)):
        o = orc.run(w.kind, w.u0, w.coef, w.steps, w.power)
        g = it["grid_out"].cpu().numpy()
        assert max_rel(g, o) <= TOL, (i, w.nx, w.ny, w.steps, b.grid_info(i), max_rel(g, o))
    assert b.launches() == 1                 # one persistent launch per replay
    # replay: grids not in place give the same result again; in-place ones advance further
    b.run()
    b.sync()
    for i, (w, it) in enumerate(zip(ws, items)):
        inplace = it["grid_out"].data_ptr() == it["grid_in"].data_ptr()
        steps = 2 * w.steps if inplace else w.steps
        o = orc.run(w.kind, w.u0, w.coef, steps, w.power)
        assert max_rel(it["grid_out"].cpu().numpy(), o) <= TOL, (i, inplace)
    b.close()


def test_batch_choices_and_errors(eng):
    import torch
    ws, items = _make(eng)
    b = eng.Batch(items)
    for i, (kind, nx, ny, steps) in enumerate(SPECS):
        info = b.grid_info(i)
        assert info["T"] in (4, 8) and info["vec"] in (4, 8)
        assert info["passes"] == (-(-steps // info["T"]) if steps else 0)
    b.close()
    bad = dict(items[1])
    bad["power"] = None                      # Hotspot without a power map
    with pytest.raises(eng.StencilError):
        eng.Batch([bad])


def test_batch_bounded_wait_runs_out(eng, orc):
    """The items of pass 0 are held back (they never report finished), so every pass-1 item
    waits until the limit (20 ms) runs out: the launch leaves and sync reports ST_ERR_TIMEOUT.
    Then the hook is removed and the same batch replays correctly (nothing was left waiting, the
    context is intact)."""
    import torch
    ws, items = _make(eng, inplace_every=2)   # i % 2 == 2 never holds: no grid in place
    b = eng.Batch(items)
    b.set_wait(20_000_000, hold_pass=0)
    b.run()
    with pytest.raises(eng.StencilError) as e:
        b.sync()
    assert e.value.code == eng.ST_ERR_TIMEOUT
    torch.cuda.synchronize()                 # the stream is idle: no block kept waiting
    b.set_wait(1_000_000_000, hold_pass=-1)
    b.run()
    b.sync()
    for i, (w, it) in enumerate(zip(ws, items)):
        o = orc.run(w.kind, w.u0, w.coef, w.steps, w.power)
        assert max_rel(it["grid_out"].cpu().numpy(), o) <= TOL, i
    b.close()
    with pytest.raises(eng.StencilError) as e:
        b2 = eng.Batch(items)
        b2.set_wait(0)                        # a limit must be positive
    assert e.value.code == eng.ST_ERR_INVALID_ARG
