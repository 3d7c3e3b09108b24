"""Allocation-failure injection (the host hook stencil_debug_fail_alloc; no GPU fault): for every
allocation a plan, a batch or an adjoint makes at creation, make exactly that one fail and check
that creation reports ST_ERR_OOM, that the library holds no more allocations than before
(stencil_debug_live_allocs), and that the same object then creates and runs correctly."""
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


def sweep(eng, make):
    """Fail allocation 1, 2, ... of make() until one creation needs fewer; returns how many
    allocations creation makes."""
    live = eng.lib.stencil_debug_live_allocs()
    n = 1
    while True:
        assert eng.lib.stencil_debug_fail_alloc(n) == eng.ST_OK
        try:
            obj = make()
        except eng.StencilError as e:
            assert e.code == eng.ST_ERR_OOM, (n, e.code)
            assert eng.lib.stencil_debug_live_allocs() == live, ("leak after failure", n)
            n += 1
            assert n < 64
            continue
        finally:
            eng.lib.stencil_debug_fail_alloc(0)
        obj.close()
        assert eng.lib.stencil_debug_live_allocs() == live, ("leak after destroy", n)
        return n - 1


def test_plans(eng, orc):
    import torch
    cases = [(1, 2, (700, 300, 1), dict(resident=-1)),              # streaming, source map
             (0, 2, (301, 77, 1), dict(resident=1, force_T=8)),     # resident tiles
             (1, 2, (700, 300, 1), dict(storage=1)),                # 16-bit storage
             (0, 3, (70, 60, 20), dict(force_T=3)),                 # 3D
             (1, 2, (300, 200, 1), dict(exact=1, resident=-1))]     # exact
    for kind, ndim, (nx, ny, nz), kw in cases:
        n = sweep(eng, lambda: eng.Plan(kind, ndim, nx, ny, nz, **kw))
        assert n >= 1, (kind, ndim, kw)
        # the context is healthy: the same plan runs and matches the oracle
        w = synth.make(kind, ndim, nx, ny, nz, seed=8600 + kind)
        u = torch.from_numpy(w.u0).cuda()
        p = None if w.power is None else torch.from_numpy(w.power).cuda()
        out = torch.empty_like(u)
        plan = eng.Plan(kind, ndim, nx, ny, nz, **kw)
        plan.run(u, out, w.coef, 9, power=p)
        plan.sync()
        plan.close()
        ref = orc.run(kind, w.u0, w.coef, 9, w.power)
        o = out.cpu().numpy().astype(np.float64)
        tol = 2e-2 if kw.get("storage") else 1e-5
        err = np.max(np.abs(o - ref) / np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max()))
        assert err <= tol, (kind, ndim, kw, err)


def test_batch_and_adjoint(eng):
    import torch
    ws = [synth.make(k, 2, nx, ny, steps=s, seed=8700 + i)
          for i, (k, nx, ny, s) in enumerate([(0, 301, 77, 19), (1, 260, 333, 23)])]
    items = []
    for w in ws:
        u = torch.from_numpy(w.u0).cuda()
        items.append({"kind": w.kind, "nx": w.nx, "ny": w.ny, "steps": w.steps, "grid_in": u,
                      "grid_out": torch.empty_like(u),
                      "power": None if w.power is None else torch.from_numpy(w.power).cuda(),
                      "coeffs": w.coef})
    assert sweep(eng, lambda: eng.Batch(items)) >= 4
    assert sweep(eng, lambda: eng.Adjoint(0, 256, 192, 40, ckpt=10)) >= 6
