"""Slab decomposition on the GPU: the grid cut into slabs held as separate device buffers, each
advanced by its own engine plan, halos exchanged by device copies before every pass (the
single-device stand-in for the multi-device split; the paper's future work, arXiv 1802.00438
Sec. 1 and 8).  Exact plans must reproduce the oracle's whole-grid run bit for bit, contracted
plans within the contracted bar."""
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


def _run(st, w, parts, T, steps, exact):
    import torch
    from paper_1802_00438_gb300 import slab as S
    n = w.u0.shape[0]
    sls = S.slabs(n, parts, T)
    grids, adv = [], []
    for s in sls:
        grids.append(torch.from_numpy(np.ascontiguousarray(w.u0[s.ext_lo:s.ext_hi])).cuda())
        p = None if w.power is None else \
            torch.from_numpy(np.ascontiguousarray(w.power[s.ext_lo:s.ext_hi])).cuda()
        adv.append(S.PlanAdvance(st, w.kind, w.ndim, s, w.nx, w.ny, coeffs=w.coef, power=p,
                                 exact=exact))
    S.run_local(sls, grids, steps, T, lambda r, g, ts: adv[r](g, ts))
    torch.cuda.synchronize()
    for a in adv:
        a.close()
    return np.concatenate([g[s.own()[0]:s.own()[1]].cpu().numpy() for s, g in zip(sls, grids)])


@pytest.mark.parametrize("kind,ndim,shape,parts,T,steps", [
    (0, 2, (700, 301), 2, 8, 35), (1, 2, (513, 390), 3, 8, 29), (1, 2, (300, 97), 2, 4, 13),
    (0, 3, (70, 66, 40), 2, 4, 11), (1, 3, (64, 50, 33), 3, 4, 9)])
def test_slabs_match_oracle(eng, orc, kind, ndim, shape, parts, T, steps):
    w = synth.make(kind, ndim, *shape, steps=steps, seed=4500 + kind + 10 * ndim)
    o = orc.run(kind, w.u0, w.coef, steps, w.power)
    g = _run(eng, w, parts, T, steps, exact=True)
    assert np.array_equal(g, o)
    g = _run(eng, w, parts, T, steps, exact=False)
    floor = 1e-6 * np.abs(o).max()
    err = np.max(np.abs(g.astype(np.float64) - o) / np.maximum(np.abs(o), floor))
    assert err <= 1e-5, err
