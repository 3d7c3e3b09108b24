"""Grids of more than 2^31 cells: every index of the plan path that could overflow 32 bits is
exercised (cell offsets, row pitches, plane offsets, work ranges).  The oracle cannot run the
whole grid in a test's time, so sampled cells are checked against the oracle run on a window
around each sample: after S steps a cell depends only on cells within distance S (Sec. 3.2's
halo argument, Eq. 2), so a window reaching 2S beyond the sample in every direction (or the
grid's own edge, where the clamp of Sec. 5.1 applies as in the full grid) gives the sample's
exact oracle value even though the window's artificial edges clamp differently.
"""
import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 48 * 2**30:
        pytest.skip("needs 48 GiB of free device memory")
    import paper_1802_00438_gb300 as st
    return st


def _samples(shape, rng_seed, n=24):
    """Corners, edge midpoints, the last cells in memory order and seeded interior points."""
    dims = shape
    pts = set()
    for corner in np.ndindex(*([2] * len(dims))):
        pts.add(tuple((d - 1) if c else 0 for c, d in zip(corner, dims)))
    pts.add(tuple(d - 1 for d in dims[:-1]) + (dims[-1] // 2,))
    pts.add(tuple(d // 2 for d in dims))
    u = synth.uniform01(rng_seed, n * len(dims))
    for i in range(n):
        pts.add(tuple(int(u[i * len(dims) + a] * dims[a]) for a in range(len(dims))))
    return sorted(pts)


def _big(kind, ndim, shape, seed):
    """A seeded workload tiled from a block of co-prime odd sides (so that no index error by a
    power of two, such as a 32-bit wrap, lands on an equal value): generating 2^31 draws one by
    one would take minutes."""
    blk = (4099, 4093) if ndim == 2 else (67, 131, 257)
    base = synth.make(kind, ndim, blk[-1], blk[-2], blk[0] if ndim == 3 else 1, seed=seed)

    def tile(a):
        reps = tuple(-(-n // b) for n, b in zip(shape, a.shape))
        return np.ascontiguousarray(np.tile(a, reps)[tuple(slice(0, n) for n in shape)])

    u0 = tile(base.u0)
    pw = None if base.power is None else tile(base.power)
    nz, ny, nx = (1,) + shape if ndim == 2 else shape
    return synth.Workload(f"big{ndim}d", kind, ndim, nx, ny, nz, 1, seed, u0, pw, base.coef)


def _window(shape, p, reach):
    return tuple(slice(max(0, c - reach), min(d, c + reach + 1)) for c, d in zip(p, shape))


def _check(orc, w, g, steps):
    shape = w.u0.shape
    for p in _samples(shape, 77 + w.kind):
        win = _window(shape, p, 2 * steps)
        sub = np.ascontiguousarray(w.u0[win])
        pw = None if w.power is None else np.ascontiguousarray(w.power[win])
        o = orc.run(w.kind, sub, w.coef, steps, pw)
        local = tuple(c - s.start for c, s in zip(p, win))
        ov, gv = float(o[local]), float(g[p])
        assert abs(gv - ov) <= TOL * max(abs(ov), 1e-6), (p, gv, ov)


def _run(st, w, steps):
    import torch
    u = torch.from_numpy(w.u0).cuda()
    p = None if w.power is None else torch.from_numpy(w.power).cuda()
    out = torch.empty_like(u)
    plan = st.Plan(w.kind, w.ndim, w.nx, w.ny, w.nz)
    T = plan.info()["T"]
    plan.run(u, out, w.coef, steps or T + 3, power=p)
    plan.sync()
    plan.close()
    g = out.cpu().numpy()
    del u, out, p
    torch.cuda.empty_cache()
    return g, T


@pytest.mark.parametrize("kind", [0, 1])
def test_2d_more_than_2_31_cells(eng, orc, kind):
    nx, ny = 65536 + 12, 33000          # 2.163e9 cells, ragged last tile column
    assert nx * ny > 2**31
    w = _big(kind, 2, (ny, nx), 8100 + kind)
    g, T = _run(eng, w, 0)
    _check(orc, w, g, T + 3)


def test_3d_more_than_2_31_cells(eng, orc):
    nx, ny, nz = 2048 + 4, 1100, 1000   # 2.257e9 cells
    assert nx * ny * nz > 2**31
    w = _big(0, 3, (nz, ny, nx), 8200)
    g, T = _run(eng, w, 0)
    _check(orc, w, g, T + 3)
