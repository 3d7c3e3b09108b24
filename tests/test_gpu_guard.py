"""Guard bands around the caller's buffers: every grid, power map and output the library is given
sits inside a larger allocation whose padding holds a NaN with a marked payload; after the run
the padding must be bit-for-bit unchanged (no write outside the buffers) and the result must
match the oracle (a read of the padding would have put a NaN into it).  Covers the streaming 2D
kernels (contracted two-row and in place, exact), resident tiles, 16-bit storage, the 3D
kernels, the allocation-free entry point and the batch queue, each on ragged sizes, out of place
and in place."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

G = 4096                    # guard floats before and after each buffer (16 KiB: aligned)
CANARY = np.uint32(0x7FA5A5A5)   # a quiet NaN with a payload no float arithmetic produces
TOL = 1e-5


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_00438_gb300 as st
    return st


class Guarded:
    """A float32 CUDA buffer of `a`'s shape with guard bands of G floats on both sides."""

    def __init__(self, a):
        import torch
        a = np.ascontiguousarray(a, dtype=np.float32)
        self.n = a.size
        self.shape = a.shape
        host = np.full(self.n + 2 * G, CANARY, dtype=np.uint32).view(np.float32)
        host[G:G + self.n] = a.ravel()
        self.buf = torch.from_numpy(host).cuda()
        self.t = self.buf[G:G + self.n].view(*self.shape)

    def intact(self):
        h = self.buf.cpu().numpy().view(np.uint32)
        return bool(np.all(h[:G] == CANARY) and np.all(h[G + self.n:] == CANARY))

    def array(self):
        return self.t.cpu().numpy()


def max_rel(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    floor = 1e-6 * max(np.max(np.abs(o)), 1e-300)
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), floor)))


def check(o, ref, exact, tol=TOL):
    if exact:
        assert np.array_equal(o, ref), max_rel(o, ref)
    else:
        assert max_rel(o, ref) <= tol, max_rel(o, ref)


# (label, plan keywords, exact): the 2D plan families
PLANS_2D = [
    ("streaming two-row", dict(resident=-1, force_T=8, force_vec=4, partial_rows=2), False),
    ("streaming in place", dict(resident=-1, force_T=8, force_vec=8, partial_rows=1), False),
    ("exact", dict(resident=-1, exact=1, force_T=4), True),
    ("resident", dict(resident=1, force_T=8), False),
    ("resident exact", dict(resident=1, exact=1, force_T=4), True),
]


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("label,kw,exact", PLANS_2D)
def test_2d_plans(eng, orc, kind, label, kw, exact):
    for t, (nx, ny, steps) in enumerate([(301, 77, 19), (517, 263, 9), (33, 1000, 17)]):
        w = synth.make(kind, 2, nx, ny, seed=8100 + 10 * t + kind)
        ref = orc.run(kind, w.u0, w.coef, steps, w.power)
        u = Guarded(w.u0)
        p = None if w.power is None else Guarded(w.power)
        out = Guarded(np.zeros_like(w.u0))
        kw2 = dict(kw)
        exact_flag = kw2.pop("exact", 0)
        plan = eng.Plan(kind, 2, nx, ny, exact=bool(exact_flag), **kw2)
        plan.run(u.t, out.t, w.coef, steps, power=None if p is None else p.t)
        plan.sync()
        # in place, on the same guarded buffer
        v = Guarded(w.u0)
        plan.run(v.t, v.t, w.coef, steps, power=None if p is None else p.t)
        plan.sync()
        plan.close()
        for b in (u, out, v) + ((p,) if p is not None else ()):
            assert b.intact(), (label, nx, ny, "guard band written")
        check(out.array(), ref, exact)
        check(v.array(), ref, exact)


@pytest.mark.parametrize("stor", [1, 2])
def test_16bit(eng, orc, stor):
    for t, (nx, ny, steps) in enumerate([(301, 77, 19), (700, 300, 17)]):
        w = synth.make(1, 2, nx, ny, seed=8200 + t)
        u, p, out = Guarded(w.u0), Guarded(w.power), Guarded(np.zeros_like(w.u0))
        plan = eng.Plan(1, 2, nx, ny, storage=stor)
        plan.run(u.t, out.t, w.coef, steps, power=p.t)
        plan.sync()
        plan.close()
        for b in (u, p, out):
            assert b.intact(), (stor, nx, ny)
        o = out.array()
        assert np.all(np.isfinite(o))


@pytest.mark.parametrize("kind", [0, 1])
def test_3d(eng, orc, kind):
    for t, (nx, ny, nz, steps, kw) in enumerate([(70, 60, 20, 9, dict(force_T=3)),
                                               (131, 67, 33, 7, dict(force_T=4)),
                                               (70, 60, 20, 5, dict(exact=1, force_T=2))]):
        w = synth.make(kind, 3, nx, ny, nz, seed=8300 + 10 * t + kind)
        ref = orc.run(kind, w.u0, w.coef, steps, w.power)
        u = Guarded(w.u0)
        p = None if w.power is None else Guarded(w.power)
        out = Guarded(np.zeros_like(w.u0))
        kw2 = dict(kw)
        exact = bool(kw2.pop("exact", 0))
        plan = eng.Plan(kind, 3, nx, ny, nz, exact=exact, **kw2)
        plan.run(u.t, out.t, w.coef, steps, power=None if p is None else p.t)
        plan.sync()
        plan.close()
        for b in (u, out) + ((p,) if p is not None else ()):
            assert b.intact(), (nx, ny, nz, "guard band written")
        check(out.array(), ref, exact)


@pytest.mark.parametrize("kind", [0, 1])
def test_noalloc(eng, orc, kind):
    w = synth.make(kind, 2, 301, 77, seed=8400 + kind)
    ref = orc.run(kind, w.u0, w.coef, 19, w.power)
    u = Guarded(w.u0)
    p = None if w.power is None else Guarded(w.power)
    out = Guarded(np.zeros_like(w.u0))
    eng.stencil_run_noalloc(kind, u.t, out.t, None if p is None else p.t, w.coef, 301, 77, 19,
                            exact=True)
    import torch
    torch.cuda.synchronize()
    for b in (u, out) + ((p,) if p is not None else ()):
        assert b.intact()
    check(out.array(), ref, True)


def test_batch(eng, orc):
    import torch
    ws = [synth.make(k, 2, nx, ny, steps=s, seed=8500 + i)
          for i, (k, nx, ny, s) in enumerate([(0, 301, 77, 19), (1, 260, 333, 23), (0, 97, 401, 9)])]
    bufs = []
    items = []
    for w in ws:
        u = Guarded(w.u0)
        o = Guarded(np.zeros_like(w.u0))
        p = None if w.power is None else Guarded(w.power)
        bufs.append((u, o, p))
        items.append({"kind": w.kind, "nx": w.nx, "ny": w.ny, "steps": w.steps, "grid_in": u.t,
                      "grid_out": o.t, "power": None if p is None else p.t, "coeffs": w.coef})
    b = eng.Batch(items)
    b.run()
    b.sync()
    torch.cuda.synchronize()
    b.close()
    for w, (u, o, p) in zip(ws, bufs):
        for x in (u, o) + ((p,) if p is not None else ()):
            assert x.intact(), (w.nx, w.ny)
        check(o.array(), orc.run(w.kind, w.u0, w.coef, w.steps, w.power), False)
