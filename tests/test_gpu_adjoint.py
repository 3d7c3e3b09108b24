"""GPU adjoint sweep (gradients of a 2D run) against the float64 oracle gradient, which is itself
pinned to central finite differences and to the dense transpose in the oracle tests.

Tolerances follow from the arithmetic (eps = 2^-24, every float32 step rounds at most R = 6
times per cell, N steps).  The transposed operator A^T has non-negative entries, so rounding
errors stay below the adjoint of |w| entrywise: with lambda' the float64 adjoint of |w|,
    |d lambda_t| <= (N - t) R eps lambda'_t          (dL/du0 = lambda_0),
    |d dL/dp|    <= (N R + N + 2) eps dL/dp(|w|)      (float32 sum over steps, Hotspot).
The forward states satisfy |d u_t| <= N R eps U, U = 2 max|u0| (rows of A sum to at most 1; the
Hotspot source terms are far below the field).  A coefficient gradient
g_m = sum_{t,i} lambda_{t+1}[i] g_m(u_t)_i is summed in float32 by each thread over at most
64 terms (its 16 cells x 4 fused steps), the partial sums then combined by error-free
transformations, so
    |d g_m| <= N R eps Lam (G_m + D_m U) + 4 eps D_m U Lam + 68 eps S_m,
with Lam = sum_t ||lambda'_{t+1}||_1 (the oracle's cc gradient of |w| on a field of ones, or its
amb gradient over k_dt Rz), G_m a bound of |g_m| and D_m the sum of |d g_m / d u| over a cell's
neighbourhood, S_m = sum |terms| as returned by the engine.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -24
R = 6


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1802_00438_gb300 as st
    return st


def _bounds(kind, w, U):
    """(G_m, D_m) per coefficient: bounds of |g_m| and of sum |d g_m / d u|."""
    c = np.asarray(w.coef, np.float64)
    if kind == 0:
        return np.full(5, U), np.ones(5)
    kdt, rx, ry, rz, amb = c
    pmax = float(np.max(np.abs(w.power)))
    G = np.array([pmax + (4 * rx + 4 * ry + rz) * U + rz * abs(amb), kdt * 4 * U, kdt * 4 * U,
                  kdt * (U + abs(amb)), kdt * rz])
    D = np.array([4 * rx + 4 * ry + rz, 4 * kdt, 4 * kdt, kdt, 0.0])
    return G, D


def _abs_adjoint(orc, kind, w, wt, steps):
    """Oracle adjoint of |w|: (dL/du0, dL/dp) entrywise bounds and Lam = sum_t ||lambda'||_1."""
    aw = np.abs(wt).astype(np.float64)
    gu, gk, gp = orc.adjoint2d(kind, w.u0, w.coef, steps, aw, w.power, ckpt=20)
    if kind == 0:
        _, g1, _ = orc.adjoint2d(0, np.ones(w.shape), w.coef, steps, aw, None, ckpt=20)
        lam = g1[0]
    else:
        c = w.coef.astype(np.float64)
        lam = gk[4] / (c[0] * c[3])
    return gu, gp, lam


def _run(eng, w, wt, steps, ckpt):
    import torch
    u0 = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda()
    pw = None if w.power is None else torch.from_numpy(np.ascontiguousarray(w.power)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(wt)).cuda()
    adj = eng.Adjoint(w.kind, w.nx, w.ny, steps, ckpt)
    out = adj.forward(u0, w.coef, pw)
    gu, gk, gp, ga = adj.backward(g, pw, with_abs=True)
    torch.cuda.synchronize()
    adj.close()
    res = [out, gu, gk, gp, ga]
    return [None if t is None else t.cpu().numpy().astype(np.float64) for t in res]


def _check(orc, w, wt, steps, res):
    out, gu, gk, gp, ga = res
    kind = w.kind
    N = steps
    gu64, gk64, gp64 = orc.adjoint2d(kind, w.u0, w.coef, steps, wt, w.power, ckpt=20)
    gua, gpa, lam = _abs_adjoint(orc, kind, w, wt, steps)
    U = 2.0 * float(np.max(np.abs(w.u0)))
    # dL/du0 = lambda_0, entrywise
    assert np.all(np.abs(gu - gu64) <= N * R * EPS * gua + 1e-30)
    # the forward result is the plain run
    ref = orc.run(kind, w.u0, w.coef, steps, w.power, dtype=np.float64)
    assert np.max(np.abs(out - ref)) <= N * R * EPS * U + 1e-30
    # coefficients
    G, D = _bounds(kind, w, U)
    for m in range(5):
        assert ga[m] >= abs(gk64[m]) * (1 - 1e-4), (m, ga[m], gk64[m])
        tol = N * R * EPS * lam * (G[m] + D[m] * U) + 4 * EPS * D[m] * U * lam + 68 * EPS * ga[m]
        assert abs(gk[m] - gk64[m]) <= tol, (m, gk[m], gk64[m], tol)
    if kind == 1:
        assert np.all(np.abs(gp - gp64) <= (N * R + N + 2) * EPS * gpa + 1e-30)
    return gu64, gk64, gp64


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("nx,ny,steps,ckpt", [(300, 200, 45, 20), (1, 1, 5, 2), (129, 7, 9, 4),
                                              (257, 130, 20, 20), (67, 333, 3, 20)])
def test_adjoint_vs_oracle(eng, orc, kind, nx, ny, steps, ckpt):
    w = synth.make(kind, 2, nx, ny, steps=steps, seed=7000 + 13 * nx + ny + kind)
    wt = synth.loss_weights(7100 + nx, w.shape)
    res = _run(eng, w, wt, steps, ckpt)
    _check(orc, w, wt, steps, res)


@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_staged_and_plain_paths_agree_bitwise(eng, orc, kind):
    """Tiles away from the grid edge take a path without clamps or masks when their inputs come
    by tensor-map copies; an upstream gradient that starts off a 16-byte boundary forces plain
    loads everywhere.  Both evaluate the same operations in the same order: equal bits."""
    import torch
    nx, ny, steps = 612, 300, 13
    w = synth.make(kind, 2, nx, ny, steps=steps, seed=7200 + kind)
    wt = synth.loss_weights(7201, w.shape)
    u0 = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda()
    pw = None if w.power is None else torch.from_numpy(np.ascontiguousarray(w.power)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(wt)).cuda()
    raw = torch.empty(nx * ny + 1, dtype=torch.float32, device="cuda")
    g_off = raw[1:].view(ny, nx)        # 4 bytes past a 16-byte boundary
    g_off.copy_(g)
    res = []
    for grad in (g, g_off):
        adj = eng.Adjoint(w.kind, nx, ny, steps, 5)
        adj.forward(u0, w.coef, pw)
        gu, gk, gp, ga = adj.backward(grad, pw, with_abs=True)
        torch.cuda.synchronize()
        adj.close()
        res.append([t.cpu().numpy() for t in (gu, gk, ga) + ((gp,) if gp is not None else ())])
    for a, b in zip(*res):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_abs_sums_leave_gradients_unchanged(eng, orc, kind):
    """The transposed pass accumulates sum |term| only when the caller asks for it; the
    gradients are the same sums in the same order either way: equal bits."""
    import torch
    nx, ny, steps = 530, 270, 11
    w = synth.make(kind, 2, nx, ny, steps=steps, seed=7300 + kind)
    wt = synth.loss_weights(7301, w.shape)
    u0 = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda()
    pw = None if w.power is None else torch.from_numpy(np.ascontiguousarray(w.power)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(wt)).cuda()
    res = []
    for with_abs in (True, False):
        adj = eng.Adjoint(w.kind, nx, ny, steps, 4)
        adj.forward(u0, w.coef, pw)
        gu, gk, gp, ga = adj.backward(g, pw, with_abs=with_abs)
        torch.cuda.synchronize()
        adj.close()
        assert (ga is not None) == with_abs
        res.append([t.cpu().numpy() for t in (gu, gk) + ((gp,) if gp is not None else ())])
    for a, b in zip(*res):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_no_cancellation_is_tight(eng, orc, kind):
    """With w >= 0 every diffusion term is non-negative (lambda >= 0, u >= 0): the coefficient
    gradients must then match to the growth bound relative to their own size."""
    w = synth.make(kind, 2, 200, 150, steps=30, seed=7300 + kind)
    wt = np.abs(synth.loss_weights(7301, w.shape))
    res = _run(eng, w, wt, 30, 20)
    gu64, gk64, gp64 = _check(orc, w, wt, 30, res)
    gk = res[2]
    idx = range(5) if kind == 0 else (3, 4)   # Hotspot: (amb - c) < 0 and the constant term
    for m in idx:
        assert abs(gk[m] - gk64[m]) <= 2 * (30 * R + 72) * EPS * abs(gk64[m]), m


@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_directional_fd(eng, orc, kind):
    """u_N is affine in u0 (and in the power map), so a central difference along any
    direction equals the gradient's inner product up to float32 rounding of the runs."""
    import torch
    nx, ny, steps = 160, 96, 25
    w = synth.make(kind, 2, nx, ny, steps=steps, seed=7400 + kind)
    wt = synth.loss_weights(7401, w.shape).astype(np.float64)
    d = synth.loss_weights(7402, w.shape).astype(np.float32)
    _, gu, gk, gp, _ = _run(eng, w, wt.astype(np.float32), steps, 20)
    plan = eng.Plan(kind, 2, nx, ny)

    def L(u, p):
        ut = torch.from_numpy(np.ascontiguousarray(u, np.float32)).cuda()
        pt = None if p is None else torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()
        o = torch.empty_like(ut)
        plan.run(ut, o, w.coef, steps, power=pt)
        plan.sync()
        return float(np.sum(wt * o.cpu().numpy().astype(np.float64))), float(o.abs().max())

    # |d L| <= sum|w| N R eps max|u| per run; the gradient's own error <= N R eps sum lambda'|d|
    gua, gpa, _ = _abs_adjoint(orc, kind, w, wt, steps)
    h = 1.0 if kind == 0 else 100.0
    lp, mp = L(w.u0 + h * d, w.power)
    lm, mm = L(w.u0 - h * d, w.power)
    fd = (lp - lm) / (2 * h)
    noise = np.sum(np.abs(wt)) * steps * R * EPS * 2 * max(mp, mm) / h
    assert abs(fd - np.sum(gu * d)) <= noise + steps * R * EPS * np.sum(gua * np.abs(d))
    if kind == 1:
        lp, mp = L(w.u0, w.power + h * d)
        lm, mm = L(w.u0, w.power - h * d)
        fd = (lp - lm) / (2 * h)
        noise = np.sum(np.abs(wt)) * steps * R * EPS * 2 * max(mp, mm) / h
        assert abs(fd - np.sum(gp * d)) <= noise + (steps * R + steps + 2) * EPS * np.sum(gpa * np.abs(d))
    plan.close()


def test_adjoint_deterministic_and_autograd(eng, orc):
    """Two backward runs agree bit for bit; the torch.autograd path gives the same gradients."""
    import torch
    nx, ny, steps = 190, 70, 23
    w = synth.make(1, 2, nx, ny, steps=steps, seed=7500)
    wt = synth.loss_weights(7501, w.shape)
    r1 = _run(eng, w, wt, steps, 20)
    r2 = _run(eng, w, wt, steps, 20)
    for a, b in zip(r1, r2):
        assert np.array_equal(a, b)
    u0 = torch.from_numpy(np.ascontiguousarray(w.u0)).cuda().requires_grad_()
    pw = torch.from_numpy(np.ascontiguousarray(w.power)).cuda().requires_grad_()
    k = torch.tensor(w.coef, dtype=torch.float32, requires_grad=True)
    out = eng.stencil_sweep(u0, k, steps, kind=1, power=pw, ckpt=20)
    loss = (out * torch.from_numpy(wt).cuda()).sum()
    loss.backward()
    assert np.array_equal(out.detach().cpu().numpy(), r1[0].astype(np.float32))
    assert np.array_equal(u0.grad.cpu().numpy(), r1[1].astype(np.float32))
    assert np.array_equal(k.grad.numpy(), r1[2].astype(np.float32))
    assert np.array_equal(pw.grad.cpu().numpy(), r1[3].astype(np.float32))


def test_adjoint_errors(eng):
    import torch
    with pytest.raises(eng.StencilError):
        eng.Adjoint(0, 0, 5, 10)
    with pytest.raises(eng.StencilError):
        eng.Adjoint(0, 5, 5, 10, ckpt=0)
    adj = eng.Adjoint(0, 8, 8, 4)
    g = torch.zeros(8, 8, device="cuda")
    with pytest.raises(eng.StencilError):          # no forward run yet
        adj.backward(g)
    u = torch.rand(8, 8, device="cuda")
    with pytest.raises(eng.StencilError):          # diffusion takes no power map
        adj.forward(u, [0.2] * 5, power=u)
    adj.close()
    # zero steps: identity gradient
    adj = eng.Adjoint(1, 8, 8, 0)
    p = torch.rand(8, 8, device="cuda")
    out = adj.forward(u, [0.5, 0.1, 0.1, 0.001, 80.0], power=p)
    gu, gk, gp, _ = adj.backward(g + 1.0, p)
    assert torch.equal(out, u) and torch.equal(gu, g + 1.0)
    assert float(gk.abs().sum()) == 0.0 and float(gp.abs().sum()) == 0.0
    adj.close()


@pytest.mark.slow
@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_full_size(eng, orc, kind):
    """The configured case: 2048 x 2048, 200 steps, checkpoints every 20 steps."""
    w = synth.make(kind, 2, 2048, 2048, steps=200, seed=7600 + kind)
    wt = synth.loss_weights(7601, w.shape)
    res = _run(eng, w, wt, 200, 20)
    _check(orc, w, wt, 200, res)
