"""Pins of the CPU oracle to facts fixed outside it (arXiv 1802.00438, Table 2, Sec. 2.1,
Sec. 5.1) and to the mathematics of the iteration.

Each test is chosen so that a plausible mistake in the oracle (a dropped term, a wrong sign,
a swapped neighbour, a boundary that does not clamp, a different rounding order) fails it:
  - hand-worked single steps (golden fixture)            -> formulas, orientation, boundary
  - impulse response                                     -> each coefficient's direction
  - float32 rounding-order probe                         -> left-to-right evaluation
  - constant field / fixed point                         -> coefficients sum, ambient term
  - discrete maximum principle                           -> convexity of the update
  - dense iteration matrix built from index sets         -> everything, tiny grids, many steps
  - DCT-II eigenmodes (closed form)                      -> everything, large grids
  - conservation of the sum                              -> boundary handling at scale
  - adjoint: dot-product test and finite differences     -> the reverse sweep
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cell(arr, key):
    idx = tuple(int(v) for v in key.split(","))
    return arr[idx[::-1]]


# --- hand-worked steps ------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_hand_steps(orc, dtype):
    cases = json.load(open(os.path.join(GOLDEN, "hand_steps.json")))["cases"]
    for c in cases:
        shape = (c["ny"], c["nx"]) if c["ndim"] == 2 else (c["nz"], c["ny"], c["nx"])
        u0 = np.array(c["u0"], dtype=dtype).reshape(shape)
        p = None if c["power"] is None else np.array(c["power"], dtype=dtype).reshape(shape)
        out = orc.run(c["kind"], u0, c["coef"], 1, p, dtype=dtype)
        for key, val in c["expected"].items():
            assert _cell(out, key) == val, (c["name"], key, _cell(out, key), val)


# --- impulse response: pins the direction of every coefficient ----------------------------

def test_impulse_diffusion2d(orc):
    k = np.array([0.5, 0.0625, 0.125, 0.1875, 0.125], np.float32)   # distinct cw, ce, cs, cn
    u = np.zeros((7, 9), np.float32)
    x0, y0 = 4, 3
    u[y0, x0] = 1.0
    o = orc.run(0, u, k, 1)
    assert o[y0, x0] == k[0]
    assert o[y0, x0 + 1] == k[1]      # its west neighbour is the impulse -> cw
    assert o[y0, x0 - 1] == k[2]      # its east neighbour is the impulse -> ce
    assert o[y0 - 1, x0] == k[3]      # its south neighbour is the impulse -> cs
    assert o[y0 + 1, x0] == k[4]      # its north neighbour is the impulse -> cn
    assert np.count_nonzero(o) == 5
    # corner impulse: the clamped west and north neighbours are the cell itself
    u = np.zeros((5, 5), np.float32)
    u[0, 0] = 1.0
    o = orc.run(0, u, k, 1, dtype=np.float64)
    assert o[0, 0] == pytest.approx(k[0] + k[1] + k[4], abs=0)
    assert o[0, 1] == k[1] and o[1, 0] == k[4]
    # far corner: east and south clamp
    u = np.zeros((5, 5), np.float32)
    u[4, 4] = 1.0
    o = orc.run(0, u, k, 1, dtype=np.float64)
    assert o[4, 4] == np.float64(k[0]) + np.float64(k[2]) + np.float64(k[3])


def test_impulse_diffusion3d(orc):
    k = np.array([0.25, 0.0625, 0.125, 0.1875, 0.09375, 0.15625, 0.125], np.float32)
    u = np.zeros((5, 6, 7), np.float32)
    x0, y0, z0 = 3, 2, 2
    u[z0, y0, x0] = 1.0
    o = orc.run(0, u, k, 1)
    assert o[z0, y0, x0] == k[0]
    assert o[z0, y0, x0 + 1] == k[1]
    assert o[z0, y0, x0 - 1] == k[2]
    assert o[z0, y0 - 1, x0] == k[3]
    assert o[z0, y0 + 1, x0] == k[4]
    assert o[z0 + 1, y0, x0] == k[5]  # its below neighbour (z-1) is the impulse -> cb
    assert o[z0 - 1, y0, x0] == k[6]  # its above neighbour (z+1) is the impulse -> ca
    assert np.count_nonzero(o) == 7


def test_impulse_thermal2d(orc):
    kdt, rx, ry, rz = 0.75, 0.125, 0.1875, 0.0078125
    k = np.array([kdt, rx, ry, rz, 0.0], np.float32)
    u = np.zeros((7, 7), np.float32)
    u[3, 3] = 1.0
    p = np.zeros_like(u)
    o = orc.run(1, u, k, 1, p, dtype=np.float64)
    assert o[3, 3] == pytest.approx(1 - kdt * (2 * rx + 2 * ry + rz), rel=1e-15)
    assert o[3, 4] == pytest.approx(kdt * rx, rel=1e-15)
    assert o[3, 2] == pytest.approx(kdt * rx, rel=1e-15)
    assert o[2, 3] == pytest.approx(kdt * ry, rel=1e-15)
    assert o[4, 3] == pytest.approx(kdt * ry, rel=1e-15)
    assert np.count_nonzero(o) == 5
    # a unit power at one cell of a zero field adds sdc there and nowhere else
    o = orc.run(1, np.zeros_like(u), k, 1, (u > 0).astype(np.float32), dtype=np.float64)
    assert o[3, 3] == kdt and np.count_nonzero(o) == 1


def test_impulse_thermal3d(orc):
    k = np.array([0.5, 0.0625, 0.125, 0.1875, 0.09375, 0.03125, 0.0078125, 0.75, 0.0],
                 np.float32)
    u = np.zeros((5, 5, 5), np.float32)
    u[2, 2, 2] = 1.0
    o = orc.run(1, u, k, 1, np.zeros_like(u))
    assert o[2, 2, 2] == k[0]
    assert o[2, 2, 3] == k[1] and o[2, 2, 1] == k[2]
    assert o[2, 1, 2] == k[3] and o[2, 3, 2] == k[4]
    assert o[3, 2, 2] == k[5] and o[1, 2, 2] == k[6]
    o = orc.run(1, np.zeros_like(u), k, 1, u)
    assert o[2, 2, 2] == k[7] and np.count_nonzero(o) == 1
    # the ambient term ca * amb
    k2 = k.copy()
    k2[8] = 8.0
    o = orc.run(1, np.zeros_like(u), k2, 1, np.zeros_like(u))
    assert np.all(o == np.float32(k[6] * 8.0))


# --- float32 rounding order: Table 2 evaluated left to right, one rounding per op ----------

def test_float32_left_to_right_rounding(orc):
    # c=1, cc=1: r = 1.  cw*w = ce*e = 2**-24 (half an ulp of 1.0).  Left to right, each add
    # rounds 1 + 2**-24 back to 1 (ties to even); any order that adds the w and e terms
    # together first gives 1 + 2**-23.
    h = 2.0 ** -24
    k = np.array([1.0, h, h, 0.0, 0.0], np.float32)
    u = np.ones((1, 3), np.float32)
    o = orc.run(0, u, k, 1)
    assert o[0, 1] == np.float32(1.0)
    o64 = orc.run(0, u, k, 1, dtype=np.float64)
    assert o64[0, 1] == 1.0 + 2 * h
    # Hotspot 2D: (n + s) is rounded before 2c is subtracted.  n = 2**24, s = 1: in float32
    # n + s = 2**24 (tie to even), so t1 = -2c exactly.
    k = np.array([1.0, 0.0, 1.0, 0.0, 0.0], np.float32)          # sdc=1, Rx=0, Ry=1
    u = np.array([[2.0 ** 24], [1.0], [1.0]], np.float32)         # rows y=0,1,2; one column
    o = orc.run(1, u, k, 1, np.zeros_like(u))
    # cell y=1: c=1, n=2**24, s=1 -> t1 = 2**24 - 2 ; r = 1 + t1 (q = t1*Ry)
    assert o[1, 0] == np.float32(2.0 ** 24 - 2 + 1)
    # if s were added after subtracting 2c the result would be 2**24: check it is not
    assert o[1, 0] != np.float32(2.0 ** 24)


# --- invariants -------------------------------------------------------------------------

@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_constant_field_exact_with_dyadic_coefficients(orc, ndim, dtype):
    if ndim == 2:
        k = np.array([0.5, 0.125, 0.0625, 0.1875, 0.125], np.float32)
        shape = (13, 17)
    else:
        k = np.array([0.5, 0.0625, 0.0625, 0.125, 0.0625, 0.125, 0.0625], np.float32)
        shape = (5, 7, 9)
    assert float(np.sum(k.astype(np.float64))) == 1.0
    u = np.full(shape, 0.75, np.float32)
    o = orc.run(0, u, k, 37, dtype=dtype)
    assert np.all(o == 0.75)


def test_constant_field_general_coefficients(orc):
    w = synth.make(0, 2, 33, 21, steps=50, seed=11)
    u = np.full(w.shape, 0.3, np.float32)
    o = orc.run(0, u, w.coef, 50)
    ulp = np.spacing(np.float32(0.3))
    assert np.max(np.abs(o.astype(np.float64) - 0.3)) <= 2 * 50 * ulp


def test_thermal_ambient_fixed_point(orc):
    # Hotspot 2D: a field at the ambient temperature with zero power stays there exactly,
    # in any precision: every bracket of the update is an exact zero.
    w = synth.make(1, 2, 19, 23, steps=40, seed=12)
    amb = w.coef[4]
    u = np.full(w.shape, amb, np.float32)
    for dt in (np.float32, np.float64):
        o = orc.run(1, u, w.coef, 40, np.zeros_like(u), dtype=dt)
        assert np.all(o == amb)
    # Hotspot 3D with the constructed coefficients: fixed point up to rounding
    w3 = synth.make(1, 3, 9, 8, 7, steps=30, seed=13)
    u = np.full(w3.shape, w3.coef[8], np.float32)
    o = orc.run(1, u, w3.coef, 30, np.zeros_like(u), dtype=np.float64)
    cf = w3.coef.astype(np.float64)
    assert abs(cf[0] + 2 * cf[1] + 2 * cf[3] + 3 * cf[5] - 1.0) < 1e-6
    assert np.max(np.abs(o - 80.0)) < 80.0 * 30 * 1e-6


@pytest.mark.parametrize("ndim", [2, 3])
def test_max_principle_diffusion(orc, ndim):
    if ndim == 2:
        w = synth.make(0, 2, 40, 31, steps=60, seed=21)
    else:
        w = synth.make(0, 3, 12, 11, 10, steps=40, seed=22)
    lo, hi = float(w.u0.min()), float(w.u0.max())
    u = w.u0
    for s in range(4):
        u = orc.run(0, u, w.coef, 10, dtype=np.float64)
        assert u.min() >= lo - 1e-12 and u.max() <= hi + 1e-12


def test_max_principle_thermal(orc):
    w = synth.make(1, 2, 30, 20, steps=50, seed=23)
    o = orc.run(1, w.u0, w.coef, 50, w.power, dtype=np.float64)
    # with p >= 0 the temperature never falls below min(min u0, amb)
    assert o.min() >= min(float(w.u0.min()), float(w.coef[4])) - 1e-9


def test_thread_count_does_not_change_results(orc):
    w = synth.make(1, 2, 97, 61, steps=20, seed=24)
    n0 = orc.get_threads()
    try:
        orc.set_threads(1)
        a = orc.run(1, w.u0, w.coef, 20, w.power)
        orc.set_threads(max(2, n0))
        b = orc.run(1, w.u0, w.coef, 20, w.power)
    finally:
        orc.set_threads(n0)
    assert np.array_equal(a, b)


def test_zero_steps_copies(orc):
    w = synth.make(0, 3, 5, 4, 3, seed=25)
    assert np.array_equal(orc.run(0, w.u0, w.coef, 0), w.u0)


# --- brute force: dense iteration matrix from per-axis clamped index sets ------------------

def _axis_neighbours(n):
    """For each index i of an axis of length n: (i-1 clamped, i+1 clamped)."""
    return [(max(i - 1, 0), min(i + 1, n - 1)) for i in range(n)]


def _dense_affine(kind, ndim, nx, ny, nz, coef, power):
    """u -> A u + b for one step, written from the definition: cell i gets weight c_d on the
    cell reached by moving one step in direction d and clamping each axis into the grid."""
    coef = np.asarray(coef, np.float64)
    N = nx * ny * nz
    A = np.zeros((N, N))
    b = np.zeros(N)
    ax, ay, az = _axis_neighbours(nx), _axis_neighbours(ny), _axis_neighbours(nz)
    idx = lambda x, y, z: (z * ny + y) * nx + x
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        i = idx(x, y, z)
        W, E = idx(ax[x][0], y, z), idx(ax[x][1], y, z)
        Nn, S = idx(x, ay[y][0], z), idx(x, ay[y][1], z)
        B, Aa = idx(x, y, az[z][0]), idx(x, y, az[z][1])
        if kind == 0:
            wts = [(i, coef[0]), (W, coef[1]), (E, coef[2]), (S, coef[3]), (Nn, coef[4])]
            if ndim == 3:
                wts += [(B, coef[5]), (Aa, coef[6])]
        elif ndim == 2:
            kdt, rx, ry, rz, amb = coef
            wts = [(i, 1.0 - kdt * (2 * rx + 2 * ry + rz)), (W, kdt * rx), (E, kdt * rx),
                   (Nn, kdt * ry), (S, kdt * ry)]
            b[i] = kdt * (power.flat[i] + rz * amb)
        else:
            cc, cw, ce, cs, cn, cb, ca, sdc, amb = coef
            wts = [(i, cc), (W, cw), (E, ce), (S, cs), (Nn, cn), (B, cb), (Aa, ca)]
            b[i] = sdc * power.flat[i] + ca * amb
        for j, v in wts:
            A[i, j] += v
    return A, b


@pytest.mark.parametrize("kind,ndim", [(0, 2), (1, 2), (0, 3), (1, 3)])
def test_dense_matrix_brute_force(orc, kind, ndim):
    rng_sizes = ([(nx, ny, 1) for nx in range(1, 9) for ny in (1, 2, 5, 8)] if ndim == 2 else
                 [(nx, ny, nz) for nx, ny, nz in ((1, 1, 1), (2, 3, 4), (8, 1, 3), (5, 6, 2),
                                                  (4, 4, 4), (3, 8, 7), (1, 5, 8))])
    for t, (nx, ny, nz) in enumerate(rng_sizes):
        w = synth.make(kind, ndim, nx, ny, nz, seed=100 + t)
        steps = (t * 7) % 21
        A, b = _dense_affine(kind, ndim, nx, ny, nz, w.coef, w.power)
        u = w.u0.astype(np.float64).ravel()
        for _ in range(steps):
            u = A @ u + b
        o = orc.run(kind, w.u0, w.coef, steps, w.power, dtype=np.float64).ravel()
        assert np.allclose(o, u, rtol=1e-13, atol=0), (nx, ny, nz, steps)


# --- closed form: DCT-II eigenmodes of the clamped (edge-replicate) operator ---------------

def _phi(k, n):
    return np.cos(np.pi * k * (np.arange(n) + 0.5) / n)


def test_dct_eigenmode_diffusion2d(orc):
    nx = ny = 1024
    steps = 100
    cc, cwe, cns = 0.4, 0.1, 0.2                 # symmetric: cw = ce, cn = cs
    k = np.array([cc, cwe, cwe, cns, cns], np.float64)
    for (kx, ky) in [(1, 0), (3, 7), (200, 511)]:
        u0 = np.outer(_phi(ky, ny), _phi(kx, nx))
        lam = cc + 2 * cwe * math.cos(math.pi * kx / nx) + 2 * cns * math.cos(math.pi * ky / ny)
        o = orc.run(0, u0, k, steps, dtype=np.float64)
        assert np.max(np.abs(o - lam ** steps * u0)) <= 1e-12 * max(abs(lam) ** steps, 1e-300) + 1e-14


def test_dct_eigenmode_diffusion3d(orc):
    n = 48
    steps = 60
    k = np.array([0.4, 0.05, 0.05, 0.1, 0.1, 0.15, 0.15], np.float64)
    kx, ky, kz = 2, 5, 11
    u0 = np.einsum("k,j,i->kji", _phi(kz, n), _phi(ky, n), _phi(kx, n))
    lam = (k[0] + 2 * k[1] * math.cos(math.pi * kx / n) + 2 * k[3] * math.cos(math.pi * ky / n)
           + 2 * k[5] * math.cos(math.pi * kz / n))
    o = orc.run(0, u0, k, steps, dtype=np.float64)
    assert np.max(np.abs(o - lam ** steps * u0)) <= 1e-12


def test_dct_eigenmode_thermal2d(orc):
    nx, ny, steps = 256, 192, 150
    kdt, rx, ry, rz, amb = 0.8, 0.15, 0.1, 5e-4, 80.0
    p0 = 0.02
    tstar = amb + p0 / rz
    kx, ky = 5, 9
    phi = np.outer(_phi(ky, ny), _phi(kx, nx))
    u0 = tstar + 3.0 * phi
    lam = 1 - kdt * (2 * rx * (1 - math.cos(math.pi * kx / nx))
                     + 2 * ry * (1 - math.cos(math.pi * ky / ny)) + rz)
    o = orc.run(1, u0, [kdt, rx, ry, rz, amb], steps, np.full_like(u0, p0), dtype=np.float64)
    assert np.max(np.abs(o - (tstar + 3.0 * lam ** steps * phi))) <= 1e-11


def test_sum_conserved_symmetric_coefficients(orc):
    # with cw = ce, cn = cs and coefficients summing to 1 the grid sum is invariant
    w = synth.make(0, 2, 301, 257, seed=31)
    k = np.array([0.36, 0.12, 0.12, 0.2, 0.2])
    o = orc.run(0, w.u0, k, 200, dtype=np.float64)
    s0 = np.sum(w.u0.astype(np.float64))
    assert abs(o.sum() - s0) <= 1e-12 * s0
    # energy does not grow
    assert np.sum(o * o) <= np.sum(w.u0.astype(np.float64) ** 2)
    # asymmetric: the sum moves by (cw - ce) * (first column - last column) per step
    k2 = np.array([0.36, 0.16, 0.08, 0.2, 0.2])
    o1 = orc.run(0, w.u0, k2, 1, dtype=np.float64)
    u = w.u0.astype(np.float64)
    expect = u.sum() + (k2[1] - k2[2]) * (u[:, 0].sum() - u[:, -1].sum()) \
        + (k2[4] - k2[3]) * (u[0, :].sum() - u[-1, :].sum())
    assert abs(o1.sum() - expect) <= 1e-11 * abs(expect)


# --- adjoint -------------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_dot_product(orc, kind):
    # one step: <A x, y> = <x, A^T y>; the oracle's grad_u0 for L = <w, u_1> is A^T w
    for t, (nx, ny) in enumerate([(1, 1), (3, 2), (8, 5), (7, 8)]):
        w = synth.make(kind, 2, nx, ny, seed=200 + t)
        A, b = _dense_affine(kind, 2, nx, ny, 1, w.coef, w.power)
        y = synth.loss_weights(200 + t, w.shape).astype(np.float64)
        gu, _, _ = orc.adjoint2d(kind, w.u0, w.coef, 1, y, w.power)
        assert np.allclose(gu.ravel(), A.T @ y.ravel(), rtol=1e-13, atol=1e-15)
        # several steps: (A^T)^s w
        gu5, _, _ = orc.adjoint2d(kind, w.u0, w.coef, 5, y, w.power, ckpt=2)
        v = y.ravel()
        for _ in range(5):
            v = A.T @ v
        assert np.allclose(gu5.ravel(), v, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_finite_differences(orc, kind):
    nx, ny, steps = 23, 17, 30
    w = synth.make(kind, 2, nx, ny, steps=steps, seed=300 + kind)
    wt = synth.loss_weights(300 + kind, w.shape).astype(np.float64)
    u0 = w.u0.astype(np.float64)
    coef = w.coef.astype(np.float64)
    pw = None if w.power is None else w.power.astype(np.float64)
    gu, gk, gp = orc.adjoint2d(kind, u0, coef, steps, wt, pw, ckpt=7)

    def L(u, k, p):
        return orc.loss(kind, u, k, steps, wt, p)

    # coefficients (thermal: k_dt, Rx, Ry, Rz, amb)
    for j in range(5):
        h = 1e-6 * max(abs(coef[j]), 1e-3)
        kp, km = coef.copy(), coef.copy()
        kp[j] += h
        km[j] -= h
        fd = (L(u0, kp, pw) - L(u0, km, pw)) / (2 * h)
        assert fd == pytest.approx(gk[j], rel=1e-6, abs=1e-8), j
    # directional derivative along a random direction of u0 (and of p for thermal)
    d = synth.loss_weights(999, w.shape).astype(np.float64)
    h = 1e-4
    fd = (L(u0 + h * d, coef, pw) - L(u0 - h * d, coef, pw)) / (2 * h)
    assert fd == pytest.approx(np.sum(gu * d), rel=1e-7)
    if kind == 1:
        fd = (L(u0, coef, pw + h * d) - L(u0, coef, pw - h * d)) / (2 * h)
        assert fd == pytest.approx(np.sum(gp * d), rel=1e-7)


# --- star diffusion of radius R (Eqs. 1-2 with rad > 1) ------------------------------------

def _dense_star(ndim, R, nx, ny, nz, coef):
    """One step of the radius-R star as a matrix, from the definition: cell i gets weight
    c_{dir,d} on the cell d steps away in direction dir, each axis clamped into the grid."""
    coef = np.asarray(coef, np.float64)
    per = 4 if ndim == 2 else 6
    N = nx * ny * nz
    A = np.zeros((N, N))
    clamp = lambda v, n: min(max(v, 0), n - 1)
    idx = lambda x, y, z: (z * ny + y) * nx + x
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        i = idx(x, y, z)
        A[i, i] += coef[0]
        for d in range(1, R + 1):
            k = coef[1 + per * (d - 1):1 + per * d]
            A[i, idx(clamp(x - d, nx), y, z)] += k[0]
            A[i, idx(clamp(x + d, nx), y, z)] += k[1]
            A[i, idx(x, clamp(y + d, ny), z)] += k[2]
            A[i, idx(x, clamp(y - d, ny), z)] += k[3]
            if ndim == 3:
                A[i, idx(x, y, clamp(z - d, nz))] += k[4]
                A[i, idx(x, y, clamp(z + d, nz))] += k[5]
    return A


@pytest.mark.parametrize("ndim", [2, 3])
def test_star_radius1_is_table2(orc, ndim):
    for t, shape in enumerate([(1, 1, 1), (7, 5, 3), (40, 33, 9)]):
        nx, ny, nz = shape
        w = synth.make(0, ndim, nx, ny, nz, seed=600 + t)
        for dt in (np.float32, np.float64):
            a = orc.run(0, w.u0, w.coef, 9, dtype=dt)
            b = orc.run_star(1, w.u0, w.coef, 9, dtype=dt)
            assert np.array_equal(a, b), (shape, dt)


@pytest.mark.parametrize("ndim,R", [(2, 2), (2, 3), (3, 2)])
def test_star_impulse(orc, ndim, R):
    """Interior impulse: after one step each coefficient sits d cells away on the opposite
    side of its direction (the cell whose west-d neighbour is the impulse gets cw_d)."""
    per = 4 if ndim == 2 else 6
    w = synth.make_star(ndim, R, 19, 17, 15, seed=700 + R)
    k = w.coef.astype(np.float64)
    u = np.zeros(w.shape)
    c = (7, 8, 9) if ndim == 3 else (8, 9)
    u[c] = 1.0
    o = orc.run_star(R, u, k, 1, dtype=np.float64)
    expect = np.zeros_like(u)
    expect[c] = k[0]
    for d in range(1, R + 1):
        kd = k[1 + per * (d - 1):1 + per * d]
        def at(dz, dy, dx):
            return (c[0] + dz, c[1] + dy, c[2] + dx) if ndim == 3 else (c[0] + dy, c[1] + dx)
        expect[at(0, 0, d)] = kd[0]    # its west-d neighbour is the impulse
        expect[at(0, 0, -d)] = kd[1]   # east-d
        expect[at(0, -d, 0)] = kd[2]   # south-d (y + d)
        expect[at(0, d, 0)] = kd[3]    # north-d (y - d)
        if ndim == 3:
            expect[at(d, 0, 0)] = kd[4]    # below-d (z - d)
            expect[at(-d, 0, 0)] = kd[5]   # above-d (z + d)
    assert np.array_equal(o, expect)


def test_star_clamp_at_every_distance(orc):
    """Impulse on the x = 0 edge: cell j (1 <= j <= R) sees it as every west neighbour at a
    distance d >= j (clamped to x = 0), cell 0 as all R of them."""
    R = 3
    w = synth.make_star(2, R, 12, 9, seed=710)
    k = w.coef.astype(np.float64)
    u = np.zeros(w.shape)
    u[4, 0] = 1.0
    o = orc.run_star(R, u, k, 1, dtype=np.float64)
    cw = [k[1 + 4 * (d - 1)] for d in range(1, R + 1)]
    assert o[4, 0] == pytest.approx(k[0] + sum(cw), rel=1e-15)
    for j in range(1, R + 1):
        assert o[4, j] == pytest.approx(sum(cw[j - 1:]), rel=1e-15), j
    assert np.all(o[4, R + 1:] == 0)


@pytest.mark.parametrize("ndim,R", [(2, 2), (2, 3), (3, 2)])
def test_star_dense_matrix_brute_force(orc, ndim, R):
    sizes = ([(nx, ny, 1) for nx in (1, 2, 3, 5, 8) for ny in (1, 4, 7)] if ndim == 2 else
             [(1, 1, 1), (2, 3, 4), (5, 2, 3), (4, 4, 4), (3, 6, 5)])
    for t, (nx, ny, nz) in enumerate(sizes):
        w = synth.make_star(ndim, R, nx, ny, nz, seed=800 + t)
        steps = (t * 5) % 13
        A = _dense_star(ndim, R, nx, ny, nz, w.coef)
        v = w.u0.astype(np.float64).ravel()
        for _ in range(steps):
            v = A @ v
        o = orc.run_star(R, w.u0, w.coef, steps, dtype=np.float64).ravel()
        assert np.allclose(o, v, rtol=1e-13, atol=1e-15), (nx, ny, nz, steps)


def test_star_constant_field_and_max_principle(orc):
    # dyadic coefficients summing exactly to 1: a constant field is kept exactly
    k = np.array([0.5] + [0.0625] * 8, np.float64)     # 2D, R = 2: 1 + 8 coefficients
    u = np.full((13, 21), 0.375)
    for dt in (np.float32, np.float64):
        assert np.all(orc.run_star(2, u, k, 25, dtype=dt) == 0.375)
    # positive coefficients summing to 1: the range of the field never grows
    w = synth.make_star(2, 3, 64, 48, seed=820)
    o = orc.run_star(3, w.u0, w.coef, 40, dtype=np.float64)
    lo, hi = float(w.u0.min()), float(w.u0.max())
    assert o.min() >= lo - 1e-12 and o.max() <= hi + 1e-12


# --- diffusion 2D with per-cell coefficients (Table 2 row 1, coefficients as arrays) --------

def _dense_vdiff(nx, ny, k):
    """One step as a dense matrix from the definition: cell i gives its own weights cc_i, cw_i,
    ce_i, cs_i, cn_i to itself and to the cells one step west, east, south, north, each axis
    clamped into the grid."""
    k = np.asarray(k, np.float64)
    N = nx * ny
    A = np.zeros((N, N))
    ax, ay = _axis_neighbours(nx), _axis_neighbours(ny)
    for y, x in itertools.product(range(ny), range(nx)):
        i = y * nx + x
        for j, v in ((i, k[0, y, x]), (y * nx + ax[x][0], k[1, y, x]),
                     (y * nx + ax[x][1], k[2, y, x]), (ay[y][1] * nx + x, k[3, y, x]),
                     (ay[y][0] * nx + x, k[4, y, x])):
            A[i, j] += v
    return A


def test_vdiff_impulse_reads_each_cells_own_coefficients(orc):
    w = synth.make_vdiff(9, 7, seed=830)
    x0, y0 = 4, 3
    u = np.zeros((7, 9))
    u[y0, x0] = 1.0
    for dt in (np.float32, np.float64):
        o = orc.run_vdiff2d(u, w.coef, 1, dtype=dt)
        k = w.coef.astype(dt)
        expect = np.zeros((7, 9), dt)
        expect[y0, x0] = k[0, y0, x0]               # cc of the impulse cell
        expect[y0, x0 + 1] = k[1, y0, x0 + 1]       # its west neighbour is the impulse
        expect[y0, x0 - 1] = k[2, y0, x0 - 1]       # its east neighbour is the impulse
        expect[y0 - 1, x0] = k[3, y0 - 1, x0]       # its south neighbour is the impulse
        expect[y0 + 1, x0] = k[4, y0 + 1, x0]       # its north neighbour is the impulse
        assert np.array_equal(o, expect), dt


def test_vdiff_constant_planes_are_table2_diffusion(orc):
    w = synth.make(0, 2, 37, 23, seed=831)
    planes = np.broadcast_to(w.coef[:, None, None], (5, 23, 37)).copy()
    for dt in (np.float32, np.float64):
        assert np.array_equal(orc.run_vdiff2d(w.u0, planes, 17, dtype=dt),
                              orc.run(0, w.u0, w.coef, 17, dtype=dt))


def test_vdiff_dense_matrix_brute_force(orc):
    for t, (nx, ny) in enumerate([(1, 1), (1, 6), (5, 1), (2, 2), (3, 5), (8, 8), (7, 4)]):
        w = synth.make_vdiff(nx, ny, seed=840 + t)
        steps = (5 * t) % 19
        A = _dense_vdiff(nx, ny, w.coef)
        u = w.u0.astype(np.float64).ravel()
        for _ in range(steps):
            u = A @ u
        o = orc.run_vdiff2d(w.u0, w.coef, steps, dtype=np.float64).ravel()
        assert np.allclose(o, u, rtol=1e-13, atol=0), (nx, ny, steps)


def test_vdiff_constant_field_and_max_principle(orc):
    # dyadic per-cell weights summing exactly to 1 keep a dyadic constant field exactly
    ny, nx = 11, 13
    rng = synth.uniform01(850, 4 * nx * ny).reshape(4, ny, nx)
    q = np.floor(rng * 48) / 256.0                      # four weights in [0, 0.1875], dyadic
    k = np.concatenate([1.0 - q.sum(0, keepdims=True), q])
    u = np.full((ny, nx), 0.625)
    for dt in (np.float32, np.float64):
        assert np.all(orc.run_vdiff2d(u, k, 30, dtype=dt) == 0.625)
    # positive weights summing to 1 per cell: the field's range never grows
    # (the float32 weights sum to 1 within a few ulp, so the bound widens by that per step)
    w = synth.make_vdiff(64, 40, seed=851)
    o = orc.run_vdiff2d(w.u0, w.coef, 50, dtype=np.float64)
    sums = w.coef.astype(np.float64).sum(0)
    grow = float(sums.max()) ** 50
    shrink = float(sums.min()) ** 50
    lo, hi = float(w.u0.min()), float(w.u0.max())
    assert o.min() >= lo * min(shrink, 1.0) - 1e-12 and o.max() <= hi * max(grow, 1.0) + 1e-12
