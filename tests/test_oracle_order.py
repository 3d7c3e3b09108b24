"""Float32 evaluation-order probes for every update the oracle defines (arXiv 1802.00438,
Table 2, read left to right as printed, one rounding per operation; the star and per-cell
stencils extend that order as their oracle docstrings state).

Bit-exact parity of the exact GPU plans is defined against this order, so the order itself is
pinned here, term by term, independently of the oracle's code.  The probe for the adjacent
terms (i, i+1) of a sum puts 1 in the first term, 2**-24 (half an ulp of 1) in term i, 2**-23
(one ulp) in term i+1 and 0 everywhere else.  Left to right, 1 + 2**-24 rounds back to 1 (a
tie, to even) and adding 2**-23 then gives 1 + 2**-23.  With i and i+1 swapped, 1 + 2**-23 is
odd, so adding 2**-24 rounds up to 1 + 2**-22; any order that adds the two small terms together
first gives 1 + 3*2**-24, which also rounds to 1 + 2**-22.  A probe for every adjacent pair
therefore fixes the whole order (swapping the first two terms of a sum changes nothing: float
addition is commutative).  Every product in a probe is exact (one factor is 1 or 0).

The float64 oracle is not probed: 2**-24 is far above its half-ulp.
"""
import numpy as np
import pytest

H = np.float32(2.0 ** -24)
H2 = np.float32(2.0 ** -23)
IN_ORDER = np.float32(1.0) + H2               # 1 + 2**-23
SWAPPED = np.float32(1.0) + np.float32(2.0 ** -22)


def _probe_values(n_terms, i):
    """Term values for the probe of pair (i, i+1): [1, 0, .., 2**-24, 2**-23, .., 0]."""
    v = [np.float32(0.0)] * n_terms
    v[0] = np.float32(1.0)
    v[i] = H
    v[i + 1] = H2
    return v


def _check(got, label):
    assert got == IN_ORDER, (label, float(got) - 1.0)
    assert got != SWAPPED


def test_probe_arithmetic_itself():
    # the two orders really differ in float32 (round to nearest, ties to even)
    a = (np.float32(1.0) + H) + H2
    b = (np.float32(1.0) + H2) + H
    c = np.float32(1.0) + (H + H2)
    assert a == IN_ORDER and b == SWAPPED and c == SWAPPED


# --- Diffusion 2D: cc*c + cw*w + ce*e + cs*s + cn*n (Table 2 row 1) ----------------------

def _d2_cells():
    # centre (x=1, y=1) of a 3x3 grid; (y, x) index of each term's cell
    return [(1, 1), (1, 0), (1, 2), (2, 1), (0, 1)]     # c, w, e, s, n


@pytest.mark.parametrize("i", [1, 2, 3])
def test_order_diffusion2d(orc, i):
    vals = _probe_values(5, i)
    u = np.zeros((3, 3), np.float32)
    for v, cell in zip(vals, _d2_cells()):
        u[cell] = v
    k = np.ones(5, np.float32)
    o = orc.run(0, u, k, 1)
    _check(o[1, 1], ("diffusion2d", i))


# --- Diffusion 3D: ... + cb*b + ca*a (Table 2 row 2) --------------------------------------

def _d3_cells():
    # centre (1,1,1) of a 3x3x3 grid; (z, y, x) of c, w, e, s, n, b, a
    return [(1, 1, 1), (1, 1, 0), (1, 1, 2), (1, 2, 1), (1, 0, 1), (0, 1, 1), (2, 1, 1)]


@pytest.mark.parametrize("i", [1, 2, 3, 4, 5])
def test_order_diffusion3d(orc, i):
    vals = _probe_values(7, i)
    u = np.zeros((3, 3, 3), np.float32)
    for v, cell in zip(vals, _d3_cells()):
        u[cell] = v
    o = orc.run(0, u, np.ones(7, np.float32), 1)
    _check(o[1, 1, 1], ("diffusion3d", i))


# --- Hotspot 3D: c*cc + n*cn + s*cs + e*ce + w*cw + a*ca + b*cb + sdc*p + ca*amb (row 4) ----

@pytest.mark.parametrize("i", [1, 2, 3, 4, 5, 6, 7])
def test_order_thermal3d(orc, i):
    vals = _probe_values(9, i)
    # term -> cell: c, n, s, e, w, a, b (the seven field terms), then sdc*p (power at the
    # centre) and ca*amb (the ambient coefficient); all coefficients 1
    cells = [(1, 1, 1), (1, 0, 1), (1, 2, 1), (1, 1, 2), (1, 1, 0), (2, 1, 1), (0, 1, 1)]
    u = np.zeros((3, 3, 3), np.float32)
    for v, cell in zip(vals[:7], cells):
        u[cell] = v
    p = np.zeros_like(u)
    p[1, 1, 1] = vals[7]
    k = np.ones(9, np.float32)          # cc, cw, ce, cs, cn, cb, ca, sdc = 1
    k[8] = vals[8]                       # amb: ca*amb = amb
    o = orc.run(1, u, k, 1, p)
    _check(o[1, 1, 1], ("thermal3d", i))


# --- Hotspot 2D: c + sdc*(p + (n+s-2c)*Ry + (e+w-2c)*Rx + (amb-c)*Rz) (row 3) ------------

@pytest.mark.parametrize("i", [1, 2])
def test_order_thermal2d_bracket(orc, i):
    # with c = 0 and sdc = Rx = Ry = Rz = 1 the bracket is p + (n+s) + (e+w) + amb; probe its
    # three additions with n, e and amb carrying the terms (s = w = 0) and p = 1
    vals = _probe_values(4, i)          # p, (n+s)*Ry, (e+w)*Rx, (amb-c)*Rz
    u = np.zeros((3, 3), np.float32)
    u[0, 1] = vals[1]                   # n
    u[1, 2] = vals[2]                   # e
    p = np.zeros_like(u)
    p[1, 1] = vals[0]
    k = np.array([1.0, 1.0, 1.0, 1.0, vals[3]], np.float32)
    o = orc.run(1, u, k, 1, p)
    _check(o[1, 1], ("thermal2d", i))


def test_order_thermal2d_pairs_before_centre(orc):
    # (e + w) is rounded before 2c is subtracted, as (n + s) is: e = 2**24, w = 1, c = 1 gives
    # e + w = 2**24 (tie to even), so the bracket is 2**24 - 2; subtracting 2c first would give
    # 2**24 - 1 and then 2**24 after adding w
    u = np.zeros((1, 3), np.float32)
    u[0, 0] = 1.0                       # w of the centre
    u[0, 1] = 1.0                       # c
    u[0, 2] = 2.0 ** 24                 # e
    k = np.array([1.0, 1.0, 0.0, 0.0, 0.0], np.float32)   # sdc = 1, Rx = 1, Ry = Rz = 0
    o = orc.run(1, u, k, 1, np.zeros_like(u))
    assert o[0, 1] == np.float32(1.0 + 2.0 ** 24 - 2.0)
    assert o[0, 1] != np.float32(2.0 ** 24)


# --- radius-R star: cc*c, then per distance d = 1..R: w_d, e_d, s_d, n_d (b_d, a_d) -------

def _star_cells(ndim, R):
    c = R
    cells = [(c, c) if ndim == 2 else (c, c, c)]
    for d in range(1, R + 1):
        if ndim == 2:
            cells += [(c, c - d), (c, c + d), (c + d, c), (c - d, c)]
        else:
            cells += [(c, c, c - d), (c, c, c + d), (c, c + d, c), (c, c - d, c),
                      (c - d, c, c), (c + d, c, c)]
    return cells


@pytest.mark.parametrize("ndim,R", [(2, 2), (2, 3), (3, 2)])
def test_order_star(orc, ndim, R):
    cells = _star_cells(ndim, R)
    n = len(cells)
    side = 2 * R + 1
    for i in range(1, n - 1):
        vals = _probe_values(n, i)
        u = np.zeros((side,) * ndim, np.float32)
        for v, cell in zip(vals, cells):
            u[cell] = v
        o = orc.run_star(R, u, np.ones(n, np.float32), 1)
        _check(o[(R,) * ndim], ("star", ndim, R, i))


# --- per-cell coefficients: cc_i*c + cw_i*w + ce_i*e + cs_i*s + cn_i*n --------------------

@pytest.mark.parametrize("i", [1, 2, 3])
def test_order_vdiff2d(orc, i):
    vals = _probe_values(5, i)
    u = np.zeros((3, 3), np.float32)
    for v, cell in zip(vals, _d2_cells()):
        u[cell] = v
    k = np.ones((5, 3, 3), np.float32)
    o = orc.run_vdiff2d(u, k, 1)
    _check(o[1, 1], ("vdiff2d", i))
