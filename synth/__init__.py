"""Seeded synthetic inputs for the stencil workloads.

This module is shared by the CPU oracle's tests, the GPU parity tests and the benchmark.
It holds none of the stencil arithmetic: only a counter-based random stream, affine maps of
that stream onto value ranges, and the construction of coefficient sets.

Random stream: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  Draw k of stream `seed` is mix(seed + (k + 1) * 0x9E3779B97F4A7C15),
so any slice of the stream can be produced without producing what comes before it.  A draw
becomes a float in [0, 1) as (u >> 40) * 2**-24, which is exact in float32 and float64.

Draw order within one workload: the field (row-major, x fastest), then the power map (thermal
stencils only), then the coefficients.

Coefficient layouts (the order the engine and the oracle both take them in):
  diffusion 2D: [cc, cw, ce, cs, cn]
  diffusion 3D: [cc, cw, ce, cs, cn, cb, ca]
  thermal 2D:   [k_dt, Rx, Ry, Rz, amb]         (the paper's sdc, Rx_1, Ry_1, Rz_1, TEMP_AMB)
  thermal 3D:   [cc, cw, ce, cs, cn, cb, ca, sdc, amb]
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

DIFFUSION = 0
THERMAL = 1
AMBIENT = 80.0


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+n-1 of the SplitMix64 stream `seed`, as uint64."""
    out = np.empty(n, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for a in range(0, n, _CHUNK):
            b = min(n, a + _CHUNK)
            k = np.arange(offset + a + 1, offset + b + 1, dtype=np.uint64)
            z = s + k * GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            out[a:b] = z ^ (z >> np.uint64(31))
    return out


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws as float64 in [0, 1): (u >> 40) * 2**-24."""
    u = splitmix64(seed, n, offset)
    return (u >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


def uniform_f32(seed: int, n: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    """float32(lo + (hi - lo) * u), the affine map evaluated in float64 and rounded once."""
    out = np.empty(n, dtype=np.float32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        u = uniform01(seed, b - a, offset + a)
        out[a:b] = (lo + (hi - lo) * u).astype(np.float32)
    return out


@dataclass
class Workload:
    """One stencil problem: kind, shape (nz, ny, nx), step count and its seeded inputs."""
    name: str
    kind: int
    ndim: int
    nx: int
    ny: int
    nz: int
    steps: int
    seed: int
    u0: np.ndarray = field(repr=False)
    power: np.ndarray | None = field(repr=False)
    coef: np.ndarray = field(repr=False)
    rad: int = 1    # stencil radius: 1 = the Table 2 stencils, > 1 = star diffusion
    var: bool = False   # diffusion with per-cell coefficients: coef has shape (5, ny, nx)

    @property
    def shape(self):
        return (self.ny, self.nx) if self.ndim == 2 else (self.nz, self.ny, self.nx)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def diffusion_coefficients(seed: int, ndim: int, offset: int) -> np.ndarray:
    """Positive coefficients normalised to sum 1: u_k ~ U[0.05, 1) in layout order,
    divided by their float64 sum and rounded to float32."""
    m = 5 if ndim == 2 else 7
    u = 0.05 + 0.95 * uniform01(seed, m, offset)
    return (u / u.sum()).astype(np.float32)


def star_coefficients(seed: int, ndim: int, R: int, offset: int) -> np.ndarray:
    """Radius-R star diffusion: 1 + 4R (2D) or 1 + 6R (3D) positive coefficients normalised to
    sum 1, in the layout [cc, per distance d = 1..R: cw, ce, cs, cn (, cb, ca)]; u_k ~ U[0.05, 1)
    with the distance-d draws divided by d (weights fall off outwards), normalised in float64,
    rounded to float32."""
    per = 4 if ndim == 2 else 6
    m = 1 + per * R
    u = 0.05 + 0.95 * uniform01(seed, m, offset)
    for d in range(1, R + 1):
        u[1 + per * (d - 1):1 + per * d] /= d
    return (u / u.sum()).astype(np.float32)


def make_star(ndim: int, R: int, nx: int, ny: int, nz: int = 1, steps: int = 1, seed: int = 1,
              name: str = "") -> Workload:
    """Radius-R star diffusion problem: field ~ U[0, 1) then the coefficients, from stream
    `seed` (kind DIFFUSION, no power map)."""
    if ndim == 2:
        nz = 1
    n = nx * ny * nz
    shape = (ny, nx) if ndim == 2 else (nz, ny, nx)
    u0 = uniform_f32(seed, n, 0.0, 1.0, 0).reshape(shape)
    coef = star_coefficients(seed, ndim, R, n)
    return Workload(name or f"star{R}_{ndim}d", DIFFUSION, ndim, nx, ny, nz, steps, seed, u0,
                    None, coef, R)


def vdiff_coefficients(seed: int, nx: int, ny: int, offset: int) -> np.ndarray:
    """Per-cell diffusion coefficients, shape (5, ny, nx), planes [cc, cw, ce, cs, cn]: for
    every cell five draws u_k ~ U[0.05, 1) (cell-major, in layout order), divided by their
    float64 sum and rounded to float32, so each cell's weights are positive and sum to 1."""
    out = np.empty((5, ny, nx), dtype=np.float32)
    rows = max(1, _CHUNK // (5 * nx))
    for y0 in range(0, ny, rows):
        y1 = min(ny, y0 + rows)
        m = (y1 - y0) * nx
        u = 0.05 + 0.95 * uniform01(seed, 5 * m, offset + 5 * y0 * nx).reshape(y1 - y0, nx, 5)
        out[:, y0:y1, :] = np.moveaxis(u / u.sum(axis=2, keepdims=True), 2, 0).astype(np.float32)
    return out


def make_vdiff(nx: int, ny: int, steps: int = 1, seed: int = 1, name: str = "") -> Workload:
    """Diffusion 2D with per-cell coefficients: field ~ U[0, 1), then the coefficient planes,
    from stream `seed`.  The planes travel in `coef`; `var` marks the workload."""
    n = nx * ny
    u0 = uniform_f32(seed, n, 0.0, 1.0, 0).reshape(ny, nx)
    coef = vdiff_coefficients(seed, nx, ny, n)
    return Workload(name or "vardiff2d", DIFFUSION, 2, nx, ny, 1, steps, seed, u0, None, coef,
                    1, True)


def thermal_scalars(seed: int, offset: int):
    """k_dt ~ U[0.5,1), Rx, Ry ~ U[0.05,0.2), Rz ~ U[1e-4,1e-3), redrawn until the explicit
    stability bound k_dt * (2 Rx + 2 Ry + Rz) <= 1 holds (it always holds for these ranges)."""
    while True:
        u = uniform01(seed, 4, offset)
        k_dt = 0.5 + 0.5 * u[0]
        rx = 0.05 + 0.15 * u[1]
        ry = 0.05 + 0.15 * u[2]
        rz = 1e-4 + 9e-4 * u[3]
        if k_dt * (2 * rx + 2 * ry + rz) <= 1.0:
            return k_dt, rx, ry, rz
        offset += 4


def thermal_coefficients(seed: int, ndim: int, offset: int) -> np.ndarray:
    k_dt, rx, ry, rz = thermal_scalars(seed, offset)
    if ndim == 2:
        return np.array([k_dt, rx, ry, rz, AMBIENT], dtype=np.float32)
    # 3D: neighbour weights k_dt*R per axis; centre weight makes a field equal to the ambient
    # temperature with zero power a fixed point: cc + 2ce + 2cn + 2ca + ca = 1.
    ce = k_dt * rx
    cn = k_dt * ry
    ca = k_dt * rz
    cc = 1.0 - (2 * ce + 2 * cn + 3 * ca)
    assert cc >= 0.0
    return np.array([cc, ce, ce, cn, cn, ca, ca, k_dt, AMBIENT], dtype=np.float32)


def make(kind: int, ndim: int, nx: int, ny: int, nz: int = 1, steps: int = 1, seed: int = 1,
         name: str = "") -> Workload:
    """Field, power and coefficients for one problem, drawn in that order from stream `seed`.

    Diffusion: field ~ U[0, 1).  Thermal: temperature ~ U[320, 340) K, power ~ U[0, 0.5),
    ambient 80."""
    if ndim == 2:
        nz = 1
    n = nx * ny * nz
    shape = (ny, nx) if ndim == 2 else (nz, ny, nx)
    if kind == DIFFUSION:
        u0 = uniform_f32(seed, n, 0.0, 1.0, 0).reshape(shape)
        power = None
        coef = diffusion_coefficients(seed, ndim, n)
    else:
        u0 = uniform_f32(seed, n, 320.0, 340.0, 0).reshape(shape)
        power = uniform_f32(seed, n, 0.0, 0.5, n).reshape(shape)
        coef = thermal_coefficients(seed, ndim, 2 * n)
    return Workload(name or f"{'diffusion' if kind == DIFFUSION else 'thermal'}{ndim}d",
                    kind, ndim, nx, ny, nz, steps, seed, u0, power, coef)


# --- the five configurations the engine is measured and checked on -----------------------

def c1_diffusion2d(nx=1024, ny=1024, steps=100):
    """2D 5-point diffusion, 1024^2, 100 steps, seed 1."""
    return make(DIFFUSION, 2, nx, ny, 1, steps, seed=1, name="diffusion2d_1024x1024_100")


def c2_thermal2d(nx=16384, ny=16384, steps=1000):
    """2D thermal, 16384^2, 1000 steps, seed 2."""
    return make(THERMAL, 2, nx, ny, 1, steps, seed=2, name=f"thermal2d_{nx}x{ny}_{steps}")


def c3a_diffusion3d(n=512, steps=1000):
    """3D 7-point diffusion, 512^3, 1000 steps, seed 3."""
    return make(DIFFUSION, 3, n, n, n, steps, seed=3, name=f"diffusion3d_{n}^3_{steps}")


def c3b_thermal3d(nx=512, ny=512, nz=256, steps=1000):
    """3D thermal, 512x512x256, 1000 steps, seed 4."""
    return make(THERMAL, 3, nx, ny, nz, steps, seed=4, name=f"thermal3d_{nx}x{ny}x{nz}_{steps}")


def c5b_adjoint2d(n=2048, steps=200):
    """Adjoint case: 2D diffusion, 2048^2, 200 steps (checkpoints every 20), seed 6; the loss
    weights come from loss_weights(6, shape)."""
    return make(DIFFUSION, 2, n, n, 1, steps, seed=6, name=f"adjoint2d_{n}x{n}_{steps}")


def c5a_batch_specs(count=64, seed=5):
    """Shapes of the batched workload: per grid (kind, nx, ny, steps, seed).

    nx and ny are independently log-uniform in [256, 4096] (rounded), steps uniform in
    {50..500}, kind alternates diffusion/thermal by index; grid g draws its data from stream
    seed * 1000 + g."""
    u = uniform01(seed, 3 * count, 0)
    lo, hi = math.log(256.0), math.log(4096.0)
    specs = []
    for g in range(count):
        nx = int(round(math.exp(lo + (hi - lo) * u[3 * g])))
        ny = int(round(math.exp(lo + (hi - lo) * u[3 * g + 1])))
        steps = 50 + int(u[3 * g + 2] * 451)
        specs.append((DIFFUSION if g % 2 == 0 else THERMAL, nx, ny, steps, seed * 1000 + g))
    return specs


def c5a_batch(count=64, seed=5):
    return [make(k, 2, nx, ny, 1, st, seed=s, name=f"batch{g}")
            for g, (k, nx, ny, st, s) in enumerate(c5a_batch_specs(count, seed))]


def loss_weights(seed: int, shape) -> np.ndarray:
    """Weights w ~ U[-1, 1) of the scalar loss L = sum_i w_i u_N,i used by the adjoint."""
    n = int(np.prod(shape))
    return uniform_f32(seed ^ 0x5EED, n, -1.0, 1.0, 0).reshape(shape)
