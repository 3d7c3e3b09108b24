"""Plain CPU oracle for the stencil engine — TEST INFRASTRUCTURE ONLY.

Only the test suite, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg import
this package.  The engine shares no code with it: the arithmetic lives in
`stencil_oracle.c` (plain Jacobi loops, Table 2 order, -ffp-contract=off), compiled here with
gcc and called through ctypes.

Arrays are numpy, C-contiguous, shaped (ny, nx) for 2D and (nz, ny, nx) for 3D, x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "stencil_oracle.c"), os.path.join(_HERE, "stencil_oracle_body.h")]
_LIB_PATH = os.path.join(_HERE, "liborc_stencil.so")
_lib = None
_lock = threading.Lock()

DIFFUSION = 0
THERMAL = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP).  Returns the .so path."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC[0]]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L = ctypes.c_long
            I = ctypes.c_int
            for name in ("orc_run_f32", "orc_run_f64"):
                fn = getattr(lib, name)
                fn.argtypes = [I, I, P, P, P, P, L, L, L, I]
                fn.restype = I
            for name in ("orc_run_star_f32", "orc_run_star_f64"):
                fn = getattr(lib, name)
                fn.argtypes = [I, I, P, P, P, L, L, L, I]
                fn.restype = I
            for name in ("orc_run_vdiff2d_f32", "orc_run_vdiff2d_f64"):
                fn = getattr(lib, name)
                fn.argtypes = [P, P, P, L, L, I]
                fn.restype = I
            lib.orc_adjoint2d_f64.argtypes = [I, P, P, P, L, L, I, I, P, P, P, P]
            lib.orc_adjoint2d_f64.restype = I
            lib.orc_set_threads.argtypes = [I]
            lib.orc_get_threads.restype = I
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def run(kind: int, u0: np.ndarray, coef, steps: int, power: np.ndarray | None = None,
        dtype=np.float32) -> np.ndarray:
    """`steps` Jacobi iterations of the Table 2 stencil `kind` (0 diffusion, 1 thermal) on u0,
    in float32 (parity) or float64 (error reference).  Dimensionality follows u0.ndim."""
    lib = _load()
    dtype = np.dtype(dtype)
    u = np.ascontiguousarray(u0, dtype=dtype)
    ndim = u.ndim
    if ndim == 2:
        ny, nx = u.shape
        nz = 1
    elif ndim == 3:
        nz, ny, nx = u.shape
    else:
        raise ValueError("u0 must be 2D or 3D")
    k = np.ascontiguousarray(coef, dtype=dtype)
    expect = {(0, 2): 5, (0, 3): 7, (1, 2): 5, (1, 3): 9}[(kind, ndim)]
    if k.size != expect:
        raise ValueError(f"expected {expect} coefficients, got {k.size}")
    p = None
    if kind == THERMAL:
        if power is None:
            raise ValueError("thermal stencils need a power map")
        p = np.ascontiguousarray(power, dtype=dtype)
        if p.shape != u.shape:
            raise ValueError("power map shape differs from the field's")
    out = np.empty_like(u)
    fn = lib.orc_run_f32 if dtype == np.float32 else lib.orc_run_f64
    rc = fn(kind, ndim, _ptr(u), _ptr(out), _ptr(p), _ptr(k), nx, ny, nz, int(steps))
    if rc != 0:
        raise RuntimeError(f"oracle failed ({rc})")
    return out


def run_star(R: int, u0: np.ndarray, coef, steps: int, dtype=np.float32) -> np.ndarray:
    """`steps` Jacobi iterations of the radius-R star diffusion (Eqs. 1-2 with rad = R): 2D for
    a (ny, nx) array, 3D for (nz, ny, nx); coef = [cc, per distance d = 1..R: cw, ce, cs, cn
    (, cb, ca in 3D)], evaluated from the centre outwards, every operation rounded."""
    lib = _load()
    dtype = np.dtype(dtype)
    u = np.ascontiguousarray(u0, dtype=dtype)
    if u.ndim == 2:
        (ny, nx), nz = u.shape, 1
    elif u.ndim == 3:
        nz, ny, nx = u.shape
    else:
        raise ValueError("2D or 3D arrays only")
    k = np.ascontiguousarray(coef, dtype=dtype)
    if k.size != 1 + (4 if u.ndim == 2 else 6) * R:
        raise ValueError("coefficient count does not match the radius")
    out = np.empty_like(u)
    fn = lib.orc_run_star_f32 if dtype == np.float32 else lib.orc_run_star_f64
    rc = fn(u.ndim, int(R), _ptr(u), _ptr(out), _ptr(k), nx, ny, nz, int(steps))
    if rc != 0:
        raise RuntimeError(f"oracle failed ({rc})")
    return out


def run_vdiff2d(u0: np.ndarray, coef: np.ndarray, steps: int, dtype=np.float32) -> np.ndarray:
    """`steps` Jacobi iterations of diffusion 2D with per-cell coefficients: coef has shape
    (5, ny, nx), the planes [cc, cw, ce, cs, cn]; each cell is updated in Table 2's order with
    its own coefficients, every operation rounded."""
    lib = _load()
    dtype = np.dtype(dtype)
    u = np.ascontiguousarray(u0, dtype=dtype)
    if u.ndim != 2:
        raise ValueError("u0 must be 2D")
    ny, nx = u.shape
    k = np.ascontiguousarray(coef, dtype=dtype)
    if k.shape != (5, ny, nx):
        raise ValueError("coef must have shape (5, ny, nx)")
    out = np.empty_like(u)
    fn = lib.orc_run_vdiff2d_f32 if dtype == np.float32 else lib.orc_run_vdiff2d_f64
    rc = fn(_ptr(u), _ptr(out), _ptr(k), nx, ny, int(steps))
    if rc != 0:
        raise RuntimeError(f"oracle failed ({rc})")
    return out


def adjoint2d(kind: int, u0: np.ndarray, coef, steps: int, weights: np.ndarray,
              power: np.ndarray | None = None, ckpt: int = 0):
    """Float64 reverse-mode gradient of L = sum(weights * u_steps) for a 2D run.

    Returns (dL/du0, dL/dcoef[5], dL/dpower or None)."""
    lib = _load()
    u = np.ascontiguousarray(u0, dtype=np.float64)
    ny, nx = u.shape
    k = np.ascontiguousarray(coef, dtype=np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    p = None if power is None else np.ascontiguousarray(power, dtype=np.float64)
    gu = np.empty_like(u)
    gk = np.zeros(5, dtype=np.float64)
    gp = np.empty_like(u) if kind == THERMAL else None
    rc = lib.orc_adjoint2d_f64(kind, _ptr(u), _ptr(p), _ptr(k), nx, ny, int(steps), int(ckpt),
                               _ptr(w), _ptr(gu), _ptr(gk), _ptr(gp))
    if rc != 0:
        raise RuntimeError(f"oracle adjoint failed ({rc})")
    return gu, gk, gp


def loss(kind: int, u0, coef, steps, weights, power=None) -> float:
    """L = sum(weights * u_steps) with the float64 forward oracle."""
    uN = run(kind, u0, coef, steps, power, dtype=np.float64)
    return float(np.sum(np.asarray(weights, dtype=np.float64) * uN))
