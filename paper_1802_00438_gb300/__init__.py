"""Python binding of the GB300 stencil engine (libstencil.so, C ABI in include/stencil.h).

Argument marshalling only: every step of a sweep runs in the library's CUDA kernels.  There is
no fallback path: importing this package loads libstencil.so and raises if it is missing
(build it with `paper_1802_00438_gb300.build.build()` or `__graft_entry__.build()`).

Functions carry the C names.  Device buffers are torch CUDA tensors (float32, contiguous) or raw
integer device addresses; the stream defaults to torch's current stream.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstencil.so")

ST_OK = 0
ST_ERR_INVALID_ARG = -1
ST_ERR_DIMS_MISMATCH = -2
ST_ERR_UNSTABLE_COEFFS = -3
ST_ERR_CUDA = -4
ST_ERR_OOM = -5
ST_ERR_TIMEOUT = -6
ST_ERR_UNSUPPORTED = -7
ST_ERR_TOO_LARGE = -8

ST_DIFFUSION = 0
ST_THERMAL = 1
ST_DIFFUSION_VAR = 2   # per-cell coefficients: five planes passed as `power`, coeffs unused
ST_F32, ST_BF16, ST_F16, ST_F64 = 0, 1, 2, 3


class StencilError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class stencil_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ndim", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("storage", ctypes.c_int),
                ("force_T", ctypes.c_int), ("force_bx", ctypes.c_int), ("force_by", ctypes.c_int),
                ("force_vec", ctypes.c_int), ("exact", ctypes.c_int), ("strict", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("rad", ctypes.c_int), ("partial_rows", ctypes.c_int),
                ("resident", ctypes.c_int)]


class stencil_plan_info(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("bx", ctypes.c_int), ("by", ctypes.c_int),
                ("halo", ctypes.c_int), ("vec", ctypes.c_int), ("warps", ctypes.c_int),
                ("ctas", ctypes.c_int), ("sms", ctypes.c_int),
                ("scratch_bytes", ctypes.c_longlong), ("exact", ctypes.c_int),
                ("kernel_id", ctypes.c_int), ("model_gcells", ctypes.c_double),
                ("resident", ctypes.c_int), ("partial_rows", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class stencil_fpga_model_in(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("dim_x", ctypes.c_longlong), ("dim_y", ctypes.c_longlong),
                ("dim_z", ctypes.c_longlong), ("bsize_x", ctypes.c_int), ("bsize_y", ctypes.c_int),
                ("rad", ctypes.c_int), ("par_vec", ctypes.c_int), ("par_time", ctypes.c_int),
                ("size_cell", ctypes.c_int), ("num_read", ctypes.c_int), ("num_write", ctypes.c_int),
                ("iter", ctypes.c_longlong), ("fmax_hz", ctypes.c_double),
                ("th_max_gbs", ctypes.c_double)]


class stencil_fpga_model_out(ctypes.Structure):
    _fields_ = [("th_mem_gbs", ctypes.c_double), ("csize_x", ctypes.c_longlong),
                ("csize_y", ctypes.c_longlong), ("bnum_x", ctypes.c_longlong),
                ("bnum_y", ctypes.c_longlong), ("t_cell", ctypes.c_double),
                ("t_read", ctypes.c_double), ("t_write", ctypes.c_double),
                ("run_time_s", ctypes.c_double), ("throughput_gbs", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class stencil_gpu_model_in(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_longlong), ("ny", ctypes.c_longlong),
                ("nz", ctypes.c_longlong), ("steps", ctypes.c_int), ("T", ctypes.c_int),
                ("bx", ctypes.c_int), ("by", ctypes.c_int), ("halo_x", ctypes.c_int),
                ("halo_y", ctypes.c_int), ("sms", ctypes.c_int), ("sm_hz", ctypes.c_double),
                ("hbm_gbs", ctypes.c_double), ("bytes_per_cell", ctypes.c_double),
                ("ops_per_cell", ctypes.c_double), ("issue_eff", ctypes.c_double),
                ("hbm_eff", ctypes.c_double), ("stream_overhead", ctypes.c_double),
                ("launch_s", ctypes.c_double)]


class stencil_gpu_model_out(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_double), ("bytes_per_pass", ctypes.c_double),
                ("cells_computed_per_pass", ctypes.c_double), ("t_hbm_s", ctypes.c_double),
                ("t_alu_s", ctypes.c_double), ("t_pass_s", ctypes.c_double),
                ("run_time_s", ctypes.c_double), ("gcells", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class stencil_batch_grid(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("steps", ctypes.c_int), ("grid_in", ctypes.c_void_p),
                ("grid_out", ctypes.c_void_p), ("power", ctypes.c_void_p),
                ("coeffs", ctypes.c_float * 5)]


class stencil_tune_result(ctypes.Structure):
    _fields_ = [("force_T", ctypes.c_int), ("force_bx", ctypes.c_int), ("force_by", ctypes.c_int),
                ("force_vec", ctypes.c_int), ("partial_rows", ctypes.c_int),
                ("resident", ctypes.c_int), ("gcells", ctypes.c_double),
                ("model_gcells", ctypes.c_double), ("candidates", ctypes.c_int),
                ("timed", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# C ABI symbols, with their argument types
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "stencil_abi_version": ([], _I),
    "stencil_debug_fail_alloc": ([_I], _I),
    "stencil_debug_live_allocs": ([], ctypes.c_longlong),
    "stencil_strerror": ([_I], ctypes.c_char_p),
    "stencil_plan_create": ([ctypes.POINTER(_P), ctypes.POINTER(stencil_desc)], _I),
    "stencil_run": ([_P, _P, _P, _P, ctypes.POINTER(ctypes.c_float), _I, _I, _I, _I], _I),
    "stencil_plan_sync": ([_P], _I),
    "stencil_plan_set_wait": ([_P, ctypes.c_longlong, _I, _I], _I),
    "stencil_plan_get_info": ([_P, ctypes.POINTER(stencil_plan_info)], _I),
    "stencil_plan_set_timing": ([_P, _I], _I),
    "stencil_plan_kernel_time": ([_P, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_longlong), _I], _I),
    "stencil_plan_destroy": ([_P], _I),
    "stencil_batch_create": ([ctypes.POINTER(_P), ctypes.POINTER(stencil_batch_grid), _I, _P], _I),
    "stencil_batch_create_ex": ([ctypes.POINTER(_P), ctypes.POINTER(stencil_batch_grid), _I, _P, _I,
                                 _I, _I], _I),
    "stencil_batch_run": ([_P], _I),
    "stencil_batch_sync": ([_P], _I),
    "stencil_batch_set_wait": ([_P, ctypes.c_longlong, _I], _I),
    "stencil_batch_get_grid": ([_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "stencil_batch_launch_count": ([_P], _I),
    "stencil_batch_destroy": ([_P], _I),
    "stencil_reduce_workspace_bytes": ([], ctypes.c_size_t),
    "stencil_reduce": ([_P, _I, _P, _I, ctypes.c_longlong, _P, _P, _P], _I),
    "stencil_model_fpga": ([ctypes.POINTER(stencil_fpga_model_in),
                            ctypes.POINTER(stencil_fpga_model_out)], _I),
    "stencil_model_gpu": ([ctypes.POINTER(stencil_gpu_model_in),
                           ctypes.POINTER(stencil_gpu_model_out)], _I),
    "stencil_run_noalloc": ([_I, _P, _P, _P, ctypes.POINTER(ctypes.c_float), _I, _I, _I, _I, _I,
                             _P], _I),
    "stencil_adjoint_create": ([ctypes.POINTER(_P), _I, _I, _I, _I, _I, _P], _I),
    "stencil_adjoint_forward": ([_P, _P, _P, ctypes.POINTER(ctypes.c_float), _P], _I),
    "stencil_adjoint_backward": ([_P, _P, _P, _P, _P, _P, _P], _I),
    "stencil_adjoint_sync": ([_P], _I),
    "stencil_adjoint_destroy": ([_P], _I),
    "stencil_run_trajectory": ([_P, _P, _P, ctypes.c_longlong, _P, ctypes.POINTER(ctypes.c_float), _I],
                               _I),
    "stencil_tune": ([ctypes.POINTER(stencil_desc), _P, _P, _P, ctypes.POINTER(ctypes.c_float), _I,
                      _I, ctypes.POINTER(stencil_tune_result)], _I),
    "stencil_plan_tuned": ([_P], _I),
    "stencil_tune_cache_clear": ([], _I),
    "stencil_tune_cache_size": ([], _I),
    "stencil_tune_cache_save": ([ctypes.c_char_p], _I),
    "stencil_tune_cache_load": ([ctypes.c_char_p], _I),
    "stencil_fp32_peak": ([ctypes.POINTER(ctypes.c_double), _P], _I),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libstencil.so is not built ({LIB_PATH}); run the package's build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()


def strerror(code: int) -> str:
    return lib.stencil_strerror(int(code)).decode()


def _check(rc: int, what: str):
    if rc != ST_OK:
        raise StencilError(rc, what)


def _addr(t):
    """Device address of a torch tensor (float32, contiguous, on a CUDA device) or an int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor or an integer device address")
    if not t.is_cuda:
        raise ValueError("grids must live on a CUDA device")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("grids must be contiguous float32")
    return t.data_ptr()


def _coef_array(coeffs):
    if coeffs is None:   # ST_DIFFUSION_VAR plans take their coefficients from device planes
        return None
    vals = [float(v) for v in (coeffs.tolist() if hasattr(coeffs, "tolist") else coeffs)]
    return (ctypes.c_float * len(vals))(*vals)


def current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _desc(kind, ndim, nx, ny, nz, storage, force_T, force_bx, force_by, force_vec, exact, strict,
          stream, rad, partial_rows=0, resident=0):
    return stencil_desc(kind, ndim, nx, ny, nz if ndim == 3 else 1, storage, force_T, force_bx,
                        force_by, force_vec, 1 if exact else 0, 1 if strict else 0,
                        current_stream() if stream is None else stream, rad, partial_rows,
                        resident)


def stencil_plan_create(kind: int, ndim: int, nx: int, ny: int, nz: int = 1, *, storage=ST_F32,
                        force_T=0, force_bx=0, force_by=0, force_vec=0, exact=False,
                        strict=False, stream=None, rad=0, partial_rows=0, resident=0):
    d = _desc(kind, ndim, nx, ny, nz, storage, force_T, force_bx, force_by, force_vec, exact,
              strict, stream, rad, partial_rows, resident)
    h = ctypes.c_void_p()
    _check(lib.stencil_plan_create(ctypes.byref(h), ctypes.byref(d)), "stencil_plan_create")
    return h


def stencil_run(plan, grid_in, grid_out, power, coeffs, nx, ny, nz, steps):
    k = _coef_array(coeffs)
    _check(lib.stencil_run(plan, _addr(grid_in), _addr(grid_out), _addr(power), k, int(nx),
                           int(ny), int(nz), int(steps)), "stencil_run")


def stencil_run_trajectory(plan, grid_in, states, stride, power, coeffs, steps):
    """Every state of a `steps`-step run: state t+1 at states + t * stride floats."""
    _check(lib.stencil_run_trajectory(plan, _addr(grid_in), _addr(states), int(stride), _addr(power),
                                      _coef_array(coeffs), int(steps)), "stencil_run_trajectory")


def stencil_plan_sync(plan):
    _check(lib.stencil_plan_sync(plan), "stencil_plan_sync")


def stencil_plan_get_info(plan) -> dict:
    info = stencil_plan_info()
    _check(lib.stencil_plan_get_info(plan, ctypes.byref(info)), "stencil_plan_get_info")
    d = info.as_dict()
    d["tuned"] = bool(lib.stencil_plan_tuned(plan))
    return d


def stencil_tune(kind: int, ndim: int, nx: int, ny: int, nz: int, grid_in, grid_out, coeffs,
                 steps: int, power=None, *, top_k: int = 5, storage=ST_F32, exact=False,
                 strict=False, stream=None, rad=0) -> dict:
    """Time the model's top_k configurations on these grids and cache the fastest for the
    problem (kind, ndim, sizes, storage, exact, rad); later plans of that problem with nothing
    forced use it.  top_k = 5 follows the paper's fewer-than-six candidates per stencil."""
    d = _desc(kind, ndim, nx, ny, nz, storage, 0, 0, 0, 0, exact, strict, stream, rad)
    r = stencil_tune_result()
    _check(lib.stencil_tune(ctypes.byref(d), _addr(grid_in), _addr(grid_out), _addr(power),
                            _coef_array(coeffs), int(steps), int(top_k), ctypes.byref(r)),
           "stencil_tune")
    return r.as_dict()


def stencil_tune_cache_clear():
    _check(lib.stencil_tune_cache_clear(), "stencil_tune_cache_clear")


def stencil_tune_cache_size() -> int:
    return int(lib.stencil_tune_cache_size())


def stencil_tune_cache_save(path: str):
    _check(lib.stencil_tune_cache_save(os.fsencode(path)), "stencil_tune_cache_save")


def stencil_tune_cache_load(path: str):
    _check(lib.stencil_tune_cache_load(os.fsencode(path)), "stencil_tune_cache_load")


def stencil_plan_set_timing(plan, enable: bool):
    _check(lib.stencil_plan_set_timing(plan, 1 if enable else 0), "stencil_plan_set_timing")


def stencil_plan_kernel_time(plan, reset: bool = True):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(lib.stencil_plan_kernel_time(plan, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0),
           "stencil_plan_kernel_time")
    return ms.value, n.value


def stencil_plan_destroy(plan):
    _check(lib.stencil_plan_destroy(plan), "stencil_plan_destroy")


REDUCE_FIELDS = ("sum_a", "sumsq_a", "maxabs_a", "sum_b", "sumsq_b", "maxabs_b", "sumsq_diff",
                 "maxabs_diff")


def stencil_reduce(a, b=None, stream=None) -> dict:
    """Float64 statistics of grid a (float32 or float64 CUDA tensor) and, with b, of b and a-b
    (see include/stencil.h).  Synchronises the stream to return host values."""
    import torch

    def typed(t):
        if t.dtype == torch.float32:
            return ST_F32
        if t.dtype == torch.float64:
            return ST_F64
        raise ValueError("float32 or float64 tensors only")

    if not (a.is_cuda and a.is_contiguous()) or (b is not None and not (b.is_cuda and b.is_contiguous())):
        raise ValueError("contiguous CUDA tensors only")
    if b is not None and b.numel() != a.numel():
        raise ValueError("a and b differ in size")
    ws = torch.empty(lib.stencil_reduce_workspace_bytes() // 8, dtype=torch.float64, device=a.device)
    out = torch.zeros(8, dtype=torch.float64, device=a.device)
    st = current_stream() if stream is None else stream
    _check(lib.stencil_reduce(a.data_ptr(), typed(a), None if b is None else b.data_ptr(),
                              typed(b) if b is not None else 0, a.numel(), out.data_ptr(),
                              ws.data_ptr(), st), "stencil_reduce")
    vals = out.cpu().tolist()
    return dict(zip(REDUCE_FIELDS, vals))


def stencil_fp32_peak(stream=None) -> float:
    """Measured float32 fused-multiply-add rate of the current device, TFLOP/s."""
    v = ctypes.c_double()
    _check(lib.stencil_fp32_peak(ctypes.byref(v), current_stream() if stream is None else stream),
           "stencil_fp32_peak")
    return v.value


def stencil_model_fpga(**kw) -> dict:
    """The paper's performance model (Eqs. 3-9); keyword arguments are the fields of
    stencil_fpga_model_in."""
    m = stencil_fpga_model_in(**kw)
    r = stencil_fpga_model_out()
    _check(lib.stencil_model_fpga(ctypes.byref(m), ctypes.byref(r)), "stencil_model_fpga")
    return r.as_dict()


def stencil_model_gpu(**kw) -> dict:
    """GPU restatement of the model; keyword arguments are the fields of stencil_gpu_model_in."""
    m = stencil_gpu_model_in(**kw)
    r = stencil_gpu_model_out()
    _check(lib.stencil_model_gpu(ctypes.byref(m), ctypes.byref(r)), "stencil_model_gpu")
    return r.as_dict()


def _check_extent(t, need: int, name: str):
    """Refuse a tensor that holds fewer than `need` elements or lives on another device than
    the current one (the device whose buffers and SM count the library uses for the call):
    either would make the kernels read or write outside the tensor.  Integer addresses are the
    caller's responsibility.  Runs before anything is launched."""
    if t is None or isinstance(t, int):
        return
    if t.numel() < need:
        raise ValueError(f"{name} holds {t.numel()} elements, the grid needs {need}")
    import torch
    if t.get_device() != torch.cuda.current_device():
        raise ValueError(f"{name} is on device {t.get_device()}, the current device is "
                         f"{torch.cuda.current_device()}")


def stencil_run_noalloc(kind, grid_in, grid_out, power, coeffs, nx, ny, steps, exact=False, T=0,
                        stream=None):
    """2D run without a plan and without any device allocation (see include/stencil.h): for
    callers that must not allocate device memory where they advance a grid.  Uses a fixed
    16 MiB buffer the library reserves per device; larger grids raise ST_ERR_TOO_LARGE.
    Tensors smaller than nx*ny elements, or on a device other than the current one, raise
    ValueError before any work is queued."""
    n = int(nx) * int(ny)
    for name, t in (("grid_in", grid_in), ("grid_out", grid_out), ("power", power)):
        _check_extent(t, n, name)
    k = _coef_array(coeffs)
    _check(lib.stencil_run_noalloc(int(kind), _addr(grid_in), _addr(grid_out), _addr(power), k,
                                   int(nx), int(ny), int(steps), 1 if exact else 0, int(T),
                                   current_stream() if stream is None else stream),
           "stencil_run_noalloc")


class Batch:
    """Owning wrapper of stencil_batch: grids is a list of dicts with keys kind, nx, ny, steps,
    grid_in, grid_out, power (CUDA tensors or None) and coeffs."""

    def __init__(self, grids, stream=None, rows_per_item=0, force_T=0, force_vec=0):
        arr = (stencil_batch_grid * len(grids))()
        for i, g in enumerate(grids):
            arr[i].kind = g["kind"]
            arr[i].nx = g["nx"]
            arr[i].ny = g["ny"]
            arr[i].steps = g["steps"]
            arr[i].grid_in = _addr(g["grid_in"])
            arr[i].grid_out = _addr(g["grid_out"])
            arr[i].power = _addr(g.get("power"))
            for j, c in enumerate(list(g["coeffs"])[:5]):
                arr[i].coeffs[j] = float(c)
        self.keep = grids
        self.h = ctypes.c_void_p()
        _check(lib.stencil_batch_create_ex(ctypes.byref(self.h), arr, len(grids), stream,
                                           int(rows_per_item), int(force_T), int(force_vec)),
               "stencil_batch_create_ex")

    def run(self):
        _check(lib.stencil_batch_run(self.h), "stencil_batch_run")

    def sync(self):
        """Wait for the last replay; raises StencilError(ST_ERR_TIMEOUT) if a bounded wait of
        the persistent launch gave up."""
        _check(lib.stencil_batch_sync(self.h), "stencil_batch_sync")

    def set_wait(self, wait_ns: int, hold_pass: int = -1):
        """Wait limit of the launch's dependency waits; hold_pass >= 0 is the test hook that
        keeps that pass from ever reporting finished (see include/stencil.h)."""
        _check(lib.stencil_batch_set_wait(self.h, int(wait_ns), int(hold_pass)),
               "stencil_batch_set_wait")

    def grid_info(self, g):
        t, v, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.stencil_batch_get_grid(self.h, g, ctypes.byref(t), ctypes.byref(v), ctypes.byref(p)),
               "stencil_batch_get_grid")
        return {"T": t.value, "vec": v.value, "passes": p.value}

    def launches(self):
        return int(lib.stencil_batch_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _check(lib.stencil_batch_destroy(self.h), "stencil_batch_destroy")
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owning wrapper: a plan for one grid shape, destroyed with the object."""

    def __init__(self, kind, ndim, nx, ny, nz=1, **kw):
        self.kind, self.ndim, self.nx, self.ny = kind, ndim, nx, ny
        self.nz = nz if ndim == 3 else 1
        self.h = stencil_plan_create(kind, ndim, nx, ny, self.nz, **kw)

    def run(self, grid_in, grid_out, coeffs, steps, power=None):
        n = self.nx * self.ny * self.nz
        _check_extent(grid_in, n, "grid_in")
        _check_extent(grid_out, n, "grid_out")
        _check_extent(power, 5 * n if self.kind == ST_DIFFUSION_VAR else n, "power")
        stencil_run(self.h, grid_in, grid_out, power, coeffs, self.nx, self.ny, self.nz, steps)
        return grid_out

    def trajectory(self, grid_in, states, coeffs, steps, power=None):
        """Every state of a `steps`-step run into states, shaped (steps, ny, nx): states[t] is
        the field after t+1 steps."""
        stencil_run_trajectory(self.h, grid_in, states, self.nx * self.ny * self.nz, power, coeffs,
                               steps)
        return states

    def sync(self):
        stencil_plan_sync(self.h)

    def set_wait(self, wait_ns, hold_block=-1, hold_epoch=-1):
        """Bounded waits of a resident-tile plan (see stencil_plan_set_wait)."""
        _check(lib.stencil_plan_set_wait(self.h, int(wait_ns), int(hold_block), int(hold_epoch)),
               "stencil_plan_set_wait")

    def info(self):
        return stencil_plan_get_info(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            stencil_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- adjoint (reverse-mode gradient of a 2D run) ------------------------------------------------

def stencil_adjoint_create(kind, nx, ny, steps, ckpt=20, stream=None):
    h = ctypes.c_void_p()
    _check(lib.stencil_adjoint_create(ctypes.byref(h), int(kind), int(nx), int(ny), int(steps),
                                      int(ckpt), current_stream() if stream is None else stream),
           "stencil_adjoint_create")
    return h


def stencil_adjoint_forward(adj, u0, power, coeffs, u_out):
    k = _coef_array(coeffs)
    _check(lib.stencil_adjoint_forward(adj, _addr(u0), _addr(power), k, _addr(u_out)),
           "stencil_adjoint_forward")


def stencil_adjoint_backward(adj, grad_out, power, grad_u0, grad_coeffs, grad_coeffs_abs=None,
                             grad_power=None):
    _check(lib.stencil_adjoint_backward(adj, _addr(grad_out), _addr(power), _addr(grad_u0),
                                        _addr(grad_coeffs), _addr(grad_coeffs_abs),
                                        _addr(grad_power)), "stencil_adjoint_backward")


def stencil_adjoint_sync(adj):
    _check(lib.stencil_adjoint_sync(adj), "stencil_adjoint_sync")


def stencil_adjoint_destroy(adj):
    _check(lib.stencil_adjoint_destroy(adj), "stencil_adjoint_destroy")


class Adjoint:
    """Owning wrapper of stencil_adjoint: forward run with checkpoints every `ckpt` steps, then
    gradients of the last forward run for an upstream gradient dL/du_steps."""

    def __init__(self, kind, nx, ny, steps, ckpt=20, stream=None):
        self.kind, self.nx, self.ny, self.steps = kind, nx, ny, steps
        self.h = stencil_adjoint_create(kind, nx, ny, steps, ckpt, stream)

    def forward(self, u0, coeffs, power=None, out=None):
        import torch
        out = torch.empty_like(u0) if out is None else out
        stencil_adjoint_forward(self.h, u0, power, coeffs, out)
        return out

    def backward(self, grad_out, power=None, with_abs=False):
        """Returns (dL/du0, dL/dcoeffs, dL/dpower or None, sum|terms| per coefficient or None),
        all CUDA tensors on grad_out's device."""
        import torch
        gu = torch.empty_like(grad_out)
        gk = torch.empty(5, dtype=torch.float32, device=grad_out.device)
        ga = torch.empty(5, dtype=torch.float32, device=grad_out.device) if with_abs else None
        gp = torch.empty_like(grad_out) if self.kind == ST_THERMAL else None
        stencil_adjoint_backward(self.h, grad_out, power, gu, gk, ga, gp)
        return gu, gk, gp, ga

    def sync(self):
        stencil_adjoint_sync(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            stencil_adjoint_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class StencilSweep(torch.autograd.Function):
        """u_steps = sweep(u0, coeffs, power): `steps` Jacobi steps of a 2D stencil; backward by
        the adjoint sweep (checkpoints every `ckpt` steps)."""

        @staticmethod
        def forward(ctx, u0, coeffs, power, kind, steps, ckpt):
            u0c = u0.detach().contiguous()
            pw = None if power is None else power.detach().contiguous()
            adj = Adjoint(kind, u0c.shape[1], u0c.shape[0], steps, ckpt)
            out = adj.forward(u0c, coeffs.detach().cpu(), pw)
            ctx.adj, ctx.pw = adj, pw
            ctx.coef_device = coeffs.device
            return out

        @staticmethod
        def backward(ctx, grad_out):
            gu, gk, gp, _ = ctx.adj.backward(grad_out.detach().contiguous(), ctx.pw)
            ctx.adj.close()
            return gu, gk.to(ctx.coef_device), gp, None, None, None

    return StencilSweep


_SWEEP = None


def stencil_sweep(u0, coeffs, steps, kind=ST_DIFFUSION, power=None, ckpt=20):
    """Differentiable 2D sweep (torch.autograd): u0 (ny, nx) float32 CUDA tensor, coeffs a
    float32 tensor of 5 (any device), power (ny, nx) CUDA tensor for ST_THERMAL.  Gradients flow
    to u0, coeffs and power."""
    global _SWEEP
    if _SWEEP is None:
        _SWEEP = _autograd_function()
    return _SWEEP.apply(u0, coeffs, power, kind, int(steps), int(ckpt))
