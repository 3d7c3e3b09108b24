"""Benchmark of the temporally-blocked stencil engine (arXiv 1802.00438: iterated first-order
Jacobi sweeps with combined spatial and temporal blocking).

Headline workload: Hotspot 2D (thermal), 16384 x 16384 float32 cells, 1000 time steps, seeded
synthetic inputs (temperature U[320,340) K, power U[0,0.5), ambient 80).  One benchmark "step"
is one full run of the hot path: stencil_run advancing the grid by 1000 time steps
(ceil(1000/T) temporally-blocked passes).

Prints one JSON line (rank 0): throughput in GCell/s (cell updates per second, the unit the
paper's Table 4 quotes beside GB/s and GFLOP/s), the dominant kernel's roofline fraction, the
end-to-end figure through the C ABI with host buffers, the CPU oracle's throughput on a bounded
sample of the same workload, and, under "configs", the same record for every other
configuration: Diffusion 2D 1024^2 x 100, Diffusion 3D 512^3 x 1000, Hotspot 3D 512x512x256 x
1000, the 64-grid batch and the adjoint of a 2048^2 x 200 diffusion run; under "lowp" the bf16
and fp16 storage runs of the headline workload with their error against the float64 oracle,
computed on the GPU by the library's float64 reductions.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

--workload NAME measures that one workload alone.  With --gpus N > 1 (launched by
torch.distributed.run) every rank advances its own grid: the method has no cross-grid exchange,
so the job is N independent replicas (weak scaling) with a barrier around the timed region and
the time taken as the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "stencil GCell/s & GFLOP/s vs roofline; BF16-store vs FP32 speedup at err"
# per-cell counts (Table 2): counted flops, bytes per cell per pass (field in/out, power in)
FLOPS = {(0, 2): 9, (0, 3): 13, (1, 2): 15, (1, 3): 17}
BYTES = {0: 8, 1: 12}

BATCH = "batch64"   # 64 2D grids of uneven sizes and step counts in one graph launch
ADJOINT = "adjoint2048"   # gradient of a 2048^2, 200-step diffusion run, checkpoints every 20

WORKLOADS = {
    "thermal2d_16384": lambda: synth.c2_thermal2d(),
    "diffusion2d_1024": lambda: synth.c1_diffusion2d(),
    "diffusion3d_512": lambda: synth.c3a_diffusion3d(),
    "thermal3d_512x512x256": lambda: synth.c3b_thermal3d(),
    # radius-2 star diffusion (9 points; Eqs. 1-2 with rad = 2), the 2D diffusion grid size
    "star2_2d_16384": lambda: synth.make_star(2, 2, 16384, 16384, steps=1000, seed=7,
                                              name="star2_2d_16384x16384_1000"),
    # radius-2 star diffusion in 3D (13 points), the 3D diffusion grid size
    "star2_3d_512": lambda: synth.make_star(3, 2, 512, 512, 512, steps=1000, seed=9,
                                            name="star2_3d_512x512x512_1000"),
    # diffusion 2D with per-cell coefficients (Table 2 row 1, coefficients as arrays)
    "vardiff2d_8192": lambda: synth.make_vdiff(8192, 8192, steps=1000, seed=8,
                                               name="vardiff2d_8192x8192_1000"),
}
BYTES_VAR = 28   # per cell and pass: field in and out, five coefficient planes
DEFAULT = "thermal2d_16384"
# the other configurations, measured as sub-records of the default run
SUBCONFIGS = ("diffusion2d_1024", "diffusion3d_512", "thermal3d_512x512x256", BATCH, ADJOINT)
L2_BYTES = 129 * 2 ** 20


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """Nominal FP32 ALU peak: SMs x 128 FP32 lanes x 2 flops per fused multiply-add x clock."""
    return sms * 128 * 2 * mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


class Replicas:
    """The N-process launch (torch.distributed.run, one process per GPU): every rank advances
    its own copy of the workload (the method exchanges nothing between grids), the ranks meet at
    a barrier around each timed region, a region's time is the maximum over the ranks, and the
    job's rate is all ranks' units over that time.  backend "gloo" with a CPU device runs the
    same logic without GPUs."""

    def __init__(self, backend: str = "nccl", device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group(backend, device_id=device)
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max_ms(self, ms: float) -> float:
        if not self.dist:
            return ms
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_rate(self, units_per_rank: float, ms: float) -> float:
        """Units per second of the whole job: every rank did units_per_rank in at most ms."""
        return self.world * units_per_rank / (ms * 1e-3)


def reference_rank_gate() -> bool:
    """The reference arm (the CPU oracle) runs on rank 0 alone; other ranks exit at once."""
    return int(os.environ.get("RANK", "0")) == 0


def kernel_source_hash(ndim: int, resident: bool = False) -> str:
    """Hash of the sources of the benchmarked kernel family (2D streaming, 2D resident tiles
    or 3D)."""
    files = (("res2d.cu", "common.cuh") if resident else
             ("tb2f_kernel.cuh", "tb2d_kernel.cuh", "common.cuh") if ndim == 2
             else ("tb3f_kernel.cuh", "tb3d_kernel.cuh", "common.cuh"))
    h = hashlib.sha1()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1802_00438_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(workload: str, ndim: int, resident: bool = False):
    """DRAM bytes per launch recorded from an ncu capture of the current kernel source
    (profiles/traffic.txt); None when the kernel changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == workload:
            return float(f[2]) if f[1] == kernel_source_hash(ndim, resident) else None
    return None


def workload_config(w) -> dict:
    """The workload's identity (shared by the engine and the reference arm)."""
    return {"workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz, "time_steps": w.steps,
            "l2": ("inputs larger than L2 (%.0f MiB per grid)" % (w.u0.nbytes / 2 ** 20)
                   if w.u0.nbytes > L2_BYTES else
                   "grid fits in L2 (%.0f MiB): L2-resident, no flush" % (w.u0.nbytes / 2 ** 20))}


# ---- the oracle: CPU baselines and the reference arm ----------------------------------------

def _oracle_run(w, steps, dtype=np.float32):
    import oracle
    if w.var:
        return oracle.run_vdiff2d(w.u0, w.coef, steps, dtype=dtype)
    if w.rad > 1:
        return oracle.run_star(w.rad, w.u0, w.coef, steps, dtype=dtype)
    return oracle.run(w.kind, w.u0, w.coef, steps, w.power, dtype=dtype)


def _flops(w):
    """Counted flops per cell update: Table 2's for the first-order stencils, 8R + 1 (2D) or
    12R + 1 (3D) for the radius-R star (one multiply and 2 ndim R multiply-adds counted as two
    flops each)."""
    return 4 * w.ndim * w.rad + 1 if w.rad > 1 else FLOPS[(w.kind, w.ndim)]


def _oracle_sample_steps(w, budget_s: float, threads: int | None = None):
    """Time steps of the full grid that take about budget_s seconds on `threads` host cores
    (all cores of the affinity mask by default), from one timed 2-step run after a 1-step
    warm-up."""
    import oracle
    oracle.build()
    cores = threads or len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    _oracle_run(w, 1)
    t0 = time.perf_counter()
    _oracle_run(w, 2)
    per_step = max((time.perf_counter() - t0) / 2, 1e-6)
    return max(1, min(w.steps, int(budget_s / per_step))), cores


def cpu_baseline(w, budget_s: float = 10.0, threads: int | None = None):
    """The oracle as it stands, on the host cores, over a bounded sample of the workload: the
    full grid for as many time steps as fit in about `budget_s` seconds."""
    import oracle
    steps, cores = _oracle_sample_steps(w, budget_s, threads)
    t0 = time.perf_counter()
    _oracle_run(w, steps)
    t = time.perf_counter() - t0
    oracle.set_threads(len(os.sched_getaffinity(0)))
    return {"value": w.cells * steps / t / 1e9, "unit": "GCell/s", "cores": cores,
            "kind": "oracle",
            "sample": f"full {'x'.join(map(str, w.shape[::-1]))} grid, {steps} of {w.steps} "
                      f"time steps ({t:.1f} s; float32 oracle, OpenMP over rows)"}


def run_reference(args, w):
    """Reference arm: the CPU oracle, each benchmark step a bounded sample of the workload
    (about 120 s over all warm-up and timed steps)."""
    per_step = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    steps, cores = _oracle_sample_steps(w, per_step)
    for _ in range(args.warmup):
        _oracle_run(w, steps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_run(w, steps)
    t = time.perf_counter() - t0
    value = w.cells * steps * args.steps / t / 1e9
    sample = (f"full {'x'.join(map(str, w.shape[::-1]))} grid, {steps} of {w.steps} time steps "
              f"per benchmark step (float32 oracle, OpenMP over rows)")
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "GCell/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": "GCell/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GCell/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_reference(args, ws):
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    frac = 1.0 / 40          # each grid for 1/40 of its steps (at least one)
    t0 = time.perf_counter()
    done = 0
    for _ in range(max(1, args.steps)):
        for w in ws:
            s = max(1, int(w.steps * frac))
            oracle.run(w.kind, w.u0, w.coef, s, w.power)
            done += w.cells * s
    t = time.perf_counter() - t0
    return {"value": done / t / 1e9, "unit": "GCell/s", "cores": cores, "kind": "oracle",
            "sample": "all 64 grids, 1/40 of each grid's steps"}


def adjoint_reference(reps, ckpt, seed_kind):
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    side, s = 512, 20   # bounded sample: a 512^2, 20-step gradient (checkpoints every 20)
    ws = synth.make(seed_kind[1], 2, side, side, 1, s, seed=seed_kind[0])
    wts = synth.loss_weights(6, ws.shape)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.adjoint2d(ws.kind, ws.u0, ws.coef, s, wts, None, ckpt=ckpt)
    t = (time.perf_counter() - t0) / reps
    return {"value": side * side * s / t / 1e9, "unit": "GCell/s", "cores": cores,
            "kind": "oracle", "sample": f"float64 adjoint of a {side}^2, {s}-step diffusion "
                                        f"run (the transposed sweep is one thread)"}


# ---- GPU timing -----------------------------------------------------------------------------

class Gpu:
    """Device, stream and replica group shared by every measurement of a run."""

    def __init__(self):
        import torch
        self.torch = torch
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.rk = Replicas("nccl", self.dev)
        # a stream of our own, current for the whole run (a CUDA graph cannot be captured on
        # the legacy default stream)
        self.stream = torch.cuda.Stream(self.dev)
        torch.cuda.set_stream(self.stream)
        import paper_1802_00438_gb300 as st
        self.st = st
        self.sms = torch.cuda.get_device_properties(self.dev).multi_processor_count
        self.peaks, self.peak_src = load_peaks()

    def timed(self, fn, steps: int, warmup: int):
        """W untimed calls, then K timed ones between a barrier and synchronize on both sides,
        one CUDA event pair per call on the stream (device time).  Returns (total ms as the max
        over ranks, per-call ms list, clock summary)."""
        torch = self.torch
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        self.rk.barrier()
        torch.cuda.synchronize()
        with Clocks(self.local) as clk:
            ev[0].record(self.stream)
            for i in range(steps):
                fn()
                ev[i + 1].record(self.stream)
            torch.cuda.synchronize()
        self.rk.barrier()
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        total = self.rk.max_ms(ev[0].elapsed_time(ev[steps]))
        return total, per, clk.summary()


def plan_record(g: Gpu, w, args, steps: int, warmup: int, with_cpu: bool, one_thread=False,
                key: str = ""):
    """Measure one workload through a plan: value, roofline of its kernel, e2e, CPU baseline."""
    torch, st, rk = g.torch, g.st, g.rk
    stream = g.stream
    u0 = torch.from_numpy(w.u0).to(g.dev)
    # the per-cell input: the power map, or the five coefficient planes of ST_DIFFUSION_VAR
    kind = st.ST_DIFFUSION_VAR if w.var else w.kind
    h_pin = w.coef if w.var else w.power
    pw = None if h_pin is None else torch.from_numpy(h_pin).to(g.dev)
    coef = None if w.var else w.coef
    out = torch.empty_like(u0)
    tuned = None
    if args.tune > 0:
        tuned = st.stencil_tune(kind, w.ndim, w.nx, w.ny, w.nz, u0, out, coef, w.steps, pw,
                                top_k=args.tune, storage=args.storage, stream=stream.cuda_stream,
                                rad=w.rad if w.rad > 1 else 0)
    plan = st.Plan(kind, w.ndim, w.nx, w.ny, w.nz, force_T=args.T, force_bx=args.bx,
                   force_vec=args.vec, force_by=args.by, partial_rows=args.rows,
                   resident=args.resident, storage=args.storage,
                   stream=stream.cuda_stream, rad=w.rad if w.rad > 1 else 0)
    info = plan.info()
    T = info["T"]
    # resident tiles read and write the grid once per run: every step of it is fused per pass
    # over device memory (T is then the steps between halo exchanges through L2)
    resident = bool(info.get("resident"))
    T_hbm = w.steps if resident else T

    def step():
        plan.run(u0, out, coef, w.steps, power=pw)

    # A run of a small grid is a few microseconds of kernels per pass: launched one by one it
    # would measure the host's launch rate, so it is captured once in a CUDA graph (the plan
    # launches on the stream being captured) and the timed steps replay the graph.
    graph = None
    if w.cells * w.steps < 2e9:
        step()
        torch.cuda.synchronize()
        try:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                step()
            torch.cuda.synchronize()
        except RuntimeError as e:   # a launch the capture does not support: run eagerly
            print(f"bench: CUDA graph capture failed ({e}); timing eager launches",
                  file=sys.stderr)
            graph = None
            torch.cuda.synchronize()
    timed_step = graph.replay if graph is not None else step
    for _ in range(warmup):
        timed_step()
    ms, per, clocks = g.timed(timed_step, steps, 0)
    # kernel time per launch for the roofline: the same runs again with the library's event
    # pair around every launch (outside the timed region)
    st.stencil_plan_set_timing(plan.h, True)
    st.stencil_plan_kernel_time(plan.h, reset=True)
    for _ in range(steps):
        step()
    kern_ms, timed_launches = st.stencil_plan_kernel_time(plan.h, reset=True)
    st.stencil_plan_set_timing(plan.h, False)
    launches = timed_launches
    if w.kind == 1 and w.ndim == 2 and not args.storage and not w.var and not resident:
        launches += steps   # the source-map kernel (sdc*(p + amb*Rz)) before each run's passes
    cells_step = w.cells * w.steps
    value = rk.job_rate(cells_step * steps, ms) / 1e9

    # ---- end to end through the C ABI with host buffers ----------------------------------
    e2e = None
    if not args.no_e2e:
        h_u = torch.from_numpy(w.u0).pin_memory()
        h_p = None if h_pin is None else torch.from_numpy(h_pin).pin_memory()
        h_o = torch.empty_like(h_u).pin_memory()
        d_u = torch.empty_like(u0)
        d_p = None if pw is None else torch.empty_like(pw)
        d_o = torch.empty_like(u0)

        def e2e_step():
            d_u.copy_(h_u, non_blocking=True)
            if d_p is not None:
                d_p.copy_(h_p, non_blocking=True)
            st.stencil_run(plan.h, d_u, d_o, d_p, coef, w.nx, w.ny, w.nz, w.steps)
            h_o.copy_(d_o, non_blocking=True)

        e2e_steps = min(steps, 100)   # each call copies the grids both ways: fewer calls
        ems, _, _ = g.timed(e2e_step, e2e_steps, 1)
        nb = w.u0.nbytes
        serial = rk.job_rate(cells_step * e2e_steps, ems) / 1e9
        del d_u, d_p, d_o

        # Streamed: the same calls with two device buffer sets, so that step k+1's input copies
        # (copy-in stream) and step k-1's result copy (copy-out stream) overlap step k's run on
        # the plan's stream; events hand each buffer over.  Every step still copies its inputs
        # from pinned host memory and reads its result back.
        s_in, s_out = torch.cuda.Stream(g.dev), torch.cuda.Stream(g.dev)
        sets = [(torch.empty_like(u0), None if pw is None else torch.empty_like(pw),
                 torch.empty_like(u0), h_o if i == 0 else torch.empty_like(h_u).pin_memory())
                for i in range(2)]
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_run = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def streamed(k_steps):
            for k in range(k_steps):
                b = k % 2
                du, dp, do, ho = sets[b]
                if k >= 2:
                    s_in.wait_event(ev_run[b])      # step k-2's run has read du, dp
                with torch.cuda.stream(s_in):
                    du.copy_(h_u, non_blocking=True)
                    if dp is not None:
                        dp.copy_(h_p, non_blocking=True)
                    ev_in[b].record(s_in)
                stream.wait_event(ev_in[b])
                if k >= 2:
                    stream.wait_event(ev_out[b])    # step k-2's result copy has read do
                st.stencil_run(plan.h, du, do, dp, coef, w.nx, w.ny, w.nz, w.steps)
                ev_run[b].record(stream)
                s_out.wait_event(ev_run[b])
                with torch.cuda.stream(s_out):
                    ho.copy_(do, non_blocking=True)
                    ev_out[b].record(s_out)

        streamed(2)
        torch.cuda.synchronize()
        rk.barrier()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s_in)
        streamed(e2e_steps)
        t1.record(s_out)
        torch.cuda.synchronize()
        rk.barrier()
        pms = rk.max_ms(t0.elapsed_time(t1))
        # the copy bandwidth the host link gave: one timed input copy alone
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        sets[0][0].copy_(h_u, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = nb / (c0.elapsed_time(c1) * 1e-3) / 1e9
        e2e = {"value": rk.job_rate(cells_step * e2e_steps, pms) / 1e9, "unit": "GCell/s",
               "h2d_bytes_per_step": nb + (0 if h_pin is None else h_pin.nbytes),
               "d2h_bytes_per_step": nb, "streamed": True, "serial_value": serial,
               "h2d_gbs": h2d_gbs,
               "note": "streamed: step k+1's input copies and step k-1's result copy overlap "
                       "step k's run (two device buffer sets, copy-in and copy-out streams); "
                       "serial_value: copy in, run, copy out one step after another"}
        del h_u, h_p, h_o, sets

    # ---- roofline of the dominant kernel ---------------------------------------------------
    mhz = float(g.peaks.get("sm_max_mhz", 2070.0))
    fl = _flops(w)
    by = BYTES_VAR if w.var else BYTES[w.kind]
    alu_peak = fp32_peak_tflops(g.sms, mhz)
    hbm_peak = float(g.peaks["hbm_gbs"])
    avg_launch_ms = kern_ms / max(timed_launches, 1)
    # algorithmic work of one launch, averaged over the timed launches (the last pass of a
    # run fuses the remainder of the steps)
    flops_per_launch = w.cells * w.steps * steps * fl / max(timed_launches, 1)
    bytes_per_launch = w.cells * by
    tflops = flops_per_launch / (avg_launch_ms * 1e-3) / 1e12
    gbs = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
    cell_roof = min(alu_peak * 1e12 / fl, hbm_peak * 1e9 * T_hbm / by)   # cells/s at this T
    alu_bound = alu_peak * 1e12 / fl <= hbm_peak * 1e9 * T_hbm / by
    resized = bool(args.nx or args.ny or args.nz or args.time_steps)
    traffic = None if (resized or args.T or args.bx or args.vec or args.by) else \
        profiled_traffic(key, w.ndim, resident)
    if alu_bound:
        roof = {"bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": tflops / alu_peak,
                "peak_note": f"FP32 {g.sms} SMs x 128 lanes x 2 x {mhz:.0f} MHz (max SM clock)"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak, "peak_note": f"{g.peak_src} copy bandwidth (burst)"}
    kern_rate = cells_step * steps / (kern_ms * 1e-3)
    roof.update({
        "traffic": traffic,
        "algorithmic_bytes_per_launch": bytes_per_launch,
        "kernel_ms_per_launch": avg_launch_ms,
        "cell_roofline_gcells": cell_roof / 1e9,
        "frac_of_cell_roofline": kern_rate / cell_roof,
        "hbm_frac": gbs / hbm_peak,
        # the T -> infinity ceiling: FP32 issue of the counted flops alone
        "fp32_ceiling_gcells": alu_peak * 1e3 / fl,
        "frac_of_fp32_ceiling": kern_rate / (alu_peak * 1e12 / fl)})
    rec = {"value": value, "unit": "GCell/s", "ms_per_step": ms / steps,
           "median_ms_per_step": statistics.median(per), "steps": steps, "warmup": warmup,
           "gflops": value * fl, "effective_gbs": value * by,
           "config": workload_config(w),
           "plan": {"T": T, "tile": [info["bx"], info["by"]], "vec": info["vec"],
                    "cuda_graph": graph is not None, "resident": resident,
                    "warps": info["warps"], "ctas": info["ctas"],
                    "passes_per_step": 1 if resident else -(-w.steps // T),
                    "exchanges_per_step": (-(-w.steps // T) - 1) if resident else None,
                    # the library's calibrated restatement of Eqs. 3-9 for this plan, and
                    # measured / predicted (the paper's model-accuracy figure)
                    "model_gcells": info["model_gcells"] or None,
                    "model_accuracy": (value / rk.world / info["model_gcells"]
                                       if info["model_gcells"] else None),
                    "tuned": tuned},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
    if with_cpu and rk.world == 1:
        rec["cpu_baseline"] = cpu_baseline(w)
        if one_thread:
            rec["cpu_baseline"]["one_thread"] = cpu_baseline(w, budget_s=10.0, threads=1)
    else:
        rec["cpu_baseline"] = None
    rec["_plan"] = plan
    rec["_bufs"] = (u0, pw, out)
    return rec


def lowp_record(g: Gpu, w, args, base_value: float, bufs, steps: int, warmup: int,
                with_err: bool):
    """16-bit grid storage on the headline workload: speed of each format at its own
    parameter choice against the float32 engine's, and (with_err) the error after the full
    step count against the float64 oracle, as relative L2 and L-infinity norms computed on the
    GPU by the library's float64 reductions (stencil_reduce)."""
    torch, st, rk = g.torch, g.st, g.rk
    u0, pw, out = bufs
    cells_step = w.cells * w.steps
    res = {}
    ref = None
    if with_err:
        import oracle
        oracle.set_threads(len(os.sched_getaffinity(0)))
        t0 = time.perf_counter()
        ref_h = oracle.run(w.kind, w.u0, w.coef, w.steps, w.power, dtype=np.float64)
        t_or = time.perf_counter() - t0
        ref = torch.from_numpy(ref_h).to(g.dev)
        del ref_h
        res["error_reference"] = (f"float64 oracle, full {w.nx}x{w.ny} grid, {w.steps} steps "
                                  f"({t_or:.0f} s on the host cores); norms by stencil_reduce "
                                  f"(float64 on the GPU)")

    def errs(o):
        r = st.stencil_reduce(o, ref)
        return {"rel_l2": (r["sumsq_diff"] / r["sumsq_b"]) ** 0.5,
                "rel_linf": r["maxabs_diff"] / r["maxabs_b"]}

    if ref is not None:
        plan = st.Plan(w.kind, 2, w.nx, w.ny, stream=g.stream.cuda_stream)
        plan.run(u0, out, w.coef, w.steps, power=pw)
        res["f32"] = errs(out)
        plan.close()
    for name, stor in (("bf16", st.ST_BF16), ("fp16", st.ST_F16)):
        qplan = st.Plan(w.kind, 2, w.nx, w.ny, storage=stor, stream=g.stream.cuda_stream)

        def qstep():
            qplan.run(u0, out, w.coef, w.steps, power=pw)

        qms, qper, qclk = g.timed(qstep, steps, warmup)
        qv = rk.job_rate(cells_step * steps, qms) / 1e9
        info = qplan.info()
        res[name] = {"value": qv, "unit": "GCell/s", "speedup_vs_f32": qv / base_value,
                     "median_ms_per_step": statistics.median(qper), "T": info["T"],
                     "vec": info["vec"], "clocks": qclk}
        if ref is not None:
            res[name].update(errs(out))
        qplan.close()
    del ref
    return res


def batch_record(g: Gpu, args, steps: int, warmup: int, with_cpu: bool):
    """64 grids (sides log-uniform in [256, 4096], steps uniform in {50..500}, kinds
    alternating): one step = one replay of the batch's CUDA graph."""
    torch, st, rk = g.torch, g.st, g.rk
    ws = synth.c5a_batch()
    cells_steps = sum(w.cells * w.steps for w in ws)
    stream = torch.cuda.Stream(g.dev)
    items = []
    for w in ws:
        u = torch.from_numpy(w.u0).to(g.dev)
        o = torch.empty_like(u)
        p = None if w.power is None else torch.from_numpy(w.power).to(g.dev)
        items.append({"kind": w.kind, "nx": w.nx, "ny": w.ny, "steps": w.steps, "grid_in": u,
                      "grid_out": o, "power": p, "coeffs": w.coef})
    torch.cuda.synchronize()
    b = st.Batch(items, stream=stream.cuda_stream)
    saved = g.stream
    g.stream = stream
    ms, per, clocks = g.timed(b.run, steps, warmup)
    value = rk.job_rate(cells_steps * steps, ms) / 1e9
    # roofline of the mix: sum over grids of cells*steps / R_g(T_g), R = min(ALU, HBM*T/bytes)
    alu = fp32_peak_tflops(g.sms, float(g.peaks.get("sm_max_mhz", 2070.0))) * 1e12
    hbm = float(g.peaks["hbm_gbs"]) * 1e9
    ideal = 0.0
    bytes_moved = 0.0
    tv = {}
    for i, w in enumerate(ws):
        gi = b.grid_info(i)
        R = min(alu / FLOPS[(w.kind, 2)], hbm * gi["T"] / BYTES[w.kind])
        ideal += w.cells * w.steps / R
        bytes_moved += w.cells * BYTES[w.kind] * gi["passes"]
        k = f"T{gi['T']}V{gi['vec']}"
        tv[k] = tv.get(k, 0) + 1
    per_step_s = ms * 1e-3 / steps
    gbs = bytes_moved / per_step_s / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": float(g.peaks["hbm_gbs"]), "unit": "GB/s",
            "frac": gbs / float(g.peaks["hbm_gbs"]), "traffic": None,
            "frac_of_cell_roofline": ideal / per_step_s,
            "note": "mix of 64 grids: achieved = algorithmic bytes of all passes / step time; "
                    "frac_of_cell_roofline = sum_g cells*steps/R_g(T_g) / step time"}
    # end to end: host inputs in, results out, through the same batch
    h_in = [torch.from_numpy(w.u0).pin_memory() for w in ws]
    h_out = [torch.empty_like(h).pin_memory() for h in h_in]

    def e2e_step():
        for it, h in zip(items, h_in):
            it["grid_in"].copy_(h, non_blocking=True)
        b.run()
        for it, h in zip(items, h_out):
            h.copy_(it["grid_out"], non_blocking=True)

    with torch.cuda.stream(stream):
        ems, _, _ = g.timed(e2e_step, steps, 1)
    g.stream = saved
    nb = sum(w.u0.nbytes for w in ws)
    e2e = {"value": rk.job_rate(cells_steps * steps, ems) / 1e9, "unit": "GCell/s",
           "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}
    rec = {"value": value, "unit": "GCell/s", "ms_per_step": ms / steps,
           "median_ms_per_step": statistics.median(per), "steps": steps, "warmup": warmup,
           "config": {"workload": BATCH, "grids": len(ws), "cell_updates_per_step": cells_steps,
                      "l2": "inputs larger than L2 in total (%.0f MiB)" % (nb / 2 ** 20)},
           "plan": {"graph_launches_per_step": b.launches(), "per_grid_T_V": tv},
           "roofline": roof, "e2e": e2e, "gpu_launches": b.launches() * steps, "clocks": clocks,
           "cpu_baseline": batch_reference(argparse.Namespace(steps=1), ws)
           if (with_cpu and rk.world == 1) else None}
    b.close()
    return rec


def adjoint_record(g: Gpu, args, steps: int, warmup: int, with_cpu: bool, ckpt=20):
    """Gradient of L = sum(w * u_200) for a 2048^2 diffusion run: one step = the checkpointed
    forward run plus the backward sweep (state recompute, transposed passes, reductions).
    value = primal cell updates (cells x 200) per second of a whole gradient evaluation."""
    torch, st, rk = g.torch, g.st, g.rk
    w = synth.c5b_adjoint2d()
    wt = synth.loss_weights(6, w.shape)
    n = w.cells
    stream = g.stream
    u0 = torch.from_numpy(w.u0).to(g.dev)
    gr = torch.from_numpy(wt).to(g.dev)
    adj = st.Adjoint(w.kind, w.nx, w.ny, w.steps, ckpt, stream=stream.cuda_stream)
    out = torch.empty_like(u0)
    gu = torch.empty_like(u0)
    gk = torch.empty(5, dtype=torch.float32, device=g.dev)

    def step():
        st.stencil_adjoint_forward(adj.h, u0, None, w.coef, out)
        st.stencil_adjoint_backward(adj.h, gr, None, gu, gk, None, None)

    def fwd():
        st.stencil_adjoint_forward(adj.h, u0, None, w.coef, out)

    ms, per, clocks = g.timed(step, steps, warmup)
    fms, _, _ = g.timed(fwd, steps, 1)
    per_ms = ms / steps
    bwd = per_ms - fms / steps
    value = rk.job_rate(n * w.steps * steps, ms) / 1e9
    # algorithmic HBM bytes of the backward: per transposed pass of s steps lambda in + out
    # (8 B) and the s states (4 B each); per segment the checkpoint copy into the state buffer
    # (8 B) and one trajectory run that reads it and writes the L-1 recomputed states (4 B
    # each); grad_u0 copy (8 B)
    nseg = -(-w.steps // ckpt)
    seg_len = [min(w.steps, (k + 1) * ckpt) - k * ckpt for k in range(nseg)]
    bytes_b = 0
    for L in seg_len:
        bytes_b += n * (4 * (L - 1) + 4 + 8)
        left = L
        while left > 0:
            s = min(4, left)
            bytes_b += n * (8 + 4 * s)
            left -= s
    bytes_b += 8 * n
    gbs = bytes_b / (bwd * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": float(g.peaks["hbm_gbs"]), "unit": "GB/s",
            "frac": gbs / float(g.peaks["hbm_gbs"]), "traffic": None,
            "note": "whole backward (state recompute + transposed passes): algorithmic bytes / "
                    "backward time (step time minus the checkpointed forward run)"}
    h_u = torch.from_numpy(w.u0).pin_memory()
    h_g = torch.from_numpy(wt).pin_memory()
    h_gu = torch.empty_like(h_u).pin_memory()
    h_gk = torch.empty(5, dtype=torch.float32).pin_memory()

    def e2e_step():
        u0.copy_(h_u, non_blocking=True)
        gr.copy_(h_g, non_blocking=True)
        step()
        h_gu.copy_(gu, non_blocking=True)
        h_gk.copy_(gk, non_blocking=True)

    ems, _, _ = g.timed(e2e_step, steps, 1)
    e2e = {"value": rk.job_rate(n * w.steps * steps, ems) / 1e9, "unit": "GCell/s",
           "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 * n + 20}
    fwd_T = st.Plan(w.kind, 2, w.nx, w.ny).info()["T"]
    launches = sum(-(-L // fwd_T) for L in seg_len)            # forward passes
    launches += sum(-(-(L - 1) // 8) for L in seg_len)           # trajectory passes
    launches += sum(-(-L // 4) for L in seg_len) + 2             # transposed passes + 2-level sum
    rec = {"value": value, "unit": "GCell/s", "ms_per_step": per_ms,
           "median_ms_per_step": statistics.median(per), "steps": steps, "warmup": warmup,
           "config": {"workload": ADJOINT, "grid": f"{w.nx}x{w.ny}", "time_steps": w.steps,
                      "checkpoint_every": ckpt,
                      "l2": "inputs larger than L2 (200-state sweep over 16 MiB grids; "
                            "496 MiB of buffers)"},
           "plan": {"forward_ms": fms / steps, "backward_ms": bwd},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches * steps, "clocks": clocks,
           "cpu_baseline": adjoint_reference(1, ckpt, (w.seed, w.kind))
           if (with_cpu and rk.world == 1) else None}
    adj.close()
    return rec


# configurations of the model-accuracy study: 2D (T, cells per lane, variant 1 = partial rows
# in place) and 3D (T, tile width, tile height, cells per thread), every one the library compiles
STUDY_2D = [(1, 8, 0), (2, 8, 0), (4, 8, 0), (6, 8, 0), (8, 8, 0), (8, 8, 1),
            (1, 4, 0), (2, 4, 0), (4, 4, 0), (8, 4, 0), (12, 4, 0), (12, 4, 1)]
# resident tiles (small 2D grids): (T, cells per lane)
STUDY_RES = [(T, v) for v in (2, 4) for T in (2, 4, 8, 12, 16, 20)]
STUDY_3D = [(1, 64, 64, 8), (2, 64, 64, 8), (3, 64, 64, 8), (4, 64, 64, 8),
            (2, 64, 64, 4), (3, 64, 64, 4), (4, 64, 64, 4),
            (2, 128, 32, 8), (3, 128, 32, 8), (4, 128, 32, 8),
            (2, 64, 32, 8), (3, 64, 32, 8), (4, 64, 32, 8)]


def model_study(g: Gpu, args):
    """Measured / predicted rate of every compiled contracted configuration on the four grid
    configurations (the paper's Sec. 6.2 model-accuracy figure, per point): each plan timed on
    its full step count (CUDA events, best of 3 after one warm-up) beside the calibrated
    model's prediction for it."""
    torch, st = g.torch, g.st
    rows = []
    for name in ("diffusion2d_1024", "thermal2d_16384", "diffusion3d_512", "thermal3d_512x512x256"):
        w = WORKLOADS[name]()
        u0 = torch.from_numpy(w.u0).to(g.dev)
        pw = None if w.power is None else torch.from_numpy(w.power).to(g.dev)
        out = torch.empty_like(u0)
        confs = STUDY_2D if w.ndim == 2 else STUDY_3D
        if name == "diffusion2d_1024":
            confs = confs + [("resident",) + c for c in STUDY_RES]
        for cf in confs:
            if cf[0] == "resident":
                kw = dict(force_T=cf[1], force_vec=cf[2], resident=1)
            elif w.ndim == 2:
                T, vec, inplace = cf
                kw = dict(force_T=T, force_vec=vec, partial_rows=1 if inplace else 2)
            else:
                T, bx, by, vec = cf
                kw = dict(force_T=T, force_bx=bx, force_by=by, force_vec=vec)
            try:
                plan = st.Plan(w.kind, w.ndim, w.nx, w.ny, w.nz, stream=g.stream.cuda_stream, **kw)
            except st.StencilError:
                continue
            info = plan.info()
            plan.run(u0, out, w.coef, w.steps, power=pw)
            best = 1e30
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(g.stream)
                plan.run(u0, out, w.coef, w.steps, power=pw)
                e1.record(g.stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            meas = w.cells * w.steps / (best * 1e-3) / 1e9
            model = info["model_gcells"] or None
            rows.append({"workload": name, "config": list(cf), "measured_gcells": meas,
                         "model_gcells": model, "accuracy": meas / model if model else None,
                         "warps": info["warps"], "ctas": info["ctas"]})
            plan.close()
        del u0, pw, out
        torch.cuda.empty_cache()
    return rows


def headline_line(args, world, rec, extra=None):
    """The contract's top-level keys from a measurement record."""
    line = {"metric": METRIC, "value": rec["value"], "unit": rec["unit"], "n_gpus": world,
            "steps": rec["steps"], "warmup": rec["warmup"], "ms_per_step": rec["ms_per_step"],
            "median_ms_per_step": rec["median_ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    for k, v in rec.items():
        if not k.startswith("_") and k not in line:
            line[k] = v
    if world > 1:
        line["config"] = dict(line["config"], parallelism=f"replicas{world}")
    if extra:
        line.update(extra)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS) + [BATCH, ADJOINT],
                    help="measure this workload alone (default: the headline workload with "
                         "every other configuration as a sub-record)")
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--T", type=int, default=0, help="force the fused step count")
    ap.add_argument("--bx", type=int, default=0, help="force the 2D tile width")
    ap.add_argument("--vec", type=int, default=0, help="force cells per thread along x")
    ap.add_argument("--by", type=int, default=0, help="force the 3D tile height")
    ap.add_argument("--rows", type=int, default=0,
                    help="2D streaming kernels: 1 partial rows in place, 2 two-row (0: choose)")
    ap.add_argument("--resident", type=int, default=0,
                    help="2D: 1 resident tiles, -1 never (0: the plan chooses)")
    ap.add_argument("--storage", type=int, default=0, help="grid storage: 0 float32, 1 bf16, 2 fp16")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baselines")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-lowp", action="store_true", help="skip the bf16/fp16 storage runs")
    ap.add_argument("--no-configs", action="store_true", help="headline workload only")
    ap.add_argument("--nx", type=int, default=0, help="profiling: override the grid size")
    ap.add_argument("--ny", type=int, default=0)
    ap.add_argument("--nz", type=int, default=0)
    ap.add_argument("--time-steps", type=int, default=0, help="profiling: override time steps")
    ap.add_argument("--model-study", action="store_true",
                    help="measured / predicted rate of every compiled configuration (one JSON "
                         "line), the model-accuracy study")
    ap.add_argument("--tune", type=int, default=0,
                    help="before timing, run the model's top-K configurations on the workload and "
                         "use the fastest (stencil_tune); 0 = the model's own choice")
    args = ap.parse_args()
    single = args.workload is not None
    name = args.workload or DEFAULT

    if args.impl == "reference":
        if not reference_rank_gate():
            return
        if name == BATCH:
            ws = synth.c5a_batch()
            cpu = batch_reference(args, ws)
            v = cpu["value"]
            print(json.dumps({"impl": "reference", "metric": METRIC, "value": v,
                              "unit": "GCell/s", "n_gpus": args.gpus, "steps": args.steps,
                              "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
                              "data": "synthetic", "config": {"workload": BATCH},
                              "cpu_baseline": cpu,
                              "e2e": {"value": v, "unit": "GCell/s", "h2d_bytes_per_step": 0,
                                      "d2h_bytes_per_step": 0}}), flush=True)
            return
        if name == ADJOINT:
            w = synth.c5b_adjoint2d()
            cpu = adjoint_reference(args.steps, 20, (w.seed, w.kind))
            print(json.dumps({"impl": "reference", "metric": METRIC, "value": cpu["value"],
                              "unit": "GCell/s", "n_gpus": args.gpus, "steps": args.steps,
                              "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
                              "data": "synthetic", "config": {"workload": ADJOINT},
                              "cpu_baseline": cpu,
                              "e2e": {"value": cpu["value"], "unit": "GCell/s",
                                      "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
                  flush=True)
            return
        return run_reference(args, WORKLOADS[name]())

    g = Gpu()
    rk = g.rk
    with_cpu = not args.no_cpu
    if args.model_study:
        rows = model_study(g, args)
        if rk.rank == 0:
            print(json.dumps({"model_study": rows}), flush=True)
        return
    if name == BATCH:
        rec = batch_record(g, args, args.steps, args.warmup, with_cpu)
        if rk.rank == 0:
            print(json.dumps(headline_line(args, rk.world, rec)), flush=True)
        return
    if name == ADJOINT:
        rec = adjoint_record(g, args, args.steps, args.warmup, with_cpu)
        if rk.rank == 0:
            print(json.dumps(headline_line(args, rk.world, rec)), flush=True)
        return

    w = WORKLOADS[name]()
    resized = bool(args.nx or args.ny or args.nz or args.time_steps)
    if resized and w.var:
        w = synth.make_vdiff(args.nx or w.nx, args.ny or w.ny, steps=args.time_steps or w.steps,
                             seed=w.seed, name=f"{w.name.split('_')[0]}_resized")
    elif resized and w.rad > 1:
        w = synth.make_star(w.ndim, w.rad, args.nx or w.nx, args.ny or w.ny, args.nz or w.nz,
                            steps=args.time_steps or w.steps, seed=w.seed,
                            name=f"{w.name.split('_')[0]}_resized")
    elif resized:
        w = synth.make(w.kind, w.ndim, args.nx or w.nx, args.ny or w.ny, args.nz or w.nz,
                       steps=args.time_steps or w.steps, seed=w.seed,
                       name=f"{w.name.split('_')[0]}_resized")

    rec = plan_record(g, w, args, args.steps, args.warmup, with_cpu, key=name)
    extra = {}
    default_run = not single and not resized and not (args.T or args.bx or args.vec or args.by
                                                      or args.storage)
    if w.ndim == 2 and w.rad <= 1 and not w.var and not resized and not args.no_lowp \
            and not args.storage:
        extra["lowp"] = lowp_record(g, w, args, rec["value"], rec["_bufs"],
                                    max(3, min(args.steps, 10)), 2,
                                    with_err=with_cpu and rk.world == 1 and default_run)
    rec["_plan"].close()
    del rec["_bufs"]
    g.torch.cuda.empty_cache()
    if default_run:
        extra["fp32_peak_measured_tflops"] = g.st.stencil_fp32_peak(g.stream.cuda_stream)
        if not args.no_configs:
            sub = {}
            k = max(3, min(args.steps, 10))
            for cname in SUBCONFIGS:
                if cname == BATCH:
                    r = batch_record(g, args, k, 3, with_cpu)
                elif cname == ADJOINT:
                    r = adjoint_record(g, args, k, 3, with_cpu)
                else:
                    cw = WORKLOADS[cname]()
                    # the 1024^2 grid runs in well under a millisecond: enough calls that the
                    # timed region lasts about half a second, so that nvidia-smi (200 ms
                    # period) samples its clocks
                    kk = 4000 if cw.cells * cw.steps < 1e9 else k
                    r = plan_record(g, cw, args, kk, 3, with_cpu,
                                    one_thread=(cname == "diffusion2d_1024"), key=cname)
                    r["_plan"].close()
                    del r["_bufs"], r["_plan"]
                    g.torch.cuda.empty_cache()
                sub[cname] = r
            extra["configs"] = sub
    del rec["_plan"]
    if rk.rank == 0:
        print(json.dumps(headline_line(args, rk.world, rec, extra)), flush=True)
    if rk.dist:
        rk.dist.destroy_process_group()


if __name__ == "__main__":
    main()
