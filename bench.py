"""Benchmark of the temporally-blocked stencil engine on one configuration.

Default workload: Hotspot 2D (thermal), 16384 x 16384 float32 cells, 1000 time steps, seeded
synthetic inputs (temperature U[320,340) K, power U[0,0.5), ambient 80).  One benchmark "step"
is one full run of the hot path: stencil_run advancing the grid by 1000 time steps
(ceil(1000/T) temporally-blocked passes).

Prints one JSON line (rank 0): throughput in GCell/s (cell updates per second, the unit the
paper's Table 4 quotes beside GB/s and GFLOP/s), the dominant kernel's roofline fraction, the
end-to-end figure through the C ABI with host buffers, and the CPU oracle's throughput on a
bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

With --gpus N > 1 (launched by torch.distributed.run) every rank advances its own grid: the
method has no cross-grid exchange, so the job is N independent replicas (weak scaling) with a
barrier around the timed region and the time taken as the maximum over ranks.
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


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    """FP32 ALU peak: SMs x 128 FP32 lanes x 2 flops per fused multiply-add x clock."""
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


def kernel_source_hash(ndim: int) -> str:
    """Hash of the sources of the benchmarked kernel family (2D contracted or 3D)."""
    files = (("tb2f_kernel.cuh", "tb2d_kernel.cuh", "common.cuh") if ndim == 2
             else ("tb3f_kernel.cuh", "tb3d_kernel.cuh", "common.cuh"))
    h = hashlib.sha1()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1802_00438_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(workload: str, ndim: int):
    """DRAM bytes per launch recorded from an ncu capture of the current kernel source
    (profiles/traffic.txt); None when the kernel changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == workload:
            return float(f[2]) if f[1] == kernel_source_hash(ndim) else None
    return None


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


def _oracle_sample_steps(w, budget_s: float):
    """Time steps of the full grid that take about budget_s seconds on the host cores (from
    the difference of a 1-step and a 3-step run, so set-up costs do not count)."""
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    t = []
    for s in (1, 3):
        t0 = time.perf_counter()
        _oracle_run(w, s)
        t.append(time.perf_counter() - t0)
    per_step = max((t[1] - t[0]) / 2, 1e-5)
    return max(1, min(w.steps, int(budget_s / per_step))), cores


def cpu_baseline(w, budget_s: float = 15.0):
    """The oracle as it stands, on the host cores, over a bounded sample of the workload: the
    full grid for as many time steps as fit in about `budget_s` seconds."""
    import oracle
    steps, cores = _oracle_sample_steps(w, budget_s)
    t0 = time.perf_counter()
    _oracle_run(w, steps)
    t = time.perf_counter() - t0
    return {"value": w.cells * steps / t / 1e9, "unit": "GCell/s", "cores": cores,
            "kind": "oracle",
            "sample": f"full {'x'.join(map(str, w.shape[::-1]))} grid, {steps} of {w.steps} "
                      f"time steps ({t:.1f} s; float32 oracle, OpenMP over rows)"}


def lowp_errors(w, st, stream, side=2048):
    """Relative L2 / L-inf error after the full step count, float32 / bf16 / fp16 storage, vs
    the float64 oracle, on a side x side grid of the same workload (seeded like it)."""
    import torch
    import oracle
    ws = synth.make(w.kind, 2, min(side, w.nx), min(side, w.ny), steps=w.steps, seed=w.seed)
    ref = oracle.run(ws.kind, ws.u0, ws.coef, ws.steps, ws.power, dtype=np.float64)
    u = torch.from_numpy(ws.u0).cuda()
    p = None if ws.power is None else torch.from_numpy(ws.power).cuda()
    res = {"grid": f"{ws.nx}x{ws.ny}", "time_steps": ws.steps}
    for name, stor in (("f32", st.ST_F32), ("bf16", st.ST_BF16), ("fp16", st.ST_F16)):
        o = torch.empty_like(u)
        pl = st.Plan(ws.kind, 2, ws.nx, ws.ny, storage=stor, stream=stream.cuda_stream)
        pl.run(u, o, ws.coef, ws.steps, power=p)
        pl.sync()
        pl.close()
        g = o.cpu().numpy().astype(np.float64)
        d = g - ref
        res[name] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
                     "rel_linf": float(np.abs(d).max() / np.abs(ref).max())}
    return res


def run_reference(args, w):
    """Reference arm: the CPU oracle, each benchmark step a bounded sample of the workload."""
    import oracle
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
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
    line = {"impl": "reference", "metric": "stencil GCell/s & GFLOP/s vs roofline",
            "value": value, "unit": "GCell/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name},
            "cpu_baseline": {"value": value, "unit": "GCell/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GCell/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batch(args):
    """64 grids (sides log-uniform in [256, 4096], steps uniform in {50..500}, kinds
    alternating): one step = one replay of the batch's CUDA graph."""
    ws = synth.c5a_batch()
    cells_steps = sum(w.cells * w.steps for w in ws)
    if args.impl == "reference":
        import oracle
        oracle.build()
        cores = len(os.sched_getaffinity(0))
        oracle.set_threads(cores)
        frac = 1.0 / 40          # each grid for 1/40 of its steps (at least one)
        t0 = time.perf_counter()
        done = 0
        for _ in range(args.steps):
            for w in ws:
                s = max(1, int(w.steps * frac))
                oracle.run(w.kind, w.u0, w.coef, s, w.power)
                done += w.cells * s
        t = time.perf_counter() - t0
        v = done / t / 1e9
        print(json.dumps({"impl": "reference", "metric": "stencil GCell/s & GFLOP/s vs roofline",
                          "value": v, "unit": "GCell/s", "n_gpus": args.gpus, "steps": args.steps,
                          "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
                          "data": "synthetic", "config": {"workload": BATCH},
                          "cpu_baseline": {"value": v, "unit": "GCell/s", "cores": cores,
                                           "kind": "oracle",
                                           "sample": "all 64 grids, 1/40 of each grid's steps"},
                          "e2e": {"value": v, "unit": "GCell/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    import torch
    import paper_1802_00438_gb300 as st
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rk = Replicas("nccl", dev)
    world, rank = rk.world, rk.rank
    stream = torch.cuda.Stream(dev)
    items = []
    for w in ws:
        u = torch.from_numpy(w.u0).to(dev)
        o = torch.empty_like(u)
        p = None if w.power is None else torch.from_numpy(w.power).to(dev)
        items.append({"kind": w.kind, "nx": w.nx, "ny": w.ny, "steps": w.steps, "grid_in": u,
                      "grid_out": o, "power": p, "coeffs": w.coef})
    torch.cuda.synchronize()
    b = st.Batch(items, stream=stream.cuda_stream)
    for _ in range(args.warmup):
        b.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rk.barrier()
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            b.run()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = rk.max_ms(e0.elapsed_time(e1))
    value = rk.job_rate(cells_steps * args.steps, ms) / 1e9
    # roofline of the mix: sum over grids of cells*steps / R_g(T_g), R = min(ALU, HBM*T/bytes)
    peaks, src = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu = fp32_peak_tflops(sms, float(peaks.get("sm_max_mhz", 2070.0))) * 1e12
    hbm = float(peaks["hbm_gbs"]) * 1e9
    ideal = 0.0
    bytes_moved = 0.0
    for i, w in enumerate(ws):
        gi = b.grid_info(i)
        R = min(alu / FLOPS[(w.kind, 2)], hbm * gi["T"] / BYTES[w.kind])
        ideal += w.cells * w.steps / R
        bytes_moved += w.cells * BYTES[w.kind] * gi["passes"]
    per_step_s = ms * 1e-3 / args.steps
    gbs = bytes_moved / per_step_s / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
            "frac": gbs / float(peaks["hbm_gbs"]), "traffic": None,
            "frac_of_cell_roofline": ideal / per_step_s,
            "note": "mix of 64 grids: achieved = algorithmic bytes of all passes / step time; "
                    "frac_of_cell_roofline = sum_g cells*steps/R_g(T_g) / step time"}
    # end to end: host inputs in, results out, through the same batch
    h_in = [torch.from_numpy(w.u0).pin_memory() for w in ws]
    h_out = [torch.empty_like(h).pin_memory() for h in h_in]
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    rk.barrier()
    with torch.cuda.stream(stream):
        a0.record(stream)
        for _ in range(args.steps):
            for it, h in zip(items, h_in):
                it["grid_in"].copy_(h, non_blocking=True)
            b.run()
            for it, h in zip(items, h_out):
                h.copy_(it["grid_out"], non_blocking=True)
        a1.record(stream)
    torch.cuda.synchronize()
    ems = rk.max_ms(a0.elapsed_time(a1))
    nb = sum(w.u0.nbytes for w in ws)
    e2e = {"value": rk.job_rate(cells_steps * args.steps, ems) / 1e9, "unit": "GCell/s",
           "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}
    if rank == 0:
        tv = {}
        for i in range(len(ws)):
            gi = b.grid_info(i)
            k = f"T{gi['T']}V{gi['vec']}"
            tv[k] = tv.get(k, 0) + 1
        print(json.dumps({"metric": "stencil GCell/s & GFLOP/s vs roofline", "value": value,
                          "unit": "GCell/s", "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f32", "data": "synthetic",
                          "config": {"workload": BATCH, "grids": len(ws),
                                     "cell_updates_per_step": cells_steps,
                                     "graph_launches_per_step": b.launches(), "per_grid_T_V": tv,
                                     "l2": "inputs larger than L2 in total (%.0f MiB)" % (nb / 2**20)},
                          "roofline": roof, "e2e": e2e, "gpu_launches": b.launches() * args.steps,
                          "clocks": clk.summary(), "cpu_baseline": None}), flush=True)
    b.close()
    if rk.dist:
        rk.dist.destroy_process_group()


def bench_adjoint(args, ckpt=20):
    """Gradient of L = sum(w * u_200) for a 2048^2 diffusion run: one step = the checkpointed
    forward run plus the backward sweep (state recompute, transposed passes, reductions).
    value = primal cell updates (cells x 200) per second of a whole gradient evaluation."""
    w = synth.c5b_adjoint2d()
    wt = synth.loss_weights(6, w.shape)
    n = w.cells
    # the oracle's timing: the reference arm, or the CPU baseline (rank 0 of a 1-GPU run only)
    if args.impl == "reference" or (not args.no_cpu and int(os.environ.get("WORLD_SIZE", "1")) == 1):
        import oracle
        oracle.build()
        cores = len(os.sched_getaffinity(0))
        oracle.set_threads(cores)
        side, s = 512, 20   # bounded sample: a 512^2, 20-step gradient (checkpoints every 20)
        ws = synth.make(w.kind, 2, side, side, 1, s, seed=w.seed)
        wts = synth.loss_weights(6, ws.shape)
        reps = args.steps if args.impl == "reference" else 1
        t0 = time.perf_counter()
        for _ in range(reps):
            oracle.adjoint2d(ws.kind, ws.u0, ws.coef, s, wts, None, ckpt=ckpt)
        t = (time.perf_counter() - t0) / reps
        cpu = {"value": side * side * s / t / 1e9, "unit": "GCell/s", "cores": cores,
               "kind": "oracle", "sample": f"float64 adjoint of a {side}^2, {s}-step diffusion "
                                             f"run (the transposed sweep is one thread)"}
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "metric": "stencil GCell/s & GFLOP/s vs roofline",
                              "value": cpu["value"], "unit": "GCell/s", "n_gpus": args.gpus,
                              "steps": args.steps, "warmup": args.warmup,
                              "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                              "config": {"workload": ADJOINT}, "cpu_baseline": cpu,
                              "e2e": {"value": cpu["value"], "unit": "GCell/s",
                                      "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
                  flush=True)
            return
    else:
        cpu = None
    import torch
    import paper_1802_00438_gb300 as st
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rk = Replicas("nccl", dev)
    world, rank = rk.world, rk.rank
    stream = torch.cuda.current_stream(dev)
    u0 = torch.from_numpy(w.u0).to(dev)
    g = torch.from_numpy(wt).to(dev)
    adj = st.Adjoint(w.kind, w.nx, w.ny, w.steps, ckpt, stream=stream.cuda_stream)
    out = torch.empty_like(u0)
    gu = torch.empty_like(u0)
    gk = torch.empty(5, dtype=torch.float32, device=dev)

    def step():
        st.stencil_adjoint_forward(adj.h, u0, None, w.coef, out)
        st.stencil_adjoint_backward(adj.h, g, None, gu, gk, None, None)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    rk.barrier()
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        # forward alone, for the split
        e0b = torch.cuda.Event(enable_timing=True)
        e0b.record(stream)
        for _ in range(args.steps):
            st.stencil_adjoint_forward(adj.h, u0, None, w.coef, out)
        f1.record(stream)
        torch.cuda.synchronize()
    ms = rk.max_ms(e0.elapsed_time(e1))
    fms = rk.max_ms(e0b.elapsed_time(f1))
    per = ms / args.steps
    bwd = per - fms / args.steps
    value = rk.job_rate(n * w.steps * args.steps, ms) / 1e9
    # algorithmic HBM bytes of the backward: per transposed pass of s steps lambda in + out
    # (8 B) and the s states (4 B each); per segment the checkpoint copy into the state buffer
    # (8 B) and one trajectory run that reads it and writes the L-1 recomputed states (4 B
    # each); grad_u0 copy (8 B)
    nseg = -(-w.steps // ckpt)
    seg_len = [min(w.steps, (k + 1) * ckpt) - k * ckpt for k in range(nseg)]
    bytes_b = 0
    for L in seg_len:
        bytes_b += n * (4 * (L - 1) + 4 + 8)   # trajectory: read u_t0, write L-1 states; copy
        left = L
        while left > 0:
            s = min(4, left)
            bytes_b += n * (8 + 4 * s)
            left -= s
    bytes_b += 8 * n
    peaks, src = load_peaks()
    gbs = bytes_b / (bwd * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
            "frac": gbs / float(peaks["hbm_gbs"]), "traffic": None,
            "note": "whole backward (state recompute + transposed passes): algorithmic bytes / "
                    "backward time (step time minus the checkpointed forward run)"}
    # end to end: initial field and upstream gradient from pinned host memory, gradients back
    h_u = torch.from_numpy(w.u0).pin_memory()
    h_g = torch.from_numpy(wt).pin_memory()
    h_gu = torch.empty_like(h_u).pin_memory()
    h_gk = torch.empty(5, dtype=torch.float32).pin_memory()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    rk.barrier()
    a0.record(stream)
    for _ in range(args.steps):
        u0.copy_(h_u, non_blocking=True)
        g.copy_(h_g, non_blocking=True)
        step()
        h_gu.copy_(gu, non_blocking=True)
        h_gk.copy_(gk, non_blocking=True)
    a1.record(stream)
    torch.cuda.synchronize()
    ems = rk.max_ms(a0.elapsed_time(a1))
    e2e = {"value": rk.job_rate(n * w.steps * args.steps, ems) / 1e9, "unit": "GCell/s",
           "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 * n + 20}
    fwd_T = st.Plan(w.kind, 2, w.nx, w.ny).info()["T"]
    launches = sum(-(-L // fwd_T) for L in seg_len)            # forward passes
    launches += sum(-(-(L - 1) // 8) for L in seg_len)           # trajectory passes
    launches += sum(-(-L // 4) for L in seg_len) + 2             # transposed passes + 2-level sum
    if rank == 0:
        print(json.dumps({"metric": "stencil GCell/s & GFLOP/s vs roofline", "value": value,
                          "unit": "GCell/s", "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": per, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                          "data": "synthetic",
                          "config": {"workload": ADJOINT, "grid": f"{w.nx}x{w.ny}",
                                     "time_steps": w.steps, "checkpoint_every": ckpt,
                                     "forward_ms": fms / args.steps, "backward_ms": bwd,
                                     "l2": "inputs larger than L2 (200-state sweep over 16 MiB "
                                           "grids; 496 MiB of buffers)"},
                          "roofline": roof, "e2e": e2e, "gpu_launches": launches * args.steps,
                          "clocks": clk.summary(), "cpu_baseline": cpu}), flush=True)
    adj.close()
    if rk.dist:
        rk.dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + [BATCH, ADJOINT])
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--T", type=int, default=0, help="force the fused step count")
    ap.add_argument("--bx", type=int, default=0, help="force the 2D tile width")
    ap.add_argument("--vec", type=int, default=0, help="force cells per thread along x")
    ap.add_argument("--by", type=int, default=0, help="force the 3D tile height (2D: kernel variant)")
    ap.add_argument("--storage", type=int, default=0, help="grid storage: 0 float32, 1 bf16, 2 fp16")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-lowp", action="store_true", help="skip the bf16/fp16 storage runs")
    ap.add_argument("--nx", type=int, default=0, help="profiling: override the grid size")
    ap.add_argument("--ny", type=int, default=0)
    ap.add_argument("--nz", type=int, default=0)
    ap.add_argument("--time-steps", type=int, default=0, help="profiling: override time steps")
    ap.add_argument("--tune", type=int, default=0,
                    help="before timing, run the model's top-K configurations on the workload and "
                         "use the fastest (stencil_tune); 0 = the model's own choice")
    args = ap.parse_args()

    if args.impl == "reference" and not reference_rank_gate():
        return
    if args.workload == BATCH:
        return bench_batch(args)
    if args.workload == ADJOINT:
        return bench_adjoint(args)
    w = WORKLOADS[args.workload]()
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
    if args.impl == "reference":
        return run_reference(args, w)

    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rk = Replicas("nccl", dev)
    world, rank = rk.world, rk.rank

    import paper_1802_00438_gb300 as st

    stream = torch.cuda.current_stream(dev)
    u0 = torch.from_numpy(w.u0).to(dev)
    # the per-cell input: the power map, or the five coefficient planes of ST_DIFFUSION_VAR
    kind = st.ST_DIFFUSION_VAR if w.var else w.kind
    h_pin = w.coef if w.var else w.power
    pw = None if h_pin is None else torch.from_numpy(h_pin).to(dev)
    coef = None if w.var else w.coef
    out = torch.empty_like(u0)
    tuned = None
    if args.tune > 0:
        tuned = st.stencil_tune(kind, w.ndim, w.nx, w.ny, w.nz, u0, out, coef, w.steps, pw,
                                top_k=args.tune, storage=args.storage, stream=stream.cuda_stream,
                                rad=w.rad if w.rad > 1 else 0)
    plan = st.Plan(kind, w.ndim, w.nx, w.ny, w.nz, force_T=args.T, force_bx=args.bx,
                   force_vec=args.vec, force_by=args.by, storage=args.storage,
                   stream=stream.cuda_stream, rad=w.rad if w.rad > 1 else 0)
    info = plan.info()
    T = info["T"]
    passes = -(-w.steps // T)

    def step():
        plan.run(u0, out, coef, w.steps, power=pw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, device time by CUDA events on the plan's stream ----------
    st.stencil_plan_set_timing(plan.h, True)
    st.stencil_plan_kernel_time(plan.h, reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    rk.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    rk.barrier()
    ms = rk.max_ms(e0.elapsed_time(e1))
    kern_ms, timed_launches = st.stencil_plan_kernel_time(plan.h, reset=True)
    launches = timed_launches
    if w.kind == 1 and w.ndim == 2 and not args.storage:
        launches += args.steps   # the source-map kernel (p + amb*Rz) before each run's passes
    st.stencil_plan_set_timing(plan.h, False)
    cells_step = w.cells * w.steps
    value = rk.job_rate(cells_step * args.steps, ms) / 1e9

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

        e2e_step()
        torch.cuda.synchronize()
        rk.barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        a1.record(stream)
        torch.cuda.synchronize()
        ems = rk.max_ms(a0.elapsed_time(a1))
        nb = w.u0.nbytes
        e2e = {"value": rk.job_rate(cells_step * args.steps, ems) / 1e9, "unit": "GCell/s",
               "h2d_bytes_per_step": nb + (0 if h_pin is None else h_pin.nbytes),
               "d2h_bytes_per_step": nb}

    # ---- roofline of the dominant kernel ---------------------------------------------------
    peaks, src = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fl = _flops(w)
    by = BYTES_VAR if w.var else BYTES[w.kind]
    alu_peak = fp32_peak_tflops(sms, mhz)
    hbm_peak = float(peaks["hbm_gbs"])
    avg_launch_ms = kern_ms / max(timed_launches, 1)
    # algorithmic work of one launch, averaged over the timed launches (the last pass of a
    # run fuses the remainder of the steps)
    flops_per_launch = w.cells * w.steps * args.steps * fl / max(timed_launches, 1)
    bytes_per_launch = w.cells * by
    tflops = flops_per_launch / (avg_launch_ms * 1e-3) / 1e12
    gbs = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
    cell_roof = min(alu_peak * 1e12 / fl, hbm_peak * 1e9 * T / by)      # cells/s at this T
    alu_bound = alu_peak * 1e12 / fl <= hbm_peak * 1e9 * T / by
    traffic = None if (resized or args.T or args.bx or args.vec or args.by) else \
        profiled_traffic(args.workload, w.ndim)
    if alu_bound:
        roof = {"bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": tflops / alu_peak,
                "peak_note": f"FP32 {sms} SMs x 128 lanes x 2 x {mhz:.0f} MHz (max SM clock)"}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak, "peak_note": f"{src} copy bandwidth"}
    roof["traffic"] = traffic
    roof["algorithmic_bytes_per_launch"] = bytes_per_launch
    roof["cell_roofline_gcells"] = cell_roof / 1e9
    roof["frac_of_cell_roofline"] = (cells_step * args.steps / (kern_ms * 1e-3)) / cell_roof
    roof["hbm_frac"] = gbs / hbm_peak
    # the T -> infinity ceiling: FP32 issue of the counted flops alone
    roof["fp32_ceiling_gcells"] = alu_peak * 1e3 / fl
    roof["frac_of_fp32_ceiling"] = (cells_step * args.steps / (kern_ms * 1e-3)) / (alu_peak * 1e12 / fl)
    roof["kernel_ms_per_launch"] = avg_launch_ms

    clocks = clk.summary()

    # ---- 16-bit storage: speed on the same workload, error vs the float64 oracle ------------
    lowp = None
    if w.ndim == 2 and w.rad <= 1 and not w.var and not resized and not args.no_lowp and not args.storage:
        lowp = {}
        for name, stor in (("bf16", st.ST_BF16), ("fp16", st.ST_F16)):
            qplan = st.Plan(w.kind, 2, w.nx, w.ny, storage=stor, stream=stream.cuda_stream)
            for _ in range(2):
                qplan.run(u0, out, w.coef, w.steps, power=pw)
            torch.cuda.synchronize()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            rk.barrier()
            q0.record(stream)
            for _ in range(args.steps):
                qplan.run(u0, out, w.coef, w.steps, power=pw)
            q1.record(stream)
            torch.cuda.synchronize()
            qms = rk.max_ms(q0.elapsed_time(q1))
            qv = rk.job_rate(cells_step * args.steps, qms) / 1e9
            lowp[name] = {"value": qv, "unit": "GCell/s", "speedup_vs_f32": qv / value,
                          "T": qplan.info()["T"]}
            qplan.close()
        if not args.no_cpu and world == 1:
            lowp["error_vs_f64_oracle"] = lowp_errors(w, st, stream)

    rk.barrier()
    if rank == 0:
        line = {"metric": "stencil GCell/s & GFLOP/s vs roofline",
                "value": value, "unit": "GCell/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "gflops": value * fl, "effective_gbs": value * by,
                "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz,
                           "time_steps": w.steps, "T": T, "tile": [info["bx"], info["by"]],
                           "vec": info["vec"], "warps": info["warps"], "ctas": info["ctas"],
                           "passes_per_step": passes,
                           # the library's calibrated restatement of Eqs. 3-9 for this plan,
                           # and measured / predicted (the paper's model-accuracy figure)
                           "model_gcells": info["model_gcells"] or None,
                           "model_accuracy": (value / world / info["model_gcells"]
                                              if info["model_gcells"] else None),
                           "l2": "inputs larger than L2 (%.0f MiB per grid)" % (w.u0.nbytes / 2**20),
                           "parallelism": f"replicas{world}" if world > 1 else "single",
                           "tuned": tuned},
                "roofline": roof, "e2e": e2e, "lowp": lowp,
                "gpu_launches": launches, "clocks": clocks}
        if not args.no_cpu and world == 1:
            line["cpu_baseline"] = cpu_baseline(w)
        else:
            line["cpu_baseline"] = None
        print(json.dumps(line), flush=True)
    plan.close()
    if rk.dist:
        rk.dist.destroy_process_group()


if __name__ == "__main__":
    main()
