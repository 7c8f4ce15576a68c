#!/usr/bin/env python
"""Benchmark of the DG wall-model hot path on one GB300 (or N replicas under torchrun).

One step = one pass of the FP64 operator-apply path over the workload (the Q4 32x24x24 channel
by default, plain FP64): the eddy-viscosity update of the enriched cells, then FP64 applies of the
SIPG Laplacian, the velocity divergence, the convective and the viscous operator.

value = output DoFs of the step's four FP64 applies (n_p + n_p + n_u + n_u) / step time, in GDoF/s
(every unit counted is an FP64 operator application; nothing of the solves is in it). The e2e key
measures the same step through the public API with host buffers: pinned uploads of u and p and
read-backs of the four results inside the timed region, on their own streams so that they overlap the
applies (the Laplacian starts once p has arrived, each result is read back as soon as it is done).

The same run then times, each in its own loop, the pressure solves to a 1e-10 relative residual in
plain FP64 (FP64 CG + FP64 multigrid) and mixed precision (FP64 refinement around FP32 CG with the
FP32 multigrid), on this workload (rhs = the step's divergence) and on the Q3 64x32x32 channel
(seeded zero-mean uniform rhs), reported as solves/s under "solves"; the FP32 SIPG Laplacian,
the operator the FP32 multigrid applies most, with its HBM roofline under "fp32_laplace"; the same
step with every apply in double-float arithmetic under "df64_step"; and a short serving stream
(Poisson arrivals of solve and apply jobs on channels of different sizes and degrees through the
request loop with continuous batching, p50/p99 latency and solves/s against the same jobs run one at
a time with FP64 solves) under "serving".

--impl reference times the CPU oracle (the plain FP64 implementation the tests check against) on a
bounded sample of the same workload: the four operator applies on a subset of cells.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDoF/s per DG operator apply; pressure solves/s at 1e-10 (FP64 vs mixed)"
UNIT = "GDoF/s"
DEFAULT_WORKLOAD = "channel_q4_32x24x24"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # wait (at most 3 s) for the first sample so that the sampling covers the whole timed region
        t0 = time.time()
        while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0 and self.proc.poll() is None:
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_time(ms_local: float, world: int, device=None) -> float:
    """Step time of the job: the maximum over ranks of each replica's mean step time (every rank runs
    the same workload on its own GPU: weak scaling, no data-path collective)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(units_per_replica: float, world: int, ms_max: float) -> float:
    """Whole-job throughput in G units/s: all replicas' units over the slowest replica's time."""
    return world * units_per_replica / (ms_max * 1e-3) / 1e9


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ------------------------------------------------------------------------------------------------

def oracle_sample(w, target_s=12.0, max_cells=None):
    """Time the oracle's four operator applies on a bounded sample of the workload's cells.
    Returns (GDoF/s, seconds, threads, description)."""
    import numpy as np
    import oracle as O
    from paper_1705_08813_gb300 import inputs as I
    threads = os.cpu_count() or 1
    O.set_threads(threads)
    om = O.Mesh(**w.mesh_kwargs())
    u = I.workload_velocity(om.node_coords(), om.n_e, w)
    p = I.pressure_field(om.n_p, w.seed)
    n1 = w.k + 1
    # pick cells spread over the mesh, including wall cells, growing until the time budget is used
    ncell = 16
    order = np.random.default_rng(w.seed).permutation(om.nc)
    elapsed, dofs = 0.0, 0.0
    while True:
        cells = order[:ncell]
        om.set_active(cells)
        n_enr = int(sum(1 for c in cells if ((c // w.nx) % w.ny) in (0, w.ny - 1)))
        t0 = time.perf_counter()
        om.laplace(p)
        om.divergence(u)
        om.convective(u)
        om.viscous(u, u)
        dt = time.perf_counter() - t0
        d = len(cells) * n1 ** 3 * (1 + 1 + 3 + 3) + n_enr * 24 * 2
        elapsed, dofs = dt, d
        if dt * 2.0 > target_s or ncell >= om.nc or (max_cells and ncell >= max_cells):
            break
        ncell = min(om.nc, ncell * 2)
    om.set_active(None)
    desc = (f"{len(cells)} of {om.nc} cells ({n_enr} enriched): Laplace, divergence, convective and "
            f"viscous applies of the oracle on those cells' outputs, {threads} threads")
    return dofs / elapsed / 1e9, elapsed, threads, desc


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    from paper_1705_08813_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]
    import oracle as O
    O.build()
    for _ in range(args.warmup):
        oracle_sample(w, target_s=2.0, max_cells=64)
    vals, secs = [], []
    # each step is a bounded sample; the whole run stays within a few minutes
    per_step = min(args.ref_seconds, max(1.0, 150.0 / max(1, args.steps)))
    for _ in range(args.steps):
        v, s, threads, desc = oracle_sample(w, target_s=per_step)
        vals.append(v)
        secs.append(s)
    val = statistics.mean(vals)
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w.name, "cells": [w.nx, w.ny, w.nz], "degree": w.k, "re_tau": w.re_tau},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------

def laplace_flops_per_cell(k, curved=False):
    """Floating-point operations of one cell of the Laplace kernel (2 flops per FMA), counted from
    its passes with n = k + 1.
    Boxes (laplace_box_kernel): neighbour trace derivatives 6n^3; x-lines 2n^4 + 4n^3; M_x on the
    y- and z-face traces 8n^3; y-lines 3n^4 + 4n^3; M_y on the z-face traces 4n^3; z-lines
    2n^4 + 4n^3.
    Curved cells (vector_op_kernel, OP_LAP): reference gradient at the points and back 16n^4; metric
    products 21n^3; per face direction (both faces, both sides) normal derivatives 4n^3, tangential
    passes 28n^3, integration 14n^3, scatter 2n^3 and about 40 per face point (2n^2 points)."""
    n = k + 1
    if curved:
        return 2 * (16 * n ** 4 + 21 * n ** 3 + 3 * (48 * n ** 3 + 80 * n ** 2))
    return 2 * (7 * n ** 4 + 30 * n ** 3)


def vector_flops_per_cell(op, k, curved=False):
    """Floating-point operations (2 per multiply-add) of one standard box cell of the divergence,
    convective and viscous operators, n = k + 1 nodes, counted for the algorithms the box kernels
    use. Every 1-D product of a volume pass uses the even-odd form: with P(a, b) the flops of one
    product from a inputs to b outputs (sums and differences of mirrored inputs, half-size products
    per mirrored pair of outputs, the middle row); a product scaled into an accumulator adds 2 b.
    The divergence and the viscous term have polynomial integrands that the k+1 Gauss points
    integrate exactly, so they are Kronecker products of 1-D n x n matrices on the nodes:
      divergence  n^2 (8 P(n, n) + 6 n) (volume: 8 line products, 3 of them scaled)
                  + 2 * 12 n^3 (faces: averages, two face-grid passes)
      viscous     3 n^2 (12 P(n, n) + 6 n) (volume: 12 line products per output component)
                  + 2 * 174 n^3 (faces: normal and tangential derivatives, two face-grid passes of
                  eight coefficient arrays, normal-derivative test terms) + 180 n^2 (coefficients)
    Curved cells (the general kernel) take plain 1-D products, P(a, b) = 2 a b: the counts above with
    that P and 2 n^3 per scaled line product, the metric terms not counted.
    The convective term is evaluated at q = floor(3k/2)+1 Gauss points (Sec. 4.4), its products
    (n nodes -> q points and back) in the same even-odd form:
      values (n^2 + q n + q^2) P(n, q) per component, integration (3 q^2 + 3 q n + 2 n^2) P(q, n)
      + (q n + n^2) n per output component, 9 q^3 for the products, and per face direction
      12 (n + q) P(n, q) (traces of both sides), 40 q^2 (flux), 6 (q + n) P(q, n) (integration back)."""
    n = k + 1

    def P(a, b):
        if curved:
            return 2 * a * b
        return 2 * (a // 2) + (b // 2) * (4 * (a // 2) + a % 2 + 2) + (b % 2) * (2 * (a // 2) + a % 2)
    sc = 0 if curved else 6 * n   # the scaling multiply-add of a scaled product (inside P when plain)
    if op == "divergence":
        return n * n * (8 * P(n, n) + sc) + 2 * 12 * n ** 3
    if op == "viscous":
        return 3 * n * n * (12 * P(n, n) + sc) + 2 * 174 * n ** 3 + 180 * n * n
    q = (3 * k) // 2 + 1
    fwd, bwd = P(n, q), P(q, n)
    acc = 0 if curved else (q * n + n * n) * n   # adds of the accumulated even-odd products
    vol = 3 * (n * n + q * n + q * q) * fwd + 3 * ((3 * q * q + 3 * q * n + 2 * n * n) * bwd + acc)
    faces = 3 * (12 * (n + q) * fwd + 6 * (q + n) * bwd)
    return vol + faces + 9 * q ** 3 + 3 * 40 * q * q


FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12    # 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 FMA/clk x 2 flops x 2.07 GHz


def _time_solves(m, b, p, modes, reps, flush):
    """solves/s of dgw_pressure_solve per mode (median host time of `reps` solves after one
    untimed solve that builds the hierarchy; L2 flushed before each)."""
    import torch
    out = {}
    for name, mode in modes:
        m.pressure_solve(b, p, rtol=1e-10, max_iter=500, mode=mode)
        ts, its, res = [], [], []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = m.pressure_solve(b, p, rtol=1e-10, max_iter=500, mode=mode)
            ts.append(time.perf_counter() - t0)
            its.append(info["iterations"])
            res.append(info["rel_residual"])
        out[name] = {"solves_per_s": 1.0 / statistics.median(ts), "ms": 1e3 * statistics.median(ts),
                     "iterations": statistics.mean(its), "rel_residual": max(res)}
    out["mixed_over_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    return out


def _time_block_solves(m, b, ncols, reps, flush):
    """solves/s of one block solve of ncols right-hand sides (dgw_pressure_solve_batch; the columns
    are b scaled by 1..ncols, so every column runs the same iterations as b alone)."""
    import torch
    from paper_1705_08813_gb300 import dgw
    bs = [b * (c + 1) for c in range(ncols)]
    ps = [torch.zeros_like(b) for _ in range(ncols)]
    dgw.pressure_solve_batch(m, bs, ps, rtol=1e-10, max_iter=500)
    ts, infos = [], None
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = dgw.pressure_solve_batch(m, bs, ps, rtol=1e-10, max_iter=500)
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    return {"columns": ncols, "solves_per_s": ncols / t, "ms": 1e3 * t,
            "iterations": max(i["iterations"] for i in infos), "rel_residual": max(i["rel_residual"] for i in infos)}


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1705_08813_gb300 import dgw, inputs as I

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = I.WORKLOADS[args.workload]
    dgw.load()
    m = dgw.mesh_for(w)
    nodes = m.node_coords()
    u_host = torch.from_numpy(I.workload_velocity(nodes, m.n_e, w)).pin_memory()
    p_host = torch.from_numpy(I.pressure_field(m.n_p, w.seed)).pin_memory()
    ud = u_host.to(dev)
    pd = p_host.to(dev)
    y_lap = torch.empty(m.n_p, dtype=torch.float64, device=dev)
    b_div = torch.empty(m.n_p, dtype=torch.float64, device=dev)
    y_conv = torch.empty(m.n_u, dtype=torch.float64, device=dev)
    y_visc = torch.empty(m.n_u, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2
    stream = torch.cuda.current_stream()
    ops = ["eddy_viscosity", "laplace", "divergence", "convective", "viscous"]
    ev = {o: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for o in ops}

    def step(timed):
        for o in ops:
            if timed:
                ev[o][0].record(stream)
            if o == "eddy_viscosity":
                m.update_eddy_viscosity(ud)
            elif o == "laplace":
                m.laplace(pd, y_lap)
            elif o == "divergence":
                m.divergence(ud, b_div)
            elif o == "convective":
                m.convective(ud, y_conv)
            else:
                m.viscous(ud, y_visc)
            if timed:
                ev[o][1].record(stream)

    for _ in range(max(args.warmup, 1)):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0, _ = dgw.counters()
    step_ms, op_ms = [], {o: [] for o in ops}
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()                       # evict the previous step's data from L2 (not timed)
        torch.cuda.nvtx.range_push("dgw_step")
        step(True)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        for o in ops:
            op_ms[o].append(ev[o][0].elapsed_time(ev[o][1]))
        step_ms.append(ev[ops[0]][0].elapsed_time(ev[ops[-1]][1]))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    launches1, _ = dgw.counters()
    clk = clocks.stop()
    ms_max = replica_time(statistics.mean(step_ms), world, dev)
    dofs_ops = {"laplace": m.n_p, "divergence": m.n_p, "convective": m.n_u, "viscous": m.n_u}
    dofs_step = float(sum(dofs_ops.values()))
    value = weak_value(dofs_step, world, ms_max)
    nc = w.nx * w.ny * w.nz
    curved = w.geometry == 1
    per_op = {o: {"ms": statistics.mean(op_ms[o])} for o in ops}
    for o, d in dofs_ops.items():
        per_op[o]["gdofs"] = d / (per_op[o]["ms"] * 1e-3) / 1e9
        fl = laplace_flops_per_cell(w.k, curved) if o == "laplace" else vector_flops_per_cell(o, w.k, curved)
        per_op[o]["flops_per_cell"] = fl
        per_op[o]["fp64_tflops"] = nc * fl / (per_op[o]["ms"] * 1e-3) / 1e12
        per_op[o]["fp64_frac"] = per_op[o]["fp64_tflops"] / FP64_PEAK_TFLOPS
        nbytes = 8.0 * (m.n_p + m.n_p if o == "laplace" else (m.n_u + m.n_p if o == "divergence" else 2 * m.n_u))
        per_op[o]["hbm_gbs"] = nbytes / (per_op[o]["ms"] * 1e-3) / 1e9

    peaks, src = _peaks()
    dom = max(dofs_ops, key=lambda o: per_op[o]["ms"])
    geo = "GEO_CURVED" if curved else "GEO_BOX"
    opname = {"divergence": "OP_DIV", "convective": "OP_CONV", "viscous": "OP_VISC"}
    boxname = {"divergence": "box_div_kernel", "convective": "box_conv_kernel", "viscous": "box_visc_kernel"}
    if dom == "laplace":
        kname = f"curved_laplace_kernel<double,{w.k}>" if curved else f"laplace_box_kernel<double,double,{w.k}>"
    elif curved:
        kname = f"vector_op_kernel<double,{opname[dom]},GEO_CURVED>"
    else:
        kname = (f"{boxname[dom]}<double,double,{w.k}> (standard rows) + vector_op_kernel<double,{opname[dom]},GEO_BOX> "
                 "(rows of the enriched layers)")
    roofline = {"kernel": kname, "bound": "alu", "achieved": per_op[dom]["fp64_tflops"], "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": per_op[dom]["fp64_frac"],
                "traffic": args.traffic_bytes,
                "algorithmic_flops_per_launch": nc * per_op[dom]["flops_per_cell"],
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz",
                "hbm_frac": per_op[dom]["hbm_gbs"] / peaks["hbm_gbs"],
                "hbm_peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)" if src == "measured" else "fallback 6800 GB/s"}

    # FP32 SIPG Laplacian (the operator of the FP32 multigrid), timed alone with CUDA events after an
    # L2 flush, per launch: HBM roofline with 8 B per DoF (read p, write y)
    p32 = pd.float()
    y32 = torch.empty(m.n_p, dtype=torch.float32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        m.laplace(p32, y32)
    lap32 = []
    for _ in range(10):
        flush.zero_()
        e0.record(stream)
        m.laplace(p32, y32)
        e1.record(stream)
        torch.cuda.synchronize()
        lap32.append(e0.elapsed_time(e1))
    lap32_ms = statistics.median(lap32)
    ach32 = 8.0 * m.n_p / (lap32_ms * 1e-3) / 1e9
    fp32_laplace = {"kernel": ("curved_laplace_kernel<float,%d>" if curved else "laplace_box_kernel<float,%d>") % w.k,
                    "bound": "hbm", "ms": lap32_ms, "gdofs": m.n_p / (lap32_ms * 1e-3) / 1e9,
                    "achieved": ach32, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach32 / peaks["hbm_gbs"],
                    "fp32_flop_frac": nc * laplace_flops_per_cell(w.k, curved) / (lap32_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS}

    # the same step with every apply in double-float arithmetic on the FP32 units (DGW_DF64: double
    # vectors, FP64-accurate; the rows of the enriched layers stay in FP64), box cells
    df64_step = None
    if not curved:
        DF = dgw.DGW_DF64
        dsteps, dops = [], {o: [] for o in ops}
        def dstep(timed):
            for o in ops:
                if timed:
                    ev[o][0].record(stream)
                if o == "eddy_viscosity":
                    m.update_eddy_viscosity(ud)
                elif o == "laplace":
                    m.laplace(pd, y_lap, prec=DF)
                elif o == "divergence":
                    m.divergence(ud, b_div, prec=DF)
                elif o == "convective":
                    m.convective(ud, y_conv, prec=DF)
                else:
                    m.viscous(ud, y_visc, prec=DF)
                if timed:
                    ev[o][1].record(stream)
        for _ in range(3):
            dstep(False)
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            dstep(True)
            torch.cuda.synchronize()
            for o in ops:
                dops[o].append(ev[o][0].elapsed_time(ev[o][1]))
            dsteps.append(ev[ops[0]][0].elapsed_time(ev[ops[-1]][1]))
        dms = statistics.mean(dsteps)
        df64_step = {"value": dofs_step / (dms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": dms,
                     "dtype": "df64 (double vectors, FP32-pair arithmetic)",
                     "per_op_ms": {o: statistics.mean(dops[o]) for o in ops}}
        step(False)   # restore the FP64 outputs used below

    # the same Laplacian with double vectors in double-float arithmetic on the FP32 units (FP64-accurate
    # emulation) against the native FP64 apply, each timed alone after an L2 flush (box cells only)
    emulation = None
    if not curved:
        def t_alone(fn):
            for _ in range(3):
                fn()
            ts = []
            for _ in range(10):
                flush.zero_()
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.median(ts)
        ydf = torch.empty_like(y_lap)
        ms64 = t_alone(lambda: m.laplace(pd, y_lap))
        msdf = t_alone(lambda: m.laplace(pd, ydf, prec=dgw.DGW_DF64))
        diff = float(torch.linalg.norm(ydf - y_lap) / torch.linalg.norm(y_lap))
        fl = nc * laplace_flops_per_cell(w.k)
        emulation = {"kernel": f"laplace_box_kernel<double,df64,{w.k}> vs laplace_box_kernel<double,double,{w.k}>", "fp64_ms": ms64, "df64_ms": msdf,
                     "speedup": ms64 / msdf, "rel_diff_vs_fp64": diff,
                     "df64_gdofs": m.n_p / (msdf * 1e-3) / 1e9,
                     "fp64_equiv_tflops": fl / (msdf * 1e-3) / 1e12,
                     "hbm_frac": 16.0 * m.n_p / (msdf * 1e-3) / 1e9 / peaks["hbm_gbs"]}

    # pressure solves to 1e-10: FP64 (FP64 CG + FP64 multigrid) vs mixed, on this workload (rhs = the
    # step's divergence) and on the Q3 64x32x32 channel (seeded zero-mean rhs)
    solves = {}
    p_sol = torch.zeros(m.n_p, dtype=torch.float64, device=dev)
    solves[w.name] = _time_solves(m, b_div, p_sol, (("fp64", 0), ("mixed", 1)), 3, flush)
    # the same mixed solve as a block of 8 right-hand sides (the request loop's batched form; box
    # meshes)
    if w.geometry == 0:
        solves[w.name]["mixed_block"] = _time_block_solves(m, b_div, 8, 3, flush)
        solves[w.name]["block_over_mixed"] = (solves[w.name]["mixed_block"]["solves_per_s"] /
                                              solves[w.name]["mixed"]["solves_per_s"])
    if not args.no_extra_solves and world == 1:
        w3 = I.WORKLOADS["channel_q3_64x32x32"]
        m3 = dgw.mesh_for(w3)
        b3 = torch.tensor(I.pressure_rhs(m3.n_p, w3.seed), device=dev)
        p3 = torch.zeros_like(b3)
        solves[w3.name] = _time_solves(m3, b3, p3, (("fp64", 0), ("mixed", 1)), 2, flush)
        m3.close()

    # end to end through the public API with host buffers (copies inside the timed region)
    out_host = {n: torch.empty(t.numel(), dtype=torch.float64).pin_memory()
                for n, t in (("lap", y_lap), ("div", b_div), ("conv", y_conv), ("visc", y_visc))}
    # the uploads run on one copy stream (p first: the Laplacian starts while u is still in flight), the
    # read-backs on another as each result is ready; every copy is inside the timed region
    up_s, down_s, main_s = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.current_stream()
    e_p, e_u = torch.cuda.Event(), torch.cuda.Event()
    e_out = {n: torch.cuda.Event() for n in out_host}
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(up_s):
            pd.copy_(p_host, non_blocking=True)
            e_p.record(up_s)
            ud.copy_(u_host, non_blocking=True)
            e_u.record(up_s)
        main_s.wait_event(e_p)
        m.laplace(pd, y_lap)
        e_out["lap"].record(main_s)
        main_s.wait_event(e_u)
        # the smallest result (the divergence, n_p values) last, so the read-back left after the
        # last apply is the shortest
        m.update_eddy_viscosity(ud)
        m.convective(ud, y_conv)
        e_out["conv"].record(main_s)
        m.viscous(ud, y_visc)
        e_out["visc"].record(main_s)
        m.divergence(ud, b_div)
        e_out["div"].record(main_s)
        with torch.cuda.stream(down_s):
            for n, t in (("lap", y_lap), ("conv", y_conv), ("visc", y_visc), ("div", b_div)):
                down_s.wait_event(e_out[n])
                out_host[n].copy_(t, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    h2d = 8 * (m.n_u + m.n_p)
    d2h = 8 * (2 * m.n_p + 2 * m.n_u)
    e2e_ms_max = replica_time(statistics.mean(e2e_ms), world, dev)
    e2e = {"value": weak_value(dofs_step, world, e2e_ms_max), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_max}

    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        serving = serving_stream(args.serving_short_jobs, args.rate, args.serving_slots, args.serving_budget_gb)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, secs, threads, desc = oracle_sample(w, target_s=args.ref_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc, "seconds": secs}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": w.name, "cells": [w.nx, w.ny, w.nz], "degree": w.k, "re_tau": w.re_tau,
                           "n_p": m.n_p, "n_u": m.n_u, "n_enriched": m.n_e,
                           "step": "nu_t update + FP64 Laplace, divergence, convective, viscous applies",
                           "parallelism": f"replicas{world}", "l2": "flushed between steps (512 MB write)"},
                "per_op": per_op, "dof_applies_per_step": dofs_step, "solves": solves,
                "roofline": roofline, "fp32_laplace": fp32_laplace, "df64_emulation": emulation, "df64_step": df64_step,
                "serving": serving, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk, "gpu_launches": int(launches1 - launches0), "launches_before_timed": int(launches0),
                "wall_s": t_wall}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def serving_stream(n, rate, slots, budget_gb, seed=999):
    """Serving workload: Poisson arrivals (mean `rate` jobs/s, seeded) of pressure solves (3/4, mixed
    precision to 1e-10) and operator applies (1/4) on channels with N_x uniform in
    {8,16,24,32,40,48}, N_y = N_z = max(8, N_x/2), k uniform in {2,3,4,5}; per-job seeded inputs. Every
    distinct (mesh, job kind) is warmed first (resident mesh, multigrid and block solver). Returns
    p50/p99 latency (arrival to completion) and solves/s through the request loop, and the same jobs
    run one at a time with FP64 solves on meshes warmed the same way."""
    import numpy as np
    import torch
    from paper_1705_08813_gb300 import dgw, inputs as I
    rng_u = I.uniform(seed, 4 * n, 0.0, 1.0, stream=41)
    gaps = -np.log(1.0 - rng_u[:n]) / rate
    arrivals = np.cumsum(gaps)
    nxs = [8, 16, 24, 32, 40, 48]
    specs = []
    for j in range(n):
        nx = nxs[int(rng_u[n + j] * 6)]
        k = 2 + int(rng_u[2 * n + j] * 4)
        kind = 0 if rng_u[3 * n + j] < 0.75 else 1 + int((rng_u[3 * n + j] - 0.75) * 16)
        w = I.Workload(f"s{j}", nx, max(8, nx // 2), max(8, nx // 2), k, 590.0, 1.0 / 12000.0, seed=1000 + j)
        specs.append((kind, w))
    gen = torch.Generator(device="cuda")
    bufs = []
    for j, (kind, w) in enumerate(specs):
        n1 = w.k + 1
        npd = w.nx * w.ny * w.nz * n1 ** 3
        nud = 3 * npd + 24 * 2 * w.nx * w.nz
        gen.manual_seed(1000 + j)
        nin = npd if kind in (0, 1) else nud
        nout = npd if kind in (0, 1, 2) else nud
        inp = torch.rand(nin, dtype=torch.float64, device="cuda", generator=gen) * 2 - 1
        if kind == 0:
            inp -= inp.mean()
        aux = inp if kind == 4 else None
        bufs.append((inp, torch.zeros(nout, dtype=torch.float64, device="cuda"), aux))
    torch.cuda.synchronize()
    srv = dgw.Server(int(budget_gb * (1 << 30)), max_inflight=slots)

    def drain(tickets):
        pend = set(tickets)
        while pend:
            for t in list(pend):
                if srv.poll(t) is not None:
                    pend.discard(t)
            time.sleep(0.001)

    # warm the resident meshes and solver state: one job per distinct (mesh, kind)
    seen, warm = set(), []
    for j, (kind, w) in enumerate(specs):
        key = (w.nx, w.k, kind)
        if key not in seen:
            seen.add(key)
            inp, out, aux = bufs[j]
            warm.append(srv.submit(kind, dgw.mesh_params(w), inp, out, aux=aux, mode=1))
    drain(warm)
    # timed stream
    t0 = time.perf_counter()
    tickets, submitted, done = {}, 0, {}
    while len(done) < n:
        now = time.perf_counter() - t0
        while submitted < n and arrivals[submitted] <= now:
            kind, w = specs[submitted]
            inp, out, aux = bufs[submitted]
            tickets[srv.submit(kind, dgw.mesh_params(w), inp, out, aux=aux, mode=1)] = submitted
            submitted += 1
        for t in list(tickets):
            r = srv.poll(t)
            if r is not None:
                j = tickets.pop(t)
                done[j] = (r, time.perf_counter() - t0)
        time.sleep(0.0002)
    makespan = max(v[1] for v in done.values())
    lat = np.array([1e3 * (done[j][1] - arrivals[j]) for j in range(n)])
    slat = np.array([lat[j] for j in range(n) if specs[j][0] == 0])
    ok = all(done[j][0]["status"] == 0 for j in range(n))
    failures = [{"job": j, "kind": specs[j][0], "cells": [specs[j][1].nx, specs[j][1].ny, specs[j][1].nz],
                 "degree": specs[j][1].k, "status": done[j][0]["status"]} for j in range(n) if done[j][0]["status"] != 0]
    n_solves = sum(1 for kind, _ in specs if kind == 0)
    srv.close()
    # one at a time, FP64 solves, meshes and hierarchies warmed by one untimed job each
    meshes = {}
    def run_one(j, mesh):
        kind, w = specs[j]
        inp, out, aux = bufs[j]
        if kind == 0:
            mesh.pressure_solve(inp, out, rtol=1e-10, max_iter=500, mode=0)
        elif kind == 1:
            mesh.laplace(inp, out)
        elif kind == 2:
            mesh.divergence(inp, out)
        elif kind == 3:
            mesh.convective(inp, out)
        else:
            mesh.update_eddy_viscosity(aux)
            mesh.viscous(inp, out)
    warmed = set()
    for j, (kind, w) in enumerate(specs):
        key = (w.nx, w.k)
        if key not in meshes:
            meshes[key] = dgw.mesh_for(w)
        if (key, kind) not in warmed:
            warmed.add((key, kind))
            run_one(j, meshes[key])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for j in range(n):
        run_one(j, meshes[(specs[j][1].nx, specs[j][1].k)])
        torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    for mm in meshes.values():
        mm.close()
    return {"metric": "serving: p50/p99 latency and solves/s (mixed, request loop with continuous batching) vs "
                      "one-at-a-time FP64",
            "jobs": n, "solves": n_solves, "rate_per_s": rate, "slots": slots, "all_ok": ok, "failures": failures[:10],
            "arrival_span_s": float(arrivals[-1]), "makespan_s": makespan,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "solve_p50_ms": float(np.percentile(slat, 50)) if len(slat) else None,
            "solve_p99_ms": float(np.percentile(slat, 99)) if len(slat) else None,
            "solves_per_s": n_solves / makespan, "sequential_fp64_solves_per_s": n_solves / seq,
            "sequential_s": seq, "speedup_solves": (n_solves / makespan) / (n_solves / seq)}


def run_serving(args):
    import torch
    from paper_1705_08813_gb300 import dgw
    torch.cuda.set_device(0)
    dgw.load()
    line = serving_stream(args.serving_jobs, args.rate, args.serving_slots, args.serving_budget_gb)
    print(json.dumps(line), flush=True)
    return 0


def run_helmholtz(args):
    """Viscous step of the dual-splitting scheme on the workload: velocity mass apply (FP64, FP32; the FP64
    viscous, convective and divergence applies beside it) and the
    Helmholtz solve gamma M u - F^nu(u) = gamma M u^ (gamma = 1.5 / dt, BDF2, dt = args.dt) to 1e-10 with
    restarted GMRES, nu_t frozen from the workload's velocity field, initial guess u^. --enrich-l 0 takes the
    constant enrichment weight (one coefficient per component and wall cell) instead of the trilinear one."""
    import torch
    from paper_1705_08813_gb300 import dgw, inputs as I
    torch.cuda.set_device(0)
    w = I.WORKLOADS[args.workload]
    m = dgw.mesh_for(w, enrich_l=args.enrich_l)
    nef = 8 if args.enrich_l == 1 else 1
    u_hat = torch.from_numpy(I.workload_velocity(m.node_coords(), m.n_e, w, nef=nef)).cuda()
    m.update_eddy_viscosity(u_hat)
    gamma = 1.5 / args.dt
    rhs = torch.empty_like(u_hat)
    m.mass(u_hat, rhs)
    rhs *= gamma
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    y = torch.empty_like(u_hat)
    y32 = torch.empty(m.n_u, dtype=torch.float32, device="cuda")
    u32 = u_hat.float()
    times = {}
    b = torch.empty(m.n_p, dtype=torch.float64, device="cuda")
    for name, fn in (("mass64", lambda: m.mass(u_hat, y)), ("mass32", lambda: m.mass(u32, y32)),
                     ("viscous64", lambda: m.viscous(u_hat, y)), ("convective64", lambda: m.convective(u_hat, y)),
                     ("divergence64", lambda: m.divergence(u_hat, b))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(10):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        times[name] = ev0.elapsed_time(ev1) / 10
    u = u_hat.clone()
    m.helmholtz_solve(gamma, rhs, u, rtol=1e-10, max_iter=5000, restart=args.restart)   # setup and warm-up
    ts, infos = [], []
    for _ in range(max(1, args.steps)):
        u.copy_(u_hat)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos.append(m.helmholtz_solve(gamma, rhs, u, rtol=1e-10, max_iter=5000, restart=args.restart))
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.median(ts)
    print(json.dumps({"metric": "viscous Helmholtz step: mass apply GDoF/s and GMRES solves/s at 1e-10",
                      "workload": w.name, "enrich_l": args.enrich_l, "n_u": m.n_u, "gamma": gamma, "dt": args.dt, "restart": args.restart,
                      "mass_fp64_ms": times["mass64"], "mass_fp64_gdofs": m.n_u / (times["mass64"] * 1e-3) / 1e9,
                      "mass_fp32_ms": times["mass32"], "mass_fp32_gdofs": m.n_u / (times["mass32"] * 1e-3) / 1e9,
                      "viscous_fp64_ms": times["viscous64"], "convective_fp64_ms": times["convective64"],
                      "divergence_fp64_ms": times["divergence64"],
                      "solve_ms": ms, "solves_per_s": 1e3 / ms, "iterations": infos[-1]["iterations"],
                      "rel_residual": infos[-1]["rel_residual"]}), flush=True)
    return 0


def run_wall_update(args):
    """Adaptive part of the wall model at the start of a time step (Sec. 3.2): nodal tau_w,B from the
    velocity, the cell-wise L2 projection of the velocity onto the new enrichment space, and nu_t in
    the new space; each timed with CUDA events on the workload (median of --steps runs)."""
    import torch
    from paper_1705_08813_gb300 import dgw, inputs as I
    torch.cuda.set_device(0)
    w = I.WORKLOADS[args.workload]
    m = dgw.mesh_for(w, enrich_l=args.enrich_l)
    nef = 8 if args.enrich_l == 1 else 1
    u = torch.from_numpy(I.workload_velocity(m.node_coords(), m.n_e, w, nef=nef)).cuda()
    tau = torch.empty(m.n_wall_nodes, dtype=torch.float64, device="cuda")
    u2 = torch.empty_like(u)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    rec = {"tau_ms": [], "project_ms": [], "nut_ms": []}
    for it in range(args.warmup + max(1, args.steps)):
        torch.cuda.synchronize()
        ev[0].record()
        m.wall_shear_stress(u, tau)
        ev[1].record()
        m.project_velocity(tau, u, u2)
        ev[2].record()
        m.update_eddy_viscosity(u2)
        ev[3].record()
        torch.cuda.synchronize()
        if it >= args.warmup:
            rec["tau_ms"].append(ev[0].elapsed_time(ev[1]))
            rec["project_ms"].append(ev[1].elapsed_time(ev[2]))
            rec["nut_ms"].append(ev[2].elapsed_time(ev[3]))
        u, u2 = u2, u
    tn = tau.cpu().numpy()
    out = {"metric": "wall-model update: tau_w,B, L2 projection onto the new space, nu_t (ms)",
           "workload": w.name, "enrich_l": args.enrich_l, "n_u": m.n_u, "n_enriched": m.n_e,
           "tau_w_range": [float(tn.min()), float(tn.max())]}
    for k, v in rec.items():
        out[k] = statistics.median(v)
    out["total_ms"] = out["tau_ms"] + out["project_ms"] + out["nut_ms"]
    print(json.dumps(out), flush=True)
    return 0


def run_ns_step(args):
    """Dual-splitting time steps on the workload (convective step, pressure solve, projection, viscous
    step; with --wall-update-steps also tau_w and the L2 projection at the start of every step),
    constant dt (with --adaptive-dt the CFL step with Cr = 0.14, dt as its upper bound), body force
    u_tau^2 / delta along x; host wall time per step after --warmup steps."""
    import torch
    from paper_1705_08813_gb300 import dgw, inputs as I
    torch.cuda.set_device(0)
    w = I.WORKLOADS[args.workload]
    m = dgw.mesh_for(w, enrich_l=args.enrich_l)
    nef = 8 if args.enrich_l == 1 else 1
    u0 = torch.from_numpy(I.workload_velocity(m.node_coords(), m.n_e, w, nef=nef)).cuda()
    delta = 0.5 * w.ly
    ns = dgw.DualSplitting(m, u0, dt=args.dt, force=(w.tau_w / delta, 0.0, 0.0), rtol_pressure=1e-10,
                           rtol_projection=1e-10, rtol_viscous=1e-10, pressure_mode=args.solve_mode,
                           update_wall_model=args.wall_update_steps, adaptive_dt=args.adaptive_dt)
    infos = []
    for it in range(args.warmup + max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = ns.step()
        torch.cuda.synchronize()
        info["wall_ms"] = 1e3 * (time.perf_counter() - t0)
        if it >= args.warmup:
            infos.append(info)
    med = lambda k: statistics.median(i[k] for i in infos)
    print(json.dumps({"metric": "dual-splitting time step (ms per step)", "workload": w.name,
                      "enrich_l": args.enrich_l, "n_u": m.n_u, "n_p": m.n_p, "dt": args.dt,
                      "wall_model_update": bool(args.wall_update_steps), "pressure_mode": args.solve_mode,
                      "adaptive_dt": bool(args.adaptive_dt), "dt_taken": [i["dt"] for i in infos],
                      "steps": len(infos), "ms_per_step": med("wall_ms"),
                      "pressure_iterations": med("pressure_iterations"),
                      "projection_iterations": med("projection_iterations"),
                      "viscous_iterations": med("viscous_iterations")}), flush=True)
    return 0


def run_profile_kernel(args):
    """A few launches of one operator kernel on a channel of the given size (used for ncu captures:
    a small number of launches, inputs larger than L2 when the mesh is large enough)."""
    import torch
    from paper_1705_08813_gb300 import dgw, inputs as I
    nx, ny, nz, k = args.profile_cells
    if args.profile_geometry == 1:
        w = I.bump_workload("profile", nx, ny, nz, k, seed=7)
    else:
        w = I.Workload("profile", nx, ny, nz, k, 590.0, 1.0 / 12000.0, seed=7)
    m = dgw.mesh_for(w)
    kind = args.profile_kernel
    dt = torch.float32 if kind.endswith("32") else torch.float64
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    if kind.startswith("laplace"):
        x = torch.rand(m.n_p, dtype=dt, device="cuda", generator=gen)
        y = torch.empty_like(x)
        prec = dgw.DGW_DF64 if kind == "laplace_df64" else None
        op = lambda: m.laplace(x, y, prec=prec)
    else:
        u = torch.rand(m.n_u, dtype=torch.float64, device="cuda", generator=gen)
        m.update_eddy_viscosity(u)
        x = u.to(dt)
        y = torch.empty(m.n_p if kind.startswith("divergence") else m.n_u, dtype=dt, device="cuda")
        if kind.startswith("divergence"):
            x = u
        tau = torch.full((m.nc,), 1e-3, dtype=torch.float64, device="cuda")
        DF = dgw.DGW_DF64
        op = {"divergence": lambda: m.divergence(x, y), "convective": lambda: m.convective(x, y),
              "divergence_df64": lambda: m.divergence(x, y, prec=DF), "viscous_df64": lambda: m.viscous(x, y, prec=DF),
              "convective_df64": lambda: m.convective(x, y, prec=DF),
              "convective32": lambda: m.convective(x, y), "viscous": lambda: m.viscous(x, y),
              "viscous32": lambda: m.viscous(x, y), "mass": lambda: m.mass(x, y),
              "divdiv": lambda: m.divdiv(tau, x, y), "curl": lambda: m.curl(x, y),
              "inverse_mass": lambda: m.inverse_mass(x, y)}[kind]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        op()
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.profile_reps):
        op()
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.profile_reps
    print(json.dumps({"kernel": kind, "geometry": args.profile_geometry, "cells": [nx, ny, nz], "degree": k,
                      "n_p": m.n_p, "n_u": m.n_u, "ms_per_launch": ms}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dgw", choices=["dgw", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--solve-mode", type=int, default=1, help="pressure solve mode of --ns-step")
    ap.add_argument("--no-extra-solves", action="store_true", help="skip the Q3 64x32x32 solves")
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # DRAM bytes (read + write) per launch of the roofline kernel, from an ncu capture of the same
    # kernel build; none unless given
    ap.add_argument("--traffic-bytes", type=float, default=None)
    ap.add_argument("--serving", action="store_true")
    ap.add_argument("--serving-jobs", type=int, default=400)
    ap.add_argument("--serving-short-jobs", type=int, default=120, help="serving stream of the default run")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream of the default run")
    ap.add_argument("--serving-slots", type=int, default=8)
    ap.add_argument("--serving-budget-gb", type=float, default=120.0)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--helmholtz", action="store_true", help="time the mass apply and the Helmholtz solve")
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--enrich-l", type=int, default=1, choices=[0, 1],
                    help="enrichment weight degree (--helmholtz, --wall-update)")
    ap.add_argument("--wall-update", action="store_true", help="time the tau_w update and the L2 projection")
    ap.add_argument("--ns-step", action="store_true", help="time dual-splitting time steps")
    ap.add_argument("--wall-update-steps", action="store_true", help="--ns-step: update the wall model every step")
    ap.add_argument("--adaptive-dt", action="store_true", help="--ns-step: the CFL step (Cr = 0.14), --dt its upper bound")
    ap.add_argument("--profile-kernel", default=None,
                    choices=["laplace64", "laplace32", "laplace_df64", "divergence_df64", "viscous_df64",
                             "convective_df64", "divergence", "convective", "convective32", "viscous",
                             "viscous32", "mass", "divdiv", "curl", "inverse_mass"])
    ap.add_argument("--profile-cells", type=int, nargs=4, default=[64, 48, 48, 4], metavar=("NX", "NY", "NZ", "K"))
    ap.add_argument("--profile-reps", type=int, default=3)
    ap.add_argument("--profile-geometry", type=int, default=0, choices=[0, 1], help="0 channel, 1 bump")
    args = ap.parse_args()
    if args.profile_kernel:
        return run_profile_kernel(args)
    if args.serving:
        return run_serving(args)
    if args.helmholtz:
        return run_helmholtz(args)
    if args.wall_update:
        return run_wall_update(args)
    if args.ns_step:
        return run_ns_step(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
