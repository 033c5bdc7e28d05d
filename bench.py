"""Benchmark: SHO projection + expansion throughput on one GB300 (psi GB/s at stated error).

One step = one pass of the hot path over the 96^3 workload: project psi onto every atom's SHO basis
(1D tables, cube gather, x/y/z passes), then expand random FP64 coefficients into a second wave-function
buffer (z/y/x passes, row gather).  Inputs are resident in HBM before the timed region; psi (906 MB)
is larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead, on a bounded
sample of the same workload.  Under torchrun (N > 1) every rank runs its own replica of the workload
(weak scaling, no collective); the reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "SHO project+expand psi GB/s vs HBM peak at stated error; p50/p99 request latency"
WORKLOAD = "c96"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# DRAM bytes (read + write) of one call, summed over its kernels' launches, from one ncu capture of the
# default FF64 bench step (96^3 / 64 atoms / 128 bands), by (call, expansion engine); valid only while
# those kernels are unchanged (None otherwise).
NCU_TRAFFIC = {("k_project", e): 1985944576 + 43182592 + 44085248 for e in ("auto", "mma_sync")}  # x/y + z-pass
NCU_TRAFFIC.update({("k_expand", e): 3760128 + 44259584 + 951985408 + 841280512 for e in ("auto", "tcgen05")})

# FP64 FMA peak of the GB300 measured by a DFMA throughput loop (152 SMs x 2 DFMA/clk/SM x 2 flop,
# 1.19 TFLOP/s at the clocks seen under load); the kernels of the FP64 form are bound by this pipe.
FP64_PEAK_TFLOPS = 1.19


def union_cube_points(w, pos):
    """Number of distinct grid points covered by the atoms' cubes (counted exactly on the host)."""
    nx, ny, nz = w.grid
    mask = np.zeros((nz, ny, nx), dtype=bool)
    i = np.arange(w.cube)
    for X in pos:
        o = np.floor(X / w.h).astype(int) - w.cube // 2 + 1
        idx = []
        for d, n in enumerate((nx, ny, nz)):
            j = o[d] + i
            if w.periodic:
                j = j % n
            else:
                j = j[(j >= 0) & (j < n)]
            idx.append(j)
        mask[np.ix_(idx[2], idx[1], idx[0])] = True
    return int(mask.sum())


def algorithmic(w, pos, nstates, elem=8):
    """Algorithmic bytes and flops of one step (projection + expansion)."""
    U = union_cube_points(w, pos)
    A, B, C, nu = w.natoms, w.nbands, w.cube, w.numax
    P = (nu + 1) * (nu + 2) // 2
    coeff = A * nstates * B * elem
    bytes_prj = U * B * elem + coeff
    bytes_add = 2 * U * B * elem + coeff
    flop_per_atom_band = 2 * (C ** 3 * (nu + 1) + C ** 2 * P + C * nstates)
    flops = A * B * flop_per_atom_band
    return dict(union_points=U, bytes_prj=bytes_prj, bytes_add=bytes_add, flops_prj=flops, flops_add=flops)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.dev = device_index
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, value):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def launches_per_step(api, psi, w, prec, expand_kernel="auto", project_kernel="auto"):
    """Kernels of this library that one project + expand step launches (mirrors the library's dispatch)."""
    if prec == "ff64":
        full = 4 * w.nbands >= 3 * 128 * ((w.nbands + 127) // 128)  # the automatic choice wants full tiles
        oz = ((expand_kernel == "tcgen05" or (expand_kernel == "auto" and full)) and w.numax <= 7 and w.cube <= 32
              and w.cube % 2 == 0 and w.nbands % 2 == 0 and (not w.periodic or w.grid[0] >= w.cube + 32))
        # projection: the digit tables, the tensor-core x-pass and the z-pass (or the float-float x/y-pass
        # and the z-pass); expansion: the float-pair z-pass (with the tables), then the digit tables and
        # the tensor-core x-pass (or the block gather)
        ozp = project_kernel == "tcgen05" and w.numax <= 7 and w.cube <= 32
        return (3 if ozp else 2) + (3 if oz else 2)
    if prec == "fp64":
        return 1 + 2  # cluster projection; z-pass + row gather
    tc = prec in ("tf32", "3xtf32", "bf16", "split_fp16")
    prj = 3 if api.project_path(psi, w.numax, w.cube, w.h, w.periodic, prec=prec) == "plane" else 1
    stream_ok = (w.nbands * psi.element_size()) % 16 == 0 and w.nbands % 4 == 0
    add = (3 if tc else 2) if stream_ok else 2
    return prj + add


# --------------------------------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import torch
    from paper_1905_00480_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workloads.WORKLOADS[args.workload]
    if args.bands:
        w = workloads.Workload(**{**w.__dict__, "nbands": args.bands})
    prec = args.prec or ("ff64" if w.dtype == "f64" else "fp32")
    sdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[args.storage or w.dtype]
    cdt = torch.float64 if prec in ("fp64", "ff64") else torch.float32
    elem = torch.tensor([], dtype=sdt).element_size()
    # every rank runs its own replica with its own seed stream (weak scaling)
    rng = np.random.default_rng([w.seed, rank])
    pos, sig = workloads.atoms(w, rng if rank else None)
    nst = api.nstates(w.numax)
    alg = algorithmic(w, pos, nst, elem=elem)
    g = torch.Generator(device=dev)
    g.manual_seed(w.seed + 7919 * rank)
    nx, ny, nz = w.grid
    psi = torch.randn((nz, ny, nx, w.nbands), generator=g, device=dev, dtype=torch.float64).to(sdt)
    cin = torch.randn((w.natoms, nst, w.nbands), generator=g, device=dev, dtype=torch.float64).to(cdt)
    hpsi = torch.zeros_like(psi)
    coeff = torch.empty((w.natoms, nst, w.nbands), dtype=cdt, device=dev)
    handle = api.Handle(local)
    if args.expand_kernel != "auto":
        handle.set_expand_kernel(args.expand_kernel)
    if args.project_kernel != "auto":
        handle.set_project_kernel(args.project_kernel)
    stream = torch.cuda.current_stream(dev)

    def step():
        api.project(psi, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=prec, out=coeff, handle=handle,
                    stream=stream)
        api.add(hpsi, cin, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=prec, handle=handle, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(K):
        ev[i][0].record(stream)
        api.project(psi, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=prec, out=coeff, handle=handle,
                    stream=stream)
        ev[i][1].record(stream)
        api.add(hpsi, cin, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=prec, handle=handle, stream=stream)
        ev[i][2].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms_total = t0.elapsed_time(t1)
    ms_total = max_over_ranks(ws, ms_total)
    ms_step = ms_total / K
    t_prj = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    t_add = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    bytes_step = alg["bytes_prj"] + alg["bytes_add"]
    value = ws * bytes_step / (ms_step * 1e-3) / 1e9

    # end to end through the public API: pinned host psi and coefficients in, expansion result out.  Steps
    # are pipelined over two device buffer sets on three streams (copy in, compute, copy out), as a caller
    # streaming many steps would drive it: step i's copies overlap step i-1's kernels; every step's copies
    # lie inside the timed region.
    psi_h = torch.empty(psi.shape, dtype=psi.dtype, pin_memory=True)
    psi_h.copy_(psi)
    cin_h = torch.empty(cin.shape, dtype=cin.dtype, pin_memory=True)
    cin_h.copy_(cin)
    out_h = [torch.empty(psi.shape, dtype=psi.dtype, pin_memory=True) for _ in range(2)]
    del hpsi
    psi_d = [psi if i == 0 else torch.empty_like(psi) for i in range(2)]
    cin_d = [torch.empty_like(cin) for _ in range(2)]
    hps = [torch.empty_like(psi) for _ in range(2)]
    co = [coeff, torch.empty_like(coeff)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    s_cmp = stream
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    started = [False, False]

    def e2e_step(i):
        b = i % 2
        if started[b]:
            s_in.wait_event(ev_cmp[b])       # the compute of step i-2 is done with psi_d[b], cin_d[b]
        with torch.cuda.stream(s_in):
            psi_d[b].copy_(psi_h, non_blocking=True)
            cin_d[b].copy_(cin_h, non_blocking=True)
            ev_in[b].record(s_in)
        s_cmp.wait_event(ev_in[b])
        if started[b]:
            s_cmp.wait_event(ev_out[b])      # the copy-out of step i-2 is done with hps[b]
        with torch.cuda.stream(s_cmp):
            api.project(psi_d[b], pos, sig, w.numax, w.cube, w.h, w.periodic, prec=prec, out=co[b], handle=handle,
                        stream=s_cmp)
            hps[b].zero_()
            api.add(hps[b], cin_d[b], pos, sig, w.numax, w.cube, w.h, w.periodic, prec=prec, handle=handle,
                    stream=s_cmp)
            ev_cmp[b].record(s_cmp)
        s_out.wait_event(ev_cmp[b])
        with torch.cuda.stream(s_out):
            out_h[b].copy_(hps[b], non_blocking=True)
            ev_out[b].record(s_out)
        started[b] = True

    for i in range(max(2, args.warmup)):
        e2e_step(i)
    torch.cuda.synchronize()
    K2 = max(2, min(K, 10))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # three timed windows of K2 steps; the median is reported with all three (the host link is shared
    # with the machine's other GPUs, and one window can catch another job's traffic)
    e2e_runs = []
    for _ in range(3):
        barrier(ws)
        torch.cuda.synchronize()
        e0.record(s_in)
        for i in range(K2):
            e2e_step(i)
        s_in.wait_stream(s_out)
        e1.record(s_in)
        torch.cuda.synchronize()
        e2e_runs.append(max_over_ranks(ws, e0.elapsed_time(e1) / K2))
    ms_e2e = float(np.median(e2e_runs))
    h2d = psi.numel() * psi.element_size() + cin.numel() * cin.element_size()
    d2h = psi.numel() * psi.element_size()

    # the copy floor of that pipeline: the same copies on the same streams with no kernels in between
    def copy_step(i):
        b = i % 2
        with torch.cuda.stream(s_in):
            psi_d[b].copy_(psi_h, non_blocking=True)
            cin_d[b].copy_(cin_h, non_blocking=True)
        with torch.cuda.stream(s_out):
            out_h[b].copy_(hps[b], non_blocking=True)

    copy_step(0)
    torch.cuda.synchronize()
    e0.record(s_in)
    s_out.wait_stream(s_in)
    for i in range(K2):
        copy_step(i)
    s_in.wait_stream(s_out)
    e1.record(s_in)
    torch.cuda.synchronize()
    ms_copy = max_over_ranks(ws, e0.elapsed_time(e1) / K2)

    # the paper's timing protocol (Sec. 6): median over 15 runs of 10 back-to-back steps
    def step_p():
        api.project(psi, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=prec, out=coeff, handle=handle,
                    stream=stream)
        api.add(hps[0], cin, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=prec, handle=handle, stream=stream)

    step_p()
    per = []
    for _ in range(15):
        e0.record(stream)
        for _ in range(10):
            step_p()
        e1.record(stream)
        e1.synchronize()
        per.append(e0.elapsed_time(e1) / 10)
    ms_paper = max_over_ranks(ws, float(np.median(per)))
    # atoms that move every step (molecular dynamics): new positions each step, so the plan caches miss and
    # the host plans and uploads every time
    rng_md = np.random.default_rng([w.seed, rank, 17])
    moved = [pos + rng_md.normal(0.0, 0.02, size=pos.shape) for _ in range(10 + 2)]
    for i in range(2):
        api.project(psi, moved[i], sig, w.numax, w.cube, w.h, w.periodic, prec=prec, out=co[1], handle=handle,
                    stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(10):
        api.project(psi, moved[2 + i], sig, w.numax, w.cube, w.h, w.periodic, prec=prec, out=co[1], handle=handle,
                    stream=stream)
        api.add(hps[0], cin, moved[2 + i], sig, w.numax, w.cube, w.h, w.periodic, prec=prec, handle=handle,
                stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_md = max_over_ranks(ws, e0.elapsed_time(e1) / 10)

    result = None
    if rank == 0:
        peaks = _peaks()
        dom = "k_project" if t_prj >= t_add else "k_expand"
        t_dom = max(t_prj, t_add)
        if prec == "fp64":
            flops_dom = alg["flops_prj"] if dom == "k_project" else alg["flops_add"]
            achieved = flops_dom / (t_dom * 1e-3) / 1e12
            roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 4), "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": None,
                    "peak_source": "measured FP64 DFMA throughput (152 SMs x 4 flop/clk)"}
        else:
            bytes_dom = alg["bytes_prj"] if dom == "k_project" else alg["bytes_add"]
            achieved = bytes_dom / (t_dom * 1e-3) / 1e9
            hbm = peaks.get("hbm_gbs", 6793.4)
            traffic = (NCU_TRAFFIC.get((dom, args.project_kernel if dom == "k_project" else args.expand_kernel))
                       if (prec == "ff64" and args.workload == WORKLOAD and not args.bands) else None)
            roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 2), "peak": hbm, "unit": "GB/s",
                    "frac": round(achieved / hbm, 4), "traffic": traffic,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"}
        wl = {"c96": "periodic 96^3 grid, h=0.2, 64 atoms, sigma U[0.5,1], numax 5 (56 states), cube 32^3",
              "c160": "periodic 160^3 grid, h=0.2, 512 atoms, sigma U[0.5,1], numax 7 (120 states), cube 32^3",
              "c128": "periodic 128^3 grid, h=0.2, 128 atoms, sigma U[0.5,1], numax 5 (56 states), cube 32^3",
              "tiny": "16^3 grid, h=0.25, 1 atom, numax 3, cube 16"}[args.workload]
        result = {
            "metric": METRIC,
            "value": round(value, 3),
            "unit": "GB/s",
            "n_gpus": ws,
            "steps": K,
            "warmup": args.warmup,
            "ms_per_step": round(ms_step, 4),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"fp64": "f64", "ff64": "f64 (float-float passes; the expansion's x-pass as exact digit slices on TF32 tensor cores)", "fp32": "f32", "tf32": "tf32", "3xtf32": "3xtf32", "bf16": "bf16",
                      "split_fp16": "split-f16"}[prec],
            "data": "synthetic (seeded N(0,1) psi and coefficients, uniform atoms with min separation 2.0)",
            "config": {
                "workload": f"{wl}, {w.nbands} bands, psi {args.storage or w.dtype}, {prec} arithmetic: "
                            "project then expand",
                "global_batch": w.nbands * ws,
                "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                "l2": f"inputs larger than L2 (psi {psi.numel() * psi.element_size() / 1e6:.0f} MB per buffer), "
                      "no flush",
                **({"expand_kernel": args.expand_kernel} if args.expand_kernel != "auto" else {}),
                **({"project_kernel": args.project_kernel} if args.project_kernel != "auto" else {}),
                "union_cube_points": alg["union_points"],
                "algorithmic_bytes_per_step": bytes_step,
            },
            "kernels_ms": {"project": round(t_prj, 4), "expand": round(t_add, 4)},
            "hbm_fraction": round(value / ws / peaks.get("hbm_gbs", 6793.4), 4),
            "roofline": roof,
            "e2e": {"value": round(ws * bytes_step / (ms_e2e * 1e-3) / 1e9, 3), "unit": "GB/s",
                    "ms_per_step": round(ms_e2e, 4), "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "mode": "pinned host psi + coefficients in, expanded psi out, every step; pipelined over two "
                            "device buffer sets (copy-in, compute and copy-out streams); median of three "
                            "timed windows",
                    "ms_per_step_windows": [round(v, 4) for v in e2e_runs],
                    "copy_floor_ms_per_step": round(ms_copy, 4),
                    "copy_floor_note": "the same host<->device copies on the same streams without kernels"},
            "gpu_launches": launches_per_step(api, psi, w, prec, args.expand_kernel, args.project_kernel) * K,
            "clocks": clk,
            "paper_protocol": {"ms_per_step": round(ms_paper, 4),
                               "value": round(ws * bytes_step / (ms_paper * 1e-3) / 1e9, 3), "unit": "GB/s",
                               "protocol": "median over 15 runs of 10 back-to-back steps (Sec. 6)"},
            "moving_atoms": {"ms_per_step": round(ms_md, 4),
                             "value": round(ws * bytes_step / (ms_md * 1e-3) / 1e9, 3), "unit": "GB/s",
                             "note": "new atom positions every step (N(0, 0.02) Bohr displacements): the per-geometry "
                                     "plans are rebuilt on the host and uploaded inside the timed steps"},
        }
        default_case = args.workload == WORKLOAD and prec == "ff64" and not args.bands
        if not default_case:
            args.no_same_gpu_baselines = args.no_precision_forms = args.no_cpu_baseline = args.no_serving = True
            args.no_forces = True
        if not args.no_same_gpu_baselines:
            result["same_gpu_baselines"] = same_gpu_baselines(w, pos, sig, psi, cin, alg, api, handle, stream)
            result["roofline_fp64"] = result["same_gpu_baselines"]["fp64_dfma"]["roofline"]
        if not args.no_forces:
            result["forces"] = forces_bench(api, handle, stream)
        serve_sample = None
        if not args.no_serving:
            result["serving"], serve_sample = serving_bench(api)
            st = result["serving"]["loads"].get("0.8") or next(iter(result["serving"]["loads"].values()))
            result["p50_ms"], result["p99_ms"] = st["p50_ms"], st["p99_ms"]
        prec_samples = None
        if not args.no_precision_forms:
            del psi_h, out_h, psi_d, cin_d, hps
            torch.cuda.empty_cache()
            result["precision_forms"], prec_samples = precision_forms(api, handle, stream)
        if not args.no_cpu_baseline and ws == 1:
            result["cpu_baseline"], result["error_vs_oracle"] = cpu_baseline(
                w, pos, sig, psi, cin, coeff, hpsi_ref=None, api=api, handle=handle, prec=prec)
            if prec_samples is not None:
                oracle_precision_errors(result["precision_forms"], prec_samples)
            if serve_sample is not None:
                oracle_serving_errors(result["serving"], serve_sample)
    return result


def _time_steps(stream, fn, warmup=2, steps=5):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def fp64_gemm_peak(n=4096, reps=5):
    """FP64 throughput of cuBLAS DGEMM on this GPU (TFLOP/s, best of `reps`): the measured FP64 peak the
    native FP64 form is compared with."""
    import torch
    a = torch.randn((n, n), dtype=torch.float64, device="cuda")
    b = torch.randn((n, n), dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del a, b
    return round(best, 4)


def same_gpu_baselines(w, pos, sig, psi, cin, alg, api, handle, stream):
    """The same project + expand step on the same GPU with (1) stored FP64 projector values (the
    conventional scheme of the paper's comparison, Sec. 6) and (2) the FP32 CUDA-core form."""
    import torch
    out = {}
    bytes_step = alg["bytes_prj"] + alg["bytes_add"]
    proj = api.usu_build(pos, sig, w.numax, w.cube, w.grid, w.h, w.periodic, device=psi.device.index or 0,
                         handle=handle, stream=stream)
    coeff = torch.empty_like(cin)
    hpsi = torch.zeros_like(psi)

    def usu_step():
        api.usu_project(psi, proj, pos, sig, w.numax, w.cube, w.h, w.periodic, out=coeff, handle=handle,
                        stream=stream)
        api.usu_add(hpsi, cin, proj, pos, sig, w.numax, w.cube, w.h, w.periodic, handle=handle, stream=stream)

    ms = _time_steps(stream, usu_step)
    out["stored_projector_fp64"] = {"value": round(bytes_step / (ms * 1e-3) / 1e9, 3), "unit": "GB/s",
                                    "ms_per_step": round(ms, 4), "projector_bytes": proj.numel() * 8}
    del proj
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_prj, t_add = [], []
    for i in range(8):
        ev[0].record(stream)
        api.project(psi, pos, sig, w.numax, w.cube, w.h, w.periodic, prec="fp64", out=coeff, handle=handle,
                    stream=stream)
        ev[1].record(stream)
        api.add(hpsi, cin, pos, sig, w.numax, w.cube, w.h, w.periodic, prec="fp64", handle=handle, stream=stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            t_prj.append(ev[0].elapsed_time(ev[1]))
            t_add.append(ev[1].elapsed_time(ev[2]))
    tp, ta = float(np.median(t_prj)), float(np.median(t_add))
    fl = alg["flops_prj"]
    dgemm = fp64_gemm_peak()
    out["fp64_dfma"] = {"value": round(bytes_step / ((tp + ta) * 1e-3) / 1e9, 3), "unit": "GB/s",
                        "ms_per_step": round(tp + ta, 4), "ms_project": round(tp, 4), "ms_expand": round(ta, 4),
                        "fp64_pipe_frac_project": round(fl / (tp * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
                        "fp64_pipe_frac_expand": round(fl / (ta * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
                        "note": "native FP64 FMA form (FP64-pipe bound on GB300)"}
    dom_t = max(tp, ta)
    ach = fl / (dom_t * 1e-3) / 1e12
    out["fp64_dfma"]["roofline"] = {
        "bound": "alu", "kernel": "k_expand_rows" if ta >= tp else "k_project", "achieved": round(ach, 4),
        "peak": dgemm, "unit": "TFLOP/s", "frac": round(ach / dgemm, 4) if dgemm else None,
        "peak_source": "cuBLAS DGEMM 4096^3 (torch.matmul float64), best of 5, measured in this run",
        "frac_vs_dfma_loop": round(ach / FP64_PEAK_TFLOPS, 4)}
    # the full non-local action (project, per-atom D, expand) in the headline form
    rng = np.random.default_rng(11)
    Dm = rng.uniform(-1, 1, size=(w.natoms, cin.shape[1], cin.shape[1]))
    Dm = torch.from_numpy(0.5 * (Dm + Dm.transpose(0, 2, 1))).to(psi.device)
    hpsi.zero_()
    msn = _time_steps(stream, lambda: api.apply_nonlocal(psi, hpsi, Dm, pos, sig, w.numax, w.cube, w.h, w.periodic,
                                                         prec="ff64", handle=handle, stream=stream))
    out["nonlocal_action_ff64"] = {"value": round(bytes_step / (msn * 1e-3) / 1e9, 3), "unit": "GB/s",
                                   "ms_per_step": round(msn, 4),
                                   "note": "hpsi += E D P psi with a random symmetric N x N D per atom"}
    del hpsi
    psi32 = psi.float()
    cin32 = cin.float()
    c32 = torch.empty(cin.shape, dtype=torch.float32, device=psi.device)
    h32 = torch.zeros_like(psi32)

    def fp32_step():
        api.project(psi32, pos, sig, w.numax, w.cube, w.h, w.periodic, prec="fp32", out=c32, handle=handle,
                    stream=stream)
        api.add(h32, cin32, pos, sig, w.numax, w.cube, w.h, w.periodic, prec="fp32", handle=handle, stream=stream)

    ms32 = _time_steps(stream, fp32_step)
    bytes32 = bytes_step // 2
    out["fp32_cuda_cores"] = {"value": round(bytes32 / (ms32 * 1e-3) / 1e9, 3), "unit": "GB/s",
                              "ms_per_step": round(ms32, 4), "note": "same workload with psi and coefficients in FP32"}
    del psi32, h32
    # complex Bloch wave functions (FP64): 32 complex bands of the same geometry, Bloch vector k
    B = 32
    g = torch.Generator(device=psi.device)
    g.manual_seed(w.seed + 7)
    nx, ny, nz = w.grid
    zc = torch.complex(torch.randn((nz, ny, nx, B), generator=g, device=psi.device, dtype=torch.float64),
                       torch.randn((nz, ny, nx, B), generator=g, device=psi.device, dtype=torch.float64))
    cz = torch.complex(torch.randn((w.natoms, cin.shape[1], B), generator=g, device=psi.device, dtype=torch.float64),
                       torch.randn((w.natoms, cin.shape[1], B), generator=g, device=psi.device, dtype=torch.float64))
    oz = torch.empty_like(cz)
    hz = torch.zeros_like(zc)
    kvec = [0.9, -0.35, 1.7]

    def bloch_step():
        api.project_bloch(zc, kvec, pos, sig, w.numax, w.cube, w.h, out=oz, handle=handle, stream=stream)
        api.add_bloch(hz, cz, kvec, pos, sig, w.numax, w.cube, w.h, handle=handle, stream=stream)

    msb = _time_steps(stream, bloch_step, warmup=1, steps=3)
    bytes_b = (alg["bytes_prj"] + alg["bytes_add"]) * 2 * B // w.nbands
    out["bloch_complex_fp64"] = {"value": round(bytes_b / (msb * 1e-3) / 1e9, 3), "unit": "GB/s",
                                 "ms_per_step": round(msb, 4),
                                 "note": f"{B} complex128 bands, k = {kvec}: Bloch projection + expansion (4 DFMA "
                                         "per complex FMA)"}
    ozf = torch.empty_like(cz)
    hzf = torch.zeros_like(zc)

    def bloch_ff_step():
        api.project_bloch(zc, kvec, pos, sig, w.numax, w.cube, w.h, out=ozf, handle=handle, stream=stream,
                          prec="ff64")
        api.add_bloch(hzf, cz, kvec, pos, sig, w.numax, w.cube, w.h, handle=handle, stream=stream, prec="ff64")

    msf = _time_steps(stream, bloch_ff_step, warmup=2, steps=10)
    err_b = float(torch.linalg.vector_norm(torch.view_as_real(ozf - oz)) / torch.linalg.vector_norm(torch.view_as_real(oz)))
    out["bloch_complex_ff64"] = {"value": round(bytes_b / (msf * 1e-3) / 1e9, 3), "unit": "GB/s",
                                 "ms_per_step": round(msf, 4), "project_rel_diff_vs_fp64_form": err_b,
                                 "note": f"same {B} complex bands and k: the FP64-accurate form (float-float passes "
                                         "over the (re, im) pairs, phases turned per run)"}
    zc32, cz32 = zc.to(torch.complex64), cz.to(torch.complex64)
    oz32 = torch.empty_like(cz32)
    hz32 = torch.zeros_like(zc32)

    def bloch_fp32_step():
        api.project_bloch(zc32, kvec, pos, sig, w.numax, w.cube, w.h, out=oz32, handle=handle, stream=stream,
                          prec="fp32")
        api.add_bloch(hz32, cz32, kvec, pos, sig, w.numax, w.cube, w.h, handle=handle, stream=stream, prec="fp32")

    ms32b = _time_steps(stream, bloch_fp32_step, warmup=2, steps=10)
    err_32 = float(torch.linalg.vector_norm(torch.view_as_real(oz32.to(torch.complex128) - oz))
                   / torch.linalg.vector_norm(torch.view_as_real(oz)))
    out["bloch_complex_fp32"] = {"value": round(bytes_b // 2 / (ms32b * 1e-3) / 1e9, 3), "unit": "GB/s",
                                 "ms_per_step": round(ms32b, 4), "project_rel_diff_vs_fp64_form": err_32,
                                 "note": f"same {B} bands and k as complex64: the FP32 CUDA-core kernels over the "
                                         "(re, im) pairs, phases turned per run in FP32"}
    del zc, cz, oz, hz, ozf, hzf, zc32, cz32, oz32, hz32
    torch.cuda.empty_cache()
    return out


# Oracle sample of the 160^3 precision workload: seeded atoms / grid points / band subset whose GPU results
# the precision-forms leg keeps, and whose FP64 oracle references the CPU-baseline leg computes.
C160_SAMPLE = dict(natoms=6, npoints=400, nbands=64, seed=1603)


def _c160_sample_indices(w):
    rng = np.random.default_rng(C160_SAMPLE["seed"])
    sel = np.sort(rng.choice(w.natoms, size=C160_SAMPLE["natoms"], replace=False))
    pts = np.sort(rng.choice(w.grid[0] * w.grid[1] * w.grid[2], size=C160_SAMPLE["npoints"], replace=False))
    return sel, pts


def precision_forms(api, handle, stream, modes=("fp32", "tf32", "3xtf32", "bf16", "split_fp16"),
                    storages=("f32", "bf16"), steps=5):
    """The 160^3 / 512-atom / numax 7 / 256-band workload in every reduced-precision form: project +
    expand throughput, the error against the plain FP64 SHO form run on the same GPU on the same
    storage-rounded psi (norm-wise over all coefficients / the whole expanded grid), and each form's results
    on the oracle sample (returned separately; the CPU-baseline leg compares them with the FP64 oracle)."""
    import torch
    w = workloads.WORKLOADS["c160"]
    pos, sig = workloads.atoms(w)
    nst = api.nstates(w.numax)
    alg = algorithmic(w, pos, nst, elem=4)
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev)
    g.manual_seed(w.seed)
    nx, ny, nz = w.grid
    cin = torch.randn((w.natoms, nst, w.nbands), generator=g, device=dev, dtype=torch.float32)
    sel, pts = _c160_sample_indices(w)
    nbs = C160_SAMPLE["nbands"]
    sel_d, pts_d = torch.as_tensor(sel, device=dev), torch.as_tensor(pts, device=dev)
    samples = {"w": w, "pos": pos, "sig": sig, "sel": sel, "pts": pts, "cin": cin[:, :, :nbs].double().cpu().numpy(),
               "psi": {}, "got": {}}
    out = {"workload": "periodic 160^3, h=0.2, 512 atoms, numax 7 (120 states), cube 32, 256 bands",
           "reference": "FP64 SHO form on the same GPU, same storage-rounded psi (err_project / err_expand); "
                        "FP64 oracle on a seeded sample (err_oracle_*, filled in by the CPU-baseline leg)",
           "oracle_sample": f"{len(sel)} atoms and {len(pts)} grid points, bands 0..{nbs - 1}",
           "union_cube_points": alg["union_points"], "forms": {}}
    for st in storages:
        tdt = torch.float32 if st == "f32" else torch.bfloat16
        psi = torch.randn((nz, ny, nx, w.nbands), generator=g, device=dev, dtype=torch.float32).to(tdt)
        samples["psi"][st] = psi[..., :nbs].float().cpu().numpy()   # storage-rounded values, exactly
        # FP64 references of this storage
        psi64 = psi.double()
        c_ref = api.project(psi64, pos, sig, w.numax, w.cube, w.h, w.periodic, prec="fp64", handle=handle,
                            stream=stream)
        del psi64
        e_ref = torch.zeros((nz, ny, nx, w.nbands), dtype=torch.float64, device=dev)
        api.add(e_ref, cin.double(), pos, sig, w.numax, w.cube, w.h, w.periodic, prec="fp64", handle=handle,
                stream=stream)
        elem = 4 if st == "f32" else 2
        bytes_step = alg["bytes_prj"] * elem // 4 + alg["bytes_add"] * elem // 4
        coeff = torch.empty((w.natoms, nst, w.nbands), dtype=torch.float32, device=dev)
        hpsi = torch.zeros_like(psi)
        for mode in modes:
            def step():
                api.project(psi, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=mode, out=coeff, handle=handle,
                            stream=stream)
                api.add(hpsi, cin, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=mode, handle=handle,
                        stream=stream)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            step()
            torch.cuda.synchronize()
            t_prj, t_add = [], []
            for _ in range(steps):
                ev[0].record(stream)
                api.project(psi, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=mode, out=coeff, handle=handle,
                            stream=stream)
                ev[1].record(stream)
                api.add(hpsi, cin, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=mode, handle=handle,
                        stream=stream)
                ev[2].record(stream)
                torch.cuda.synchronize()
                t_prj.append(ev[0].elapsed_time(ev[1]))
                t_add.append(ev[1].elapsed_time(ev[2]))
            ms = float(np.median(t_prj) + np.median(t_add))
            err_c = float(torch.linalg.vector_norm(coeff.double() - c_ref) / torch.linalg.vector_norm(c_ref))
            hpsi.zero_()
            api.add(hpsi, cin, pos, sig, w.numax, w.cube, w.h, w.periodic, prec=mode, handle=handle, stream=stream)
            err_e = float(torch.linalg.vector_norm(hpsi.double() - e_ref) / torch.linalg.vector_norm(e_ref))
            samples["got"][f"{st}/{mode}"] = (
                coeff.index_select(0, sel_d)[:, :, :nbs].double().cpu().numpy(),
                hpsi.reshape(-1, w.nbands).index_select(0, pts_d)[:, :nbs].double().cpu().numpy())
            gbs = bytes_step / (ms * 1e-3) / 1e9
            out["forms"][f"{st}/{mode}"] = {
                "ms_project": round(float(np.median(t_prj)), 4), "ms_expand": round(float(np.median(t_add)), 4),
                "GB/s": round(gbs, 2), "hbm_frac": round(gbs / _peaks().get("hbm_gbs", 6793.4), 4),
                "err_project": err_c, "err_expand": err_e}
            hpsi.zero_()
        del psi, hpsi, e_ref, c_ref
        torch.cuda.empty_cache()
    return out, samples


def oracle_precision_errors(prec_out, samples):
    """CPU-baseline leg: the FP64 oracle on the precision workload's sample (storage-rounded psi) and each
    form's norm-wise error against it; also the oracle's time for this sample."""
    import oracle
    w, sel, pts = samples["w"], samples["sel"], samples["pts"]
    pos, sig = samples["pos"], samples["sig"]
    t0 = time.perf_counter()
    ref_e = oracle.expand_points(w.grid, w.h, w.periodic, pos, sig, w.numax, w.cube, samples["cin"], pts)
    secs = time.perf_counter() - t0
    for st, psi in samples["psi"].items():
        psi64 = psi.astype(np.float64)
        t0 = time.perf_counter()
        ref_c = oracle.project(w.grid, w.h, w.periodic, psi64, pos[sel], sig[sel], w.numax, w.cube)
        secs += time.perf_counter() - t0
        del psi64
        for key, (got_c, got_e) in samples["got"].items():
            if not key.startswith(st + "/"):
                continue
            ent = prec_out["forms"][key]
            ent["err_oracle_project"] = float(max(np.linalg.norm(got_c[i] - ref_c[i]) / np.linalg.norm(ref_c[i])
                                                  for i in range(len(sel))))
            ent["err_oracle_expand"] = float(np.linalg.norm(got_e - ref_e) / np.linalg.norm(ref_e))
    prec_out["oracle_seconds"] = round(secs, 3)
    # the oracle's own speed on a seeded 64-atom x 32-band subset of the workload (FP32-stored psi)
    psi32 = samples["psi"].get("f32")
    if psi32 is not None:
        rng = np.random.default_rng(C160_SAMPLE["seed"] + 1)
        sub = np.sort(rng.choice(w.natoms, size=64, replace=False))
        psi64 = np.ascontiguousarray(psi32[..., :32], dtype=np.float64)
        cin = np.ascontiguousarray(samples["cin"][sub][:, :, :32])
        t0 = time.perf_counter()
        oracle.project(w.grid, w.h, w.periodic, psi64, pos[sub], sig[sub], w.numax, w.cube)
        t1 = time.perf_counter()
        oracle.add(w.grid, w.h, w.periodic, np.zeros_like(psi64), pos[sub], sig[sub], w.numax, w.cube, cin)
        t2 = time.perf_counter()
        sw = workloads.Workload(**{**w.__dict__, "natoms": 64, "nbands": 32})
        a = algorithmic(sw, pos[sub], oracle.nstates(w.numax), elem=4)
        prec_out["oracle_subset_timing"] = {
            "sample": "64 seeded atoms x 32 bands of the 160^3 workload, FP64 direct summation",
            "project_s": round(t1 - t0, 3), "add_s": round(t2 - t1, 3), "cores": oracle.set_threads(0),
            "GB/s": round((a["bytes_prj"] + a["bytes_add"]) / (t2 - t0) / 1e9, 5)}
    prec_out["err_oracle_note"] = ("project: largest per-atom norm-wise error over the sampled atoms; expand: "
                                   "norm-wise over the sampled points (expansion into zero psi of the storage type)")


def serving_bench(api, nsys=12, warm=200, measured=1000, loads=(0.5, 0.8, 0.95), slots=4, sweep=(8, 16),
                  prec="fp32", nsample=20):
    """Poisson stream of project / expand requests (50/50) over heterogeneous device-resident systems
    (grid 48^3..192^3, 8..1024 atoms, 16..512 bands, numax 3/5/7/9, FP32 psi).  Capacity = completed
    requests per second of a saturating burst; each offered load rho submits `measured` requests at
    rate rho * capacity after `warm` warm-up requests.  Latency = submit -> completion as recorded by the
    server, per request; slowdown = latency / the same request's latency alone; GB/s = algorithmic psi +
    coefficient bytes of the completed requests / busy wall time.  The slot count is swept at rho = 0.8.
    A seeded sample of `nsample` served requests (2 % of the measured stream) keeps its inputs and results
    (16 bands) for the CPU-baseline leg to check against the FP64 oracle."""
    import torch
    from paper_1905_00480_gb300.serve import Server
    specs = workloads.serving_systems(nsys)
    geo = []
    for sp in specs:
        rng = np.random.default_rng(sp.seed)
        L = sp.grid * sp.h
        geo.append(workloads.random_atoms(rng, sp.natoms, (L, L, L), True, min_sep=1.0))

    def start(nslots):
        srv = Server(torch.cuda.current_device(), budget_bytes=96 << 30, slots=nslots)
        ids = []
        for sp, (pos, sig) in zip(specs, geo):
            g = torch.Generator(device="cuda")
            g.manual_seed(sp.seed)
            psi = torch.randn((sp.grid, sp.grid, sp.grid, sp.nbands), generator=g, device="cuda", dtype=torch.float32)
            ids.append(srv.register(psi, pos, sig, sp.numax, sp.cube, sp.h, sp.periodic))
            del psi
        torch.cuda.empty_cache()
        return srv, ids

    rng = np.random.default_rng(SERVE_SEED)

    def draw(n):
        return [(int(rng.integers(len(specs))), "project" if rng.random() < 0.5 else "expand") for _ in range(n)]

    def run_burst(srv, ids, reqs):
        t0 = time.perf_counter()
        ts = [srv.submit(ids[i], op, prec) for i, op in reqs]
        for t in ts:
            srv.wait(t, 600000)
        return time.perf_counter() - t0

    def run_load(srv, ids, cap, rho):
        srv.reset_stats()
        reqs = draw(measured)
        arrivals = workloads.poisson_arrivals(rng, measured, rho * cap)
        t0 = time.perf_counter()
        ts = []
        for (i, op), ta in zip(reqs, arrivals):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ts.append(srv.submit(ids[i], op, prec))
        lat = np.array([srv.wait(t, 600000, with_latency=True)[1] for t in ts])
        return reqs, lat, srv.stats()

    def summary(reqs, lat, st, alone, cap, rho):
        slow = np.array([l / alone[(i, op)] for (i, op), l in zip(reqs, lat)])
        size = np.array([specs[i].grid ** 3 * specs[i].nbands for i, _ in reqs], dtype=np.float64)
        cls = {}
        edges = np.quantile(size, [0.0, 0.5, 0.9, 1.0])
        for name, lo, hi in (("small (below median size)", edges[0], edges[1]),
                             ("medium (median-90 %)", edges[1], edges[2]), ("large (top 10 %)", edges[2], edges[3])):
            m = (size >= lo) & (size <= hi) if name.startswith("large") else (size >= lo) & (size < hi)
            if m.any():
                cls[name] = {"requests": int(m.sum()), "p50_ms": round(float(np.percentile(lat[m], 50)), 3),
                             "p99_ms": round(float(np.percentile(lat[m], 99)), 3),
                             "alone_p50_ms": round(float(np.median([alone[r] for r, k in zip(reqs, m) if k])), 3)}
        p50, p99 = float(np.percentile(lat, 50)), float(np.percentile(lat, 99))
        return {"offered_rps": round(rho * cap, 2), "p50_ms": round(p50, 3), "p99_ms": round(p99, 3),
                "p99_over_p50": round(p99 / p50, 2), "mean_ms": round(float(lat.mean()), 3),
                "max_ms": round(float(lat.max()), 3), "slowdown_p50": round(float(np.percentile(slow, 50)), 2),
                "slowdown_p99": round(float(np.percentile(slow, 99)), 2), "by_size": cls,
                "completed": st["completed"], "failed": st["failed"], "gbs": round(st["gbs"], 2),
                "max_inflight": st["max_inflight"], "peak_gb": round(st["peak_bytes"] / 1e9, 2)}

    srv, ids = start(slots)
    run_burst(srv, ids, draw(warm))
    # every request type alone (median of three), the denominator of the slowdown
    alone = {}
    for i in range(len(specs)):
        for op in ("project", "expand"):
            ls = []
            for _ in range(3):
                ls.append(srv.wait(srv.submit(ids[i], op, prec), 600000, with_latency=True)[1])
            alone[(i, op)] = float(np.median(ls))
    nburst = 400
    cap = nburst / run_burst(srv, ids, draw(nburst))
    out = {"systems": [dict(grid=sp.grid, atoms=sp.natoms, bands=sp.nbands, numax=sp.numax) for sp in specs],
           "slots": slots, "precision": prec, "capacity_rps": round(cap, 2), "warmup_requests": warm,
           "measured_requests": measured, "loads": {}, "slot_sweep_rho_0.8": {}}
    for rho in loads:
        reqs, lat, st = run_load(srv, ids, cap, rho)
        out["loads"][str(rho)] = summary(reqs, lat, st, alone, cap, rho)
    # seeded 2 % sample of served requests, inputs and results kept (16 bands) for the oracle check
    srng = np.random.default_rng(SERVE_SEED + 1)
    sample = []
    for k in range(nsample):
        i = int(srng.integers(len(specs)))
        op = "project" if srng.random() < 0.5 else "expand"
        sp = specs[i]
        pos, sig = geo[i]
        # a fresh copy of the system (the stream's alternating projections and expansions grow psi by about
        # the projector's norm each cycle, so long-served systems leave the FP32 range), N(0, 1) coefficients
        g = torch.Generator(device="cuda")
        g.manual_seed(sp.seed + 7777 + k)
        psi_k = torch.randn((sp.grid,) * 3 + (sp.nbands,), generator=g, device="cuda", dtype=torch.float32)
        sid = srv.register(psi_k, pos, sig, sp.numax, sp.cube, sp.h, sp.periodic)
        del psi_k
        srv.write_coeff(sid, torch.randn((sp.natoms, api.nstates(sp.numax), sp.nbands), generator=g,
                                         dtype=torch.float32, device="cuda").cpu())
        p0, c0 = srv.read(sid)
        assert srv.wait(srv.submit(sid, op, prec), 600000) == 0
        p1, c1 = srv.read(sid)
        srv.unregister(sid)
        rec = {"grid": (sp.grid,) * 3, "h": sp.h, "numax": sp.numax, "cube": sp.cube, "op": op}
        if op == "project":
            sel = np.sort(srng.choice(sp.natoms, size=min(2, sp.natoms), replace=False))
            rec.update(psi=p0[..., :16].double().numpy(), pos=pos[sel], sig=sig[sel],
                       got=c1[torch.as_tensor(sel)][:, :, :16].double().numpy())
        else:
            pts = np.sort(srng.choice(sp.grid ** 3, size=50, replace=False))
            d = (p1.reshape(-1, sp.nbands)[torch.as_tensor(pts)] - p0.reshape(-1, sp.nbands)[torch.as_tensor(pts)])
            rec.update(pos=pos, sig=sig, coeff=c0[:, :, :16].double().numpy(), pts=pts, got=d[:, :16].double().numpy())
        sample.append(rec)
        del p0, c0, p1, c1
    srv.close()
    torch.cuda.empty_cache()
    for ns in sweep:
        srv, ids = start(ns)
        run_burst(srv, ids, draw(warm // 2))
        capn = nburst / run_burst(srv, ids, draw(nburst))
        reqs, lat, st = run_load(srv, ids, capn, 0.8)
        ent = summary(reqs, lat, st, alone, capn, 0.8)
        ent["capacity_rps"] = round(capn, 2)
        ent.pop("by_size")
        out["slot_sweep_rho_0.8"][str(ns)] = ent
        srv.close()
        torch.cuda.empty_cache()
    out["slot_sweep_rho_0.8"][str(slots)] = {k: v for k, v in out["loads"]["0.8"].items() if k != "by_size"}
    out["slot_sweep_rho_0.8"][str(slots)]["capacity_rps"] = out["capacity_rps"]
    return out, sample


def oracle_serving_errors(serving_out, sample):
    """CPU-baseline leg: the served sample against the FP64 oracle (storage-rounded FP32 inputs)."""
    import oracle
    errs = {"project": [], "expand": []}
    for rec in sample:
        if rec["op"] == "project":
            ref = oracle.project(rec["grid"], rec["h"], True, rec["psi"], rec["pos"], rec["sig"], rec["numax"],
                                 rec["cube"])
            errs["project"].append(float(np.linalg.norm(rec["got"] - ref) / np.linalg.norm(ref)))
        else:
            ref = oracle.expand_points(rec["grid"], rec["h"], True, rec["pos"], rec["sig"], rec["numax"], rec["cube"],
                                       rec["coeff"], rec["pts"])
            errs["expand"].append(float(np.linalg.norm(rec["got"] - ref) / max(np.linalg.norm(ref), 1e-300)))
    serving_out["oracle_sample"] = {
        "requests": len(sample), "sample": "seeded 2 % of the measured stream, 16 bands; projections on 2 atoms, "
                                           "expansions at 50 grid points",
        "max_rel_norm_project": max(errs["project"], default=None),
        "max_rel_norm_expand": max(errs["expand"], default=None), "tolerance": 2e-6}


SERVE_SEED = 4242


def forces_bench(api, handle, stream, steps=5):
    """Differentiation workload: periodic 128^3, 128 atoms, numax 5, 64 bands FP32; E = sum D c^2 with
    D ~ U[-1,1].  Times one forward (projection) + backward (forces and dE/dpsi = h^3 E(2 D c)) through the
    autograd Function, and states the error of the FP32 forces against the FP64 form on the same GPU."""
    import torch
    from paper_1905_00480_gb300.autograd import sho_project
    w = workloads.WORKLOADS["c128"]
    pos, sig = workloads.atoms(w)
    N = api.nstates(w.numax)
    D = torch.from_numpy(workloads.dmatrix_host(w, N)).cuda().float()
    psi = workloads.psi_device(w).requires_grad_(True)
    sig_t = torch.from_numpy(sig)

    def step():
        X = torch.tensor(pos, dtype=torch.float64, requires_grad=True)
        c = sho_project(psi, X, sig_t, w.numax, w.cube, w.h, w.periodic, prec="fp32")
        E = (D[:, :, None] * c * c).sum()
        E.backward()
        return X.grad, c.detach()

    F, c = step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        psi.grad = None
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    dEdc64 = (2.0 * D[:, :, None] * c).double()
    F64 = api.forces(psi.detach().double(), dEdc64.contiguous(), pos, sig, w.numax, w.cube, w.h, w.periodic,
                     prec="ff64").cpu()
    err = float((F - F64).abs().max() / F64.abs().max())
    return {"workload": "periodic 128^3, h=0.2, 128 atoms, numax 5, cube 32, 64 bands FP32, E = sum D c^2",
            "ms_forward_backward": round(ms, 4), "forces_err_vs_fp64_form": err,
            "note": "forward projection + backward (forces via the numax+1 projection, dE/dpsi via the "
                    "expansion) through torch.autograd; finite-difference and oracle checks are in the tests"}


def _oracle_sample(w, pos, sig, nsel, nbands_sel, seed=5):
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(w.natoms, size=nsel, replace=False))
    return sel, nbands_sel


def cpu_baseline(w, pos, sig, psi_d, cin_d, coeff_d, hpsi_ref, api, handle, prec="ff64"):
    """Time the FP64 oracle, as it stands, on the workload (all atoms and bands: about ten seconds of
    host work on 16 cores) and state the GPU error against it."""
    import oracle
    sel, _ = _oracle_sample(w, pos, sig, w.natoms, w.nbands)
    psi = psi_d.cpu().numpy()
    cin = cin_d.cpu().numpy()
    sw = workloads.Workload(**{**w.__dict__, "natoms": len(sel)})
    alg = algorithmic(sw, pos[sel], api.nstates(w.numax))
    t0 = time.perf_counter()
    ref_c = oracle.project(w.grid, w.h, w.periodic, psi, pos[sel], sig[sel], w.numax, w.cube)
    t1 = time.perf_counter()
    out = oracle.add(w.grid, w.h, w.periodic, np.zeros_like(psi), pos[sel], sig[sel], w.numax, w.cube, cin[sel])
    t2 = time.perf_counter()
    secs = t2 - t0
    cores = oracle.set_threads(0)
    # one core, on two atoms (scaled per byte like the all-core figure)
    sel1 = sel[:2]
    alg1 = algorithmic(workloads.Workload(**{**w.__dict__, "natoms": len(sel1)}), pos[sel1], api.nstates(w.numax))
    oracle.set_threads(1)
    t3 = time.perf_counter()
    oracle.project(w.grid, w.h, w.periodic, psi, pos[sel1], sig[sel1], w.numax, w.cube)
    oracle.add(w.grid, w.h, w.periodic, np.zeros_like(psi), pos[sel1], sig[sel1], w.numax, w.cube, cin[sel1])
    t4 = time.perf_counter()
    oracle.set_threads(cores)
    one_core = (alg1["bytes_prj"] + alg1["bytes_add"]) / (t4 - t3) / 1e9
    got_c = coeff_d.cpu().numpy()[sel]
    err_c = float(np.linalg.norm(got_c - ref_c) / np.linalg.norm(ref_c))
    # GPU expansion of the same atoms into zeros
    import torch
    z = torch.zeros_like(psi_d)
    api.add(z, cin_d[torch.as_tensor(sel, device=cin_d.device)].contiguous(), pos[sel], sig[sel], w.numax, w.cube,
            w.h, w.periodic, prec=prec, handle=handle)
    err_a = float(np.linalg.norm(z.cpu().numpy() - out) / np.linalg.norm(out))
    base = {"value": round((alg["bytes_prj"] + alg["bytes_add"]) / secs / 1e9, 5), "unit": "GB/s", "cores": cores,
            "kind": "oracle", "seconds": round(secs, 3), "project_s": round(t1 - t0, 3), "add_s": round(t2 - t1, 3),
            "one_core_value": round(one_core, 5), "one_core_sample": "2 atoms, all bands",
            "sample": f"{len(sel)} of {w.natoms} atoms (all {w.nbands} bands), project + expand, FP64 direct "
                      "summation over fully sampled 3D projectors"}
    err = {"project_rel_norm": err_c, "expand_rel_norm": err_a, "tolerance": 1e-12, "form": prec,
           "sample": f"{len(sel)} atoms"}
    return base, err


# ----------------------------------------------------------------------------------- the paper's Table 1
# Timings of Table 1 (Sec. 6), seconds for 10 executions of one kernel: (#, USUprj, SHOprj, USUadd, SHOadd);
# None where the paper has no SHO entry (no SHO basis has 18 states).  Printed next to the GB300 figures as
# context only: other GPUs, other kernels.
PAPER_TABLE1 = {
    "P100": [(1, 0.480, 0.453, 0.274, 0.187), (4, 0.834, 0.471, 0.803, 0.363), (10, 1.259, 0.430, 1.820, 0.520),
             (18, 2.080, None, 3.173, None), (20, 2.366, 0.482, 3.511, 0.733), (35, 3.904, 0.967, 6.052, 1.027),
             (56, 6.058, 1.214, 9.625, 1.455)],
    "V100": [(1, 0.291, 0.271, 0.140, 0.118), (4, 0.354, 0.310, 0.378, 0.189), (10, 0.555, 0.284, 0.823, 0.277),
             (18, 0.830, None, 1.411, None), (20, 1.013, 0.300, 1.557, 0.398), (35, 2.087, 0.575, 2.660, 0.564),
             (56, 1.806, 0.793, 4.208, 0.792)],
}


def _median_ms(stream, fn, reps, runs):
    """The paper's protocol, shortened: one untimed run, then `runs` timed runs of `reps` executions each;
    returns the median over runs of the time per execution (ms)."""
    import torch
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    per = []
    for _ in range(runs):
        ev[0].record(stream)
        for _ in range(reps):
            fn()
        ev[1].record(stream)
        ev[1].synchronize()
        per.append(ev[0].elapsed_time(ev[1]) / reps)
    return float(np.median(per))


def _clipped_cube_points(grid, h, cube, pos, rprj=0.0):
    """Grid points inside the (non-periodic) domain summed over the atoms' cubes; with rprj > 0 only the
    points inside each atom's projection sphere ((ux^2 + uy^2) + uz^2 <= rprj^2)."""
    tot = 0
    for X in pos:
        o = np.floor(X / h).astype(int) - cube // 2 + 1
        idx = [o[d] + np.arange(cube) for d in range(3)]
        ins = [(j >= 0) & (j < grid[d]) for d, j in enumerate(idx)]
        if rprj > 0:
            u = [idx[d] * h - X[d] for d in range(3)]
            r2 = (u[0][None, None, :] * u[0][None, None, :] + u[1][None, :, None] * u[1][None, :, None]) + \
                u[2][:, None, None] * u[2][:, None, None]
            m = (r2 <= rprj * rprj) & ins[0][None, None, :] & ins[1][None, :, None] & ins[2][:, None, None]
            tot += int(m.sum())
        else:
            tot += int(ins[0].sum()) * int(ins[1].sum()) * int(ins[2].sum())
    return tot


def paper_table1(args):
    """SHO (generated on the fly) against stored projector values (USU) on the paper's benchmark system:
    64^3 grid at 0.25 A, the 665 fcc atoms (a = 4.08 A) whose 3.55 A sphere touches the 16 A domain,
    1024 FP64 wave functions, not periodic, cube 32 (Sec. 6, Tables 1 and 2)."""
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, pos, sig = workloads.fcc_paper_geometry()
    cube, B = 32, 1024
    dev = torch.device("cuda", 0)
    handle = api.Handle(0)
    # the paper's projection spheres (R_prj = 3.55 A): SHO FP64 / FP64-accurate and the stored projectors use
    # only the cube points inside them; the FP32-class SHO forms have no sphere support and keep the cube
    rprj = args.table_sphere * workloads.ANGSTROM if args.table_sphere > 0 else 0.0
    handle.set_support_radius(rprj)
    cube_handle = api.Handle(0)
    stream = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(workloads.SEED_BASE + 6)
    psi = torch.randn((grid[2], grid[1], grid[0], B), generator=g, device=dev, dtype=torch.float64)
    hpsi = torch.zeros_like(psi)
    A = len(pos)
    pts = _clipped_cube_points(grid, h, cube, pos, rprj)
    sho_reps, usu_reps, runs = args.table_reps, 1, args.table_runs
    rows = []
    sho = {}
    for nu in range(6):
        N = api.nstates(nu)
        coeff = torch.empty((A, N, B), dtype=torch.float64, device=dev)
        cin = torch.randn((A, N, B), generator=g, device=dev, dtype=torch.float64)
        for prec in ("fp64", "ff64"):
            t_prj = _median_ms(stream, lambda: api.project(psi, pos, sig, nu, cube, h, False, prec=prec, out=coeff,
                                                           handle=handle, stream=stream), sho_reps, runs)
            t_add = _median_ms(stream, lambda: api.add(hpsi, cin, pos, sig, nu, cube, h, False, prec=prec,
                                                       handle=handle, stream=stream), sho_reps, runs)
            sho[(N, prec)] = (t_prj, t_add)
        del coeff, cin
    usu = {}
    check = {}
    for N in (1, 4, 10, 18, 20, 35, 56):
        nu = next(v for v in range(6) if api.nstates(v) >= N)
        proj = api.usu_build(pos, sig, nu, cube, grid, h, False, device=0, handle=handle, stream=stream, nproj=N)
        coeff = torch.empty((A, N, B), dtype=torch.float64, device=dev)
        cin = torch.randn((A, N, B), generator=g, device=dev, dtype=torch.float64)
        t_prj = _median_ms(stream, lambda: api.usu_project(psi, proj, pos, sig, nu, cube, h, False, out=coeff,
                                                           handle=handle, stream=stream), usu_reps, runs)
        t_add = _median_ms(stream, lambda: api.usu_add(hpsi, cin, proj, pos, sig, nu, cube, h, False, handle=handle,
                                                       stream=stream), usu_reps, runs)
        usu[N] = (t_prj, t_add, proj.numel() * 8)
        if api.nstates(nu) == N:
            ref = api.project(psi, pos, sig, nu, cube, h, False, prec="ff64", handle=handle, stream=stream)
            check[N] = float((ref - coeff).norm() / ref.norm())
        del proj, coeff, cin
        torch.cuda.empty_cache()
    flop_usu = lambda N: 2.0 * pts * N * B
    for N in (1, 4, 10, 18, 20, 35, 56):
        up, ua, pbytes = usu[N]
        row = {"n": N, "usu_prj_ms": round(up, 3), "usu_add_ms": round(ua, 3),
               "usu_projector_gb": round(pbytes / 1e9, 3),
               "usu_fp64_tflops": [round(flop_usu(N) / (up * 1e-3) / 1e12, 3),
                                   round(flop_usu(N) / (ua * 1e-3) / 1e12, 3)]}
        for prec in ("fp64", "ff64"):
            if (N, prec) in sho:
                sp, sa = sho[(N, prec)]
                row[f"sho_{prec}_prj_ms"] = round(sp, 3)
                row[f"sho_{prec}_add_ms"] = round(sa, 3)
                row[f"S_{prec}"] = [round(up / sp, 2), round(ua / sa, 2)]
        if N in check:
            row["sho_ff64_vs_usu_rel_norm"] = check[N]
        rows.append(row)
    fair = {}
    up, ua, _ = usu[18]
    for prec in ("fp64", "ff64"):
        sp, sa = sho[(35, prec)]
        fair[prec] = {"prj": round(up / sp, 2), "add": round(ua / sa, 2), "both": round((up + ua) / (sp + sa), 2)}
    # float (Table 2, left half): FP32 psi, stored FP32 projectors against the FP32 SHO forms
    del hpsi
    torch.cuda.empty_cache()
    psi32 = psi.float()
    del psi
    hpsi32 = torch.zeros_like(psi32)
    flt = {}
    for N in (1, 4, 10, 18, 20, 35, 56):
        nu = next(v for v in range(6) if api.nstates(v) >= N)
        proj = api.usu_build(pos, sig, nu, cube, grid, h, False, device=0, handle=handle, stream=stream, nproj=N,
                             dtype=torch.float32)
        coeff = torch.empty((A, N, B), dtype=torch.float32, device=dev)
        cin = torch.randn((A, N, B), generator=g, device=dev, dtype=torch.float32)
        ent = {"usu_prj_ms": round(_median_ms(stream, lambda: api.usu_project(psi32, proj, pos, sig, nu, cube, h, False,
                                                                           out=coeff, handle=handle, stream=stream),
                                             usu_reps, runs), 3),
               "usu_add_ms": round(_median_ms(stream, lambda: api.usu_add(hpsi32, cin, proj, pos, sig, nu, cube, h,
                                                                       False, handle=handle, stream=stream),
                                             usu_reps, runs), 3)}
        del proj, coeff, cin
        if api.nstates(nu) == N:
            cfull = torch.randn((A, N, B), generator=g, device=dev, dtype=torch.float32)
            for prec in ("fp32", "tf32"):
                ent[f"sho_{prec}_prj_ms"] = round(_median_ms(stream, lambda: api.project(
                    psi32, pos, sig, nu, cube, h, False, prec=prec, handle=cube_handle, stream=stream), sho_reps,
                    runs), 3)
                ent[f"sho_{prec}_add_ms"] = round(_median_ms(stream, lambda: api.add(
                    hpsi32, cfull, pos, sig, nu, cube, h, False, prec=prec, handle=cube_handle, stream=stream),
                    sho_reps, runs), 3)
            del cfull
        flt[N] = ent
        torch.cuda.empty_cache()
    for prec in ("fp32", "tf32"):
        sp, sa = flt[35][f"sho_{prec}_prj_ms"], flt[35][f"sho_{prec}_add_ms"]
        up, ua = flt[18]["usu_prj_ms"], flt[18]["usu_add_ms"]
        fair[f"float_{prec}"] = {"prj": round(up / sp, 2), "add": round(ua / sa, 2),
                                 "both": round((up + ua) / (sp + sa), 2)}
    paper_fair = {"P100": {"prj": 2.2, "add": 3.1, "both": 2.6}, "V100": {"prj": 1.4, "add": 2.5, "both": 2.0}}
    paper_fair_float = {"P100": {"prj": 2.3, "add": 2.9, "both": 2.7}, "V100": {"prj": 1.4, "add": 1.7, "both": 1.6}}
    return {
        "metric": "SHO vs stored-projector (USU) kernel time and speedup S = USU/SHO, the paper's Tables 1 and 2",
        "unit": "ms per execution", "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"fcc a=4.08 A, 16 A cube at h=0.25 A (64^3), {A} atoms touching (3.55 A), "
                               f"sigma 0.59 Bohr, {B} bands FP64 N(0,1), not periodic, cube 32",
                   "protocol": f"one untimed run, median of {runs} runs of {sho_reps} (SHO) / {usu_reps} (USU) "
                               "executions; psi 2.1 GB > L2",
                   "support": (f"sphere R_prj = {args.table_sphere} A ({rprj:.4f} Bohr) inside the 32-point cube for "
                               "SHO FP64/FF64 and both stored-projector tables (zeros stored outside); SHO FP32/TF32 "
                               "on the whole cube") if rprj > 0 else "whole 32-point cube for every kernel",
                   "support_points": pts, "support_points_note": "grid points of all atoms' supports (sphere "
                   "and domain); the stored-projector FLOP rates count 2 flop per point, projector and band"},
        "rows": rows, "float_rows": flt, "fair_usu18_vs_sho35": fair,
        "paper_fair_usu18_vs_sho35_double": paper_fair, "paper_fair_usu18_vs_sho35_float": paper_fair_float,
        "paper_table1_s_per_10_executions": PAPER_TABLE1,
    }


# ----------------------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import oracle
    w = workloads.WORKLOADS[WORKLOAD]
    pos, sig = workloads.atoms(w)
    N = oracle.nstates(w.numax)
    rng = np.random.default_rng([w.seed, 1])
    psi = rng.standard_normal((w.grid[2], w.grid[1], w.grid[0], w.nbands))
    cin = rng.standard_normal((w.natoms, N, w.nbands))
    nsel = 2  # atoms per timed step: a bounded sample so the whole run takes a few minutes
    sel_all = np.arange(w.natoms)
    sw = workloads.Workload(**{**w.__dict__, "natoms": nsel})

    def step(i):
        sel = sel_all[(i * nsel) % w.natoms:(i * nsel) % w.natoms + nsel]
        oracle.project(w.grid, w.h, w.periodic, psi, pos[sel], sig[sel], w.numax, w.cube)
        oracle.add(w.grid, w.h, w.periodic, psi, pos[sel], sig[sel], w.numax, w.cube, cin[sel])
        return sel

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    byts = 0
    for i in range(args.steps):
        sel = step(args.warmup + i)
        a = algorithmic(sw, pos[sel], N)
        byts += a["bytes_prj"] + a["bytes_add"]
    secs = time.perf_counter() - t0
    cores = oracle.set_threads(0)
    value = byts / secs / 1e9
    return {
        "impl": "reference",
        "metric": METRIC, "value": round(value, 5), "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "periodic 96^3 grid, h=0.2, 64 atoms, sigma U[0.5,1], numax 5, cube 32^3, 128 bands, "
                               "FP64: project then expand"},
        "cpu_baseline": {"value": round(value, 5), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{nsel} atoms (all bands) per step of the 64-atom workload"},
        "e2e": {"value": round(value, 5), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-same-gpu-baselines", action="store_true")
    ap.add_argument("--no-precision-forms", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-forces", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--prec", default=None, choices=["fp64", "ff64", "fp32", "tf32", "3xtf32", "bf16", "split_fp16"])
    ap.add_argument("--storage", default=None, choices=["f64", "f32", "bf16"])
    ap.add_argument("--bands", type=int, default=0)
    ap.add_argument("--paper-table1", action="store_true",
                    help="time SHO against stored projectors on the paper's fcc benchmark system and exit")
    ap.add_argument("--table-reps", type=int, default=10)
    ap.add_argument("--table-runs", type=int, default=3)
    ap.add_argument("--expand-kernel", default="auto", choices=["auto", "mma_sync", "tcgen05"],
                    help="x-pass engine of the expansion (sho_set_expand_kernel); for the FF64 form auto and "
                         "tcgen05 take the digit-sliced tensor-core x-pass, mma_sync the float-float block gather")
    ap.add_argument("--project-kernel", default="auto", choices=["auto", "mma_sync", "tcgen05"],
                    help="x-pass engine of the FF64 projection (sho_set_project_kernel): auto and mma_sync take "
                         "the float-float kernel, tcgen05 the digit-sliced tensor-core x-pass")
    ap.add_argument("--table-sphere", type=float, default=3.55,
                    help="projection sphere radius in Angstrom for --paper-table1 (0: whole cube)")
    args = ap.parse_args()
    if args.paper_table1:
        print(json.dumps(paper_table1(args)), flush=True)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    ws, rank, local = dist_init()
    if args.impl == "reference":
        res = run_reference(args, ws, rank)
    else:
        res = run_ours(args, ws, rank, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
