#!/usr/bin/env python
"""Benchmark of the Wilson-Dirac hot path on the SU(3) two-index symmetric
(sextet, D_R = 6) 32^3 x 64 workload: m0 = -0.3, links exp(i 0.4 H) followed
by a random Haar gauge transform, antiperiodic in time.

One step is one pass of the whole hot path over one batch of synthetic
input, as an HMC force evaluation of the fermion monomial does it:
  1. represent the fundamental gauge field (FP64 and FP32 stored links),
  2. D_eo applications in FP32 and FP64 (the metric's kernel, event-timed),
  3. mixed-precision CG (FP32 inner, FP64 defect correction) on
     Dhat^dag Dhat x = phi to a true relative residual of 1e-10,
  4. Y = Dhat x and the fermion force of S = phi^dag (Dhat^dag Dhat)^-1 phi.

value: algorithmic ("compulsory") bytes of every hopping-kernel launch of the
step, V/2 (8 L_p + 2 S_p) each, divided by the step's device time -- the
whole step's D_eo-equivalent bandwidth.  roofline: the FP32 D_eo kernel,
bytes per launch over its CUDA-event duration, against the measured HBM copy
bandwidth.  cg: time to 1e-10 of plain FP64 CG vs FP32 / F16 / BF16-inner
defect correction on the same GPU (measured once, after the timed steps).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm: there is no runnable reference code).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "su3_sym_64x32x32x32"
METRIC = "D_eo apply GB/s (% of HBM peak); mixed/batched vs FP64 CG time to residual 1e-10"
UNIT = "GB/s"
TOL = 1e-10


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def hop_bytes(D: int, real_links: bool, prec: int, vh: int) -> int:
    """compulsory bytes of one hopping launch: V/2 (8 L_p + 2 S_p)."""
    cb = [16, 8, 4, 4][prec]
    lp = D * D * (cb // 2 if real_links else cb)
    sp = 4 * D * cb + (4 if prec >= 2 else 0)
    return vh * (8 * lp + 2 * sp)


class Clocks:
    """samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2503_06721_gb300 import build, hr, synth

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    build.build()
    hr.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = synth.WORKLOADS[args.workload]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    vh, D = lat.volume // 2, lat.D
    real = wl.rep == "ADJ"
    # replicas: every rank draws its own field
    import dataclasses
    wl_r = dataclasses.replace(wl, seed=wl.seed + 1000 * rank)
    U = wl_r.links(device=dev)
    phi = synth.gaussian_spinor(vh, D, wl_r.seed + 7, device=dev)
    g = hr.Gauge(lat, U, precs=("f64", "f32"), stored=True)
    stream = torch.cuda.current_stream()
    x32 = phi.to(torch.complex64)
    y32 = torch.empty_like(x32)
    y64 = torch.empty_like(phi)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.deo_per_step)]
    n_deo = args.deo_per_step
    deo_ms = []
    work = {"bytes": 0}

    pev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    phases = {"represent": 0.0, "deo": 0.0, "cg": 0.0, "force": 0.0}

    def step(phi_dev, U_dev):
        pev[0].record(stream)
        g.update(U_dev)
        pev[1].record(stream)
        for k in range(n_deo):
            ev[2 * k].record(stream)
            g.apply(hr.EVEN, hr.F32, x32, out=y32)
            ev[2 * k + 1].record(stream)
        g.apply(hr.EVEN, hr.F64, phi_dev, out=y64)
        pev[2].record(stream)
        x, res, st = g.cg_solve(hr.EO_PRECOND, phi_dev, tol=TOL, max_iter=20000, inner=hr.F32,
                                inner_tol=1e-5)
        pev[3].record(stream)
        Y = g.apply(hr.EO_PRECOND, hr.F64, x)
        F = g.force(hr.EO_PRECOND, x, Y, coeff=-1.0)
        pev[4].record(stream)
        torch.cuda.synchronize()
        for name, a, b in (("represent", 0, 1), ("deo", 1, 2), ("cg", 2, 3), ("force", 3, 4)):
            phases[name] += pev[a].elapsed_time(pev[b])
        r = res[0]
        # hop launches of this step by precision
        h32 = n_deo + 4 * r["iters"]
        h64 = 1 + 4 * (r["outer_iters"] + 1) + 2 + 2
        work["bytes"] += h32 * hop_bytes(D, real, hr.F32, vh) + h64 * hop_bytes(D, real, hr.F64, vh)
        work["res"] = r
        return x, F

    for _ in range(args.warmup):
        step(phi, U)
    torch.cuda.synchronize()
    work["bytes"] = 0
    for k in phases:
        phases[k] = 0.0
    clocks = Clocks(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = hr.launch_count()
    t0.record(stream)
    deo_times = []
    for _ in range(args.steps):
        torch.cuda.nvtx.range_push("hr_step")   # profiler captures select this range
        step(phi, U)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        deo_times += [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n_deo)]
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = hr.launch_count() - n0
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    step_bytes = work["bytes"] / args.steps
    res = work["res"]
    if dist:
        tt = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    ms_per_step = ms / args.steps
    phase_ms = {k: round(v / args.steps, 2) for k, v in phases.items()}
    value = world * step_bytes / (ms_per_step * 1e-3) / 1e9
    deo_ms_avg = sum(deo_times) / len(deo_times)
    deo_bytes = hop_bytes(D, real, hr.F32, vh)
    peak, peak_kind = _peaks()
    achieved = deo_bytes / (deo_ms_avg * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: inputs copied in and the
    # solution and force copied out inside the timed region
    e2e = None
    if not args.no_e2e:
        U_h = U.cpu().pin_memory()
        phi_h = phi.cpu().pin_memory()
        U_d = torch.empty_like(U)
        phi_d = torch.empty_like(phi)
        X_h = torch.empty(phi.shape, dtype=phi.dtype).pin_memory()
        F_h = torch.empty((lat.volume, 4, wl.N ** 2 - 1), dtype=torch.float64).pin_memory()
        work["bytes"] = 0
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(args.steps):
            U_d.copy_(U_h, non_blocking=True)
            phi_d.copy_(phi_h, non_blocking=True)
            x, F = step(phi_d, U_d)
            X_h.copy_(x, non_blocking=True)
            F_h.copy_(F, non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        ems = t0.elapsed_time(t1)
        if dist:
            tt = torch.tensor([ems], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ems = float(tt.item())
        e2e = {"value": world * (work["bytes"] / args.steps) / (ems / args.steps * 1e-3) / 1e9,
               "unit": UNIT, "ms_per_step": ems / args.steps,
               "h2d_bytes_per_step": U_h.numel() * 16 + phi_h.numel() * 16,
               "d2h_bytes_per_step": X_h.numel() * 16 + F_h.numel() * 8}

    # time to 1e-10: plain FP64 CG vs defect correction with low-precision inner solves
    cg = None
    if rank == 0 and not args.no_cg_compare:
        g2 = hr.Gauge(lat, U, precs=("f64", "f32", "f16", "bf16"), stored=True)
        cg = {}
        for name, inner in (("fp64", hr.F64), ("mixed_fp32", hr.F32), ("mixed_fp16", hr.F16),
                            ("mixed_bf16", hr.BF16)):
            g2.cg_solve(hr.EO_PRECOND, phi, tol=1e-3, inner=inner, max_iter=200, check=False)
            torch.cuda.synchronize()
            t0.record(stream)
            x, r, st = g2.cg_solve(hr.EO_PRECOND, phi, tol=TOL, max_iter=20000, inner=inner,
                                   inner_tol=1e-5 if inner == hr.F32 else 2e-3, check=False)
            t1.record(stream)
            torch.cuda.synchronize()
            cg[name] = {"ms": round(t0.elapsed_time(t1), 2), "iters": r[0]["iters"],
                        "outer": r[0]["outer_iters"], "true_rel_residual": r[0]["true_rel_residual"],
                        "status": r[0]["status"]}
        for name in ("mixed_fp32", "mixed_fp16", "mixed_bf16"):
            cg[name]["speedup_vs_fp64"] = round(cg["fp64"]["ms"] / cg[name]["ms"], 2)
        g2.close()

    out = None
    if rank == 0:
        cpu = None if (world > 1 or args.no_cpu_baseline) else cpu_baseline(wl, budget_s=args.cpu_seconds)
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded Philox4x32-10 links exp(i 0.4 H) + Haar gauge transform, "
                    "Gaussian pseudofermion)",
            "config": {"workload": f"SU(3) sextet (SYM, D_R=6) 32^3x64, m0=-0.3, even/odd, "
                                   f"mixed FP32/FP64 CG to 1e-10 + force",
                       "lattice": list(wl.dims), "N": wl.N, "rep": wl.rep, "m0": wl.m0,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (FP32 links 4.8 GB per parity)",
                       "deo_per_step": n_deo, "cg_iters_per_step": res["iters"],
                       "cg_outer_per_step": res["outer_iters"],
                       "true_rel_residual": res["true_rel_residual"]},
            "roofline": {"bound": "hbm", "kernel": "hop_kernel<3,SYM,F32> (D_eo, stored links)",
                         "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": args.traffic, "deo_ms": round(deo_ms_avg, 4),
                         "bytes_per_launch": deo_bytes},
            "gpu_launches": int(launches),
            "phases_ms": phase_ms,
            "clocks": ck,
            "e2e": e2e,
            "cg": cg,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    g.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------

def cpu_baseline(wl, budget_s=15.0, dims=(32, 16, 16, 16)):
    """FP64 oracle D_eo on a 16^3 x 32 sub-lattice of the same workload."""
    import numpy as np

    import oracle
    from paper_2503_06721_gb300 import synth
    oracle.build()
    L = oracle.lat(wl.N, wl.rep, dims, wl.bc, wl.m0)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    UF = synth.random_links(V, wl.N, wl.eps, wl.seed).numpy()
    UR = oracle.represent_field(L, UF)
    D = oracle.rep_dim(wl.N, wl.rep)
    psi = synth.gaussian_spinor(V // 2, D, 5).numpy()
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.hop_parity(L, UR, 0, psi)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (n >= 1 and el * (n + 1) / n > 2 * budget_s):
            break
    byts = hop_bytes(D, wl.rep == "ADJ", 0, V // 2)
    return {"value": round(n * byts / el / 1e9, 3), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle D_eo on a {dims[3]}^3x{dims[0]} sub-lattice of the workload, "
                      f"{n} applications in {el:.1f} s (same compulsory-byte model)"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle's hot path (represent, CG to 1e-10, force)
    on a bounded 8^3 x 16 sample of the workload, per step."""
    if rank != 0:
        return None
    import numpy as np

    import oracle
    from paper_2503_06721_gb300 import synth
    oracle.build()
    wl = synth.WORKLOADS[args.workload]
    dims = (16, 8, 8, 8)
    L = oracle.lat(wl.N, wl.rep, dims, wl.bc, wl.m0)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    D = oracle.rep_dim(wl.N, wl.rep)
    UF = synth.random_links(V, wl.N, wl.eps, wl.seed).numpy()
    phi = synth.gaussian_spinor(V // 2, D, 7).numpy()
    byts = {"b": 0}

    def step():
        UR = oracle.represent_field(L, UF)
        x, ok, it, rr = oracle.cg(L, UR, 1, phi, tol=TOL, max_iter=20000)
        Y = oracle.dhat(L, UR, x)
        Xp = oracle.merge(L, x, oracle.hop_parity(L, UR, 1, x))
        Yp = oracle.merge(L, Y, oracle.hop_parity(L, UR, 1, Y, dagger=True))
        oracle.force(L, UR, Xp, Yp)
        byts["b"] += (4 * (it + 2) + 2 + 2) * hop_bytes(D, wl.rep == "ADJ", 0, V // 2)

    for _ in range(args.warmup):
        step()
    byts["b"] = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = byts["b"] / el / 1e9
    cores = oracle.num_threads()
    sample = (f"FP64 oracle: represent + CG on Dhat^dag Dhat to 1e-10 + force on an "
              f"{dims[3]}^3x{dims[0]} sample of the workload, per step")
    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": "SU(3) sextet (SYM, D_R=6), m0=-0.3, even/odd CG to 1e-10 + force",
                      "lattice": list(dims)},
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def run_deo(args, local_rank):
    """D_eo applications only (for profiler captures): W untimed + K timed."""
    import torch
    from paper_2503_06721_gb300 import build, hr, synth
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    build.build()
    wl = synth.WORKLOADS[args.workload]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    prec = {"f64": hr.F64, "f32": hr.F32, "f16": hr.F16, "bf16": hr.BF16}[args.prec]
    g = hr.Gauge(lat, wl.links(device=dev), precs=(args.prec,), stored=not args.rebuild,
                 rebuild=args.rebuild)
    vh = lat.volume // 2
    n = args.nrhs
    x = synth.gaussian_spinor(vh, lat.D, 3, device=dev, nrhs=n)
    x = x if prec == hr.F64 else (x.to(torch.complex64) if prec == hr.F32 else
                                  hr.field_convert(lat, hr.EVEN, x, hr.F64, prec, n))
    y = g.apply(hr.EVEN, prec, x, nrhs=n)
    for _ in range(args.warmup):
        g.apply(hr.EVEN, prec, x, out=y, nrhs=n)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        g.apply(hr.EVEN, prec, x, out=y, nrhs=n)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    cb = [16, 8, 4, 4][prec]
    sp = 4 * lat.D * cb + (4 if prec >= 2 else 0)
    if args.rebuild:
        lp = wl.N * wl.N * cb
    else:
        lp = lat.D * lat.D * (cb // 2 if wl.rep == "ADJ" else cb)
    # compulsory bytes: every link once, every input and output spinor once
    byts = vh * (8 * lp + 2 * n * sp)
    print(json.dumps({"mode": "deo", "workload": args.workload, "prec": args.prec, "nrhs": n,
                      "links": "rebuild" if args.rebuild else "stored", "ms": round(ms, 4),
                      "GBs": round(byts / (ms * 1e-3) / 1e9, 1), "bytes_per_launch": byts}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--deo-per-step", type=int, default=8)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cg-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--mode", choices=["step", "deo"], default="step",
                    help="deo: only D_eo applications (profiler captures)")
    ap.add_argument("--prec", choices=["f64", "f32", "f16", "bf16"], default="f32")
    ap.add_argument("--rebuild", action="store_true", help="deo mode: rebuild links in-kernel")
    ap.add_argument("--nrhs", type=int, default=1, help="deo mode: right-hand sides per application")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per D_eo launch, when known for the current kernel")
    args = ap.parse_args()
    if args.warmup < 3 and args.mode == "step":
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.mode == "deo":
        run_deo(args, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
