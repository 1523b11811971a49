#!/usr/bin/env python
"""Benchmark of the Wilson-Dirac hot path on the SU(3) two-index symmetric
(sextet, D_R = 6) 32^3 x 64 workload: m0 = -0.3, links exp(i 0.4 H) followed
by a random Haar gauge transform, antiperiodic in time.

One step is one pass of the whole hot path over one batch of synthetic
input, as an HMC force evaluation of the fermion monomial does it:
  1. represent the fundamental gauge field (FP64, FP32 and float-float
     stored links, FP64 and FP32 fundamental links for the in-kernel rebuild),
  2. D_eo applications in FP32 and FP64 (the metric's kernel, event-timed),
  3. mixed-precision CG (FP32 inner, defect correction) on
     Dhat^dag Dhat x = phi to a true relative residual of 1e-10: the
     intermediate true residuals in float-float, the one that meets the
     tolerance in FP64 (--residual f64: every true residual in FP64),
  4. the fermion force of S = phi^dag (Dhat^dag Dhat)^-1 phi (fused with the
     solve: the force reuses the operator applications of its final residual).

value: algorithmic ("compulsory") bytes of every hopping-kernel launch of the
step, V/2 (8 L_p + 2 S_p) each with stored-link L_p whatever link mode the
launch used, divided by the step's device time -- the whole step's
D_eo-equivalent bandwidth.  roofline: the FP32 D_eo kernel,
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
WORKLOAD_TEXT = "SU(3) sextet (SYM, D_R=6) 32^3x64, m0=-0.3, even/odd, mixed FP32/FP64 CG to 1e-10 + force"
# DRAM bytes (read + write) of one FP32 D_eo launch of the direct hopping
# kernel on this workload (32^3 x 64 sextet, stored links), measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum = 2.624 + 0.167 GB) against
# 2.819 GB of compulsory bytes.  Reported only while the tuner picks that
# kernel.
DEO_TRAFFIC_DIRECT = 2.790e9
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


def hop_bytes(D: int, real_links: bool, prec: int, vh: int, spinor_reads: int = 1) -> int:
    """compulsory bytes of one hopping launch: V/2 (8 L_p + 2 S_p); with
    spinor_reads = 8 the conventional "effective" count V/2 (8 L_p + 9 S_p)
    that charges every neighbour gather."""
    cb = [16, 8, 4, 4][prec]
    lp = D * D * (cb // 2 if real_links else cb)
    sp = 4 * D * cb + (4 if prec >= 2 else 0)
    return vh * (8 * lp + (1 + spinor_reads) * sp)


# representations whose links are stored as reals
REAL_REPS = ("ADJ", "ASYM_REAL")


def link_bytes(N: int, D: int, rep: str, prec: int, rebuild: bool) -> int:
    """bytes of one link as a launch reads it: D_R^2 complex (D_R^2 real for
    the adjoint), or N^2 complex when rebuilt in the kernel from U_F"""
    cb = [16, 8, 4, 4, 16][prec]
    if rebuild:
        return N * N * cb
    return D * D * (cb // 2 if rep in REAL_REPS else cb)


def spinor_bytes(D: int, prec: int) -> int:
    cb = [16, 8, 4, 4, 16][prec]
    return 4 * D * cb + (4 if prec in (2, 3) else 0)


def job_throughput(step_bytes_local: float, ms_local: float, steps: int, dist=None, device=None):
    """Whole-job throughput of N replicas: every rank processed step_bytes_local
    per step; the job time is the slowest rank's.  Returns (GB/s, ms per step)."""
    import torch
    ms = float(ms_local)
    world = 1
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([ms, step_bytes_local], dtype=torch.float64, device=device)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        ms = float(tmax[0].item())
        total_bytes = float(tsum[1].item())
    else:
        total_bytes = step_bytes_local
    ms_per_step = ms / steps
    return total_bytes / (ms_per_step * 1e-3) / 1e9, ms_per_step


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
    real = wl.rep in REAL_REPS
    # replicas: every rank draws its own field
    import dataclasses
    wl_r = dataclasses.replace(wl, seed=wl.seed + 1000 * rank)
    U = wl_r.links(device=dev)
    phi = synth.gaussian_spinor(vh, D, wl_r.seed + 7, device=dev)
    res_prec = hr.PRECS[args.residual]
    # stored and fundamental links: the solver's precisions each use the way of
    # obtaining U_R the tuner measures faster (LINKS_AUTO); the D_eo launches of
    # the metric read the stored links
    g = hr.Gauge(lat, U, precs=("f64", "f32") + (("df64",) if res_prec == hr.DF64 else ()), stored=True,
                 rebuild=True)
    stream = torch.cuda.current_stream()
    # pick link modes and hopping-kernel variants (setup, outside the timed
    # region; the solver would otherwise do it at its first call)
    g.set_link_mode(hr.LINKS_STORED)
    g.tune(hr.F32)
    variants = {name: g.hop_variant(hr.F32, epi) for name, epi in
                (("store", hr.EPI_STORE), ("store_norm", hr.EPI_STORE_NORM), ("cg_update", hr.EPI_CG_UPDATE))}
    g.set_link_mode(hr.LINKS_AUTO)
    g.tune(hr.F32)
    g.tune(hr.F64)
    solver_links = {"f32": ["stored", "rebuild"][g.link_mode(hr.F32)],
                    "f64": ["stored", "rebuild"][g.link_mode(hr.F64)]}
    solver_variants = {name: g.hop_variant(hr.F32, epi) for name, epi in
                       (("store", hr.EPI_STORE), ("store_norm", hr.EPI_STORE_NORM),
                        ("cg_update", hr.EPI_CG_UPDATE))}
    x32 = phi.to(torch.complex64)
    y32 = torch.empty_like(x32)
    y64 = torch.empty_like(phi)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.deo_per_step)]
    n_deo = args.deo_per_step
    deo_ms = []
    work = {"bytes": 0, "actual": 0}

    pev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    phases = {"represent": 0.0, "deo": 0.0, "cg_force": 0.0}
    Fbuf = torch.zeros((lat.volume, 4, wl.N ** 2 - 1), dtype=torch.float64, device=dev)
    xbuf = torch.zeros_like(phi)

    def step(phi_dev, U_dev, xb=xbuf, Fb=Fbuf, phase_times=True):
        pev[0].record(stream)
        g.update(U_dev)
        pev[1].record(stream)
        g.set_link_mode(hr.LINKS_STORED)
        for k in range(n_deo):
            ev[2 * k].record(stream)
            g.apply(hr.EVEN, hr.F32, x32, out=y32)
            ev[2 * k + 1].record(stream)
        g.apply(hr.EVEN, hr.F64, phi_dev, out=y64)
        g.set_link_mode(hr.LINKS_AUTO)
        pev[2].record(stream)
        # x = (Dhat^dag Dhat)^-1 phi and the force of S = phi^dag x in one call;
        # the force's Dhat x, D_oe x and (D^dag)_oe Dhat x come from the
        # solve's final FP64 true residual
        Fb.zero_()
        x, F, _, res, st = g.cg_solve_force(hr.EO_PRECOND, phi_dev, x=xb, tol=TOL, max_iter=20000,
                                            inner=hr.F32, inner_tol=1e-5, residual=res_prec, coeff=-1.0,
                                            F=Fb)
        pev[3].record(stream)
        if phase_times:
            torch.cuda.synchronize()
            for name, a, b in (("represent", 0, 1), ("deo", 1, 2), ("cg_force", 2, 3)):
                phases[name] += pev[a].elapsed_time(pev[b])
        r = res[0]
        # hop launches of this step by precision
        h32 = n_deo + 4 * r["iters"]
        # FP64-class (FP64 or DF64, 16 bytes per complex either way) launches: the
        # D_eo and 4 per true residual after each inner solve (the first one, of
        # x = 0, is b itself), plus 4 for the FP64 confirmation of a DF64 one
        h64 = 1 + 4 * (r["outer_iters"] + (res_prec == hr.DF64))
        work["bytes"] += h32 * hop_bytes(D, real, hr.F32, vh) + h64 * hop_bytes(D, real, hr.F64, vh)
        # the same launches at the bytes they move: the D_eo launches read
        # stored links, the solver's launches use its tuned link mode
        sp32, sp64 = spinor_bytes(D, hr.F32), spinor_bytes(D, hr.F64)
        lp32 = link_bytes(wl.N, D, wl.rep, hr.F32, solver_links["f32"] == "rebuild")
        lp64 = link_bytes(wl.N, D, wl.rep, hr.F64, solver_links["f64"] == "rebuild")
        work["actual"] += (n_deo * vh * (8 * link_bytes(wl.N, D, wl.rep, hr.F32, False) + 2 * sp32)
                           + vh * (8 * link_bytes(wl.N, D, wl.rep, hr.F64, False) + 2 * sp64)
                           + 4 * r["iters"] * vh * (8 * lp32 + 2 * sp32)
                           + (h64 - 1) * vh * (8 * lp64 + 2 * sp64))
        work["res"] = r
        return x, F

    for _ in range(args.warmup):
        step(phi, U)
    torch.cuda.synchronize()
    work["bytes"] = 0
    work["actual"] = 0
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
    actual_bytes = work["actual"] / args.steps
    res = work["res"]
    value, ms_per_step = job_throughput(step_bytes, ms, args.steps, dist, dev)
    actual_value, _ = job_throughput(actual_bytes, ms, args.steps, dist, dev)
    phase_ms = {k: round(v / args.steps, 2) for k, v in phases.items()}
    deo_ms_avg = sum(deo_times) / len(deo_times)
    deo_bytes = hop_bytes(D, real, hr.F32, vh)
    peak, peak_kind = _peaks()
    achieved = deo_bytes / (deo_ms_avg * 1e-3) / 1e9
    traffic = args.traffic
    if traffic is None and args.workload == WORKLOAD and variants["store"] == hr.HOP_DIRECT:
        traffic = DEO_TRAFFIC_DIRECT

    # end to end through the C ABI with host buffers: inputs copied in and the
    # solution and force copied out inside the timed region
    # end to end with host buffers: every step copies its inputs (gauge field,
    # pseudofermion) from pinned host memory and its results (solution, force)
    # back.  The copies run on their own stream, double-buffered: step k+1's
    # inputs arrive while step k computes, and step k's results leave while
    # step k+1 computes; all of them lie inside the timed region.
    e2e = None
    if not args.no_e2e:
        U_h = U.cpu().pin_memory()
        phi_h = phi.cpu().pin_memory()
        X_h = [torch.empty(phi.shape, dtype=phi.dtype).pin_memory() for _ in range(2)]
        F_h = [torch.empty((lat.volume, 4, wl.N ** 2 - 1), dtype=torch.float64).pin_memory() for _ in range(2)]
        U_d = [torch.empty_like(U) for _ in range(2)]
        phi_d = [torch.empty_like(phi) for _ in range(2)]
        x_d = [xbuf, torch.empty_like(phi)]
        F_d = [Fbuf, torch.empty_like(Fbuf)]
        cs = torch.cuda.Stream(device=dev)
        ready = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        sent = [torch.cuda.Event() for _ in range(2)]
        work["bytes"] = 0
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0.record(stream)
        cs.wait_stream(stream)
        with torch.cuda.stream(cs):
            U_d[0].copy_(U_h, non_blocking=True)
            phi_d[0].copy_(phi_h, non_blocking=True)
            ready[0].record(cs)
        for k in range(args.steps):
            b, nb = k % 2, (k + 1) % 2
            if k + 1 < args.steps:
                with torch.cuda.stream(cs):
                    if k >= 1:
                        cs.wait_event(done[nb])      # step k-1 is finished with these buffers
                    U_d[nb].copy_(U_h, non_blocking=True)
                    phi_d[nb].copy_(phi_h, non_blocking=True)
                    ready[nb].record(cs)
            stream.wait_event(ready[b])
            if k >= 2:
                stream.wait_event(sent[b])           # step k-2's results have left
            x, F = step(phi_d[b], U_d[b], x_d[b], F_d[b], phase_times=False)
            done[b].record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(done[b])
                X_h[b].copy_(x, non_blocking=True)
                F_h[b].copy_(F, non_blocking=True)
                sent[b].record(cs)
        stream.wait_stream(cs)
        t1.record(stream)
        torch.cuda.synchronize()
        ems = t0.elapsed_time(t1)
        X_h, F_h = X_h[0], F_h[0]
        evalue, ems_step = job_throughput(work["bytes"] / args.steps, ems, args.steps, dist, dev)
        e2e = {"value": round(evalue, 1), "unit": UNIT, "ms_per_step": round(ems_step, 3),
               "h2d_bytes_per_step": U_h.numel() * 16 + phi_h.numel() * 16,
               "d2h_bytes_per_step": X_h.numel() * 16 + F_h.numel() * 8}

    # time to 1e-10: plain FP64 CG vs defect correction with low-precision inner solves
    cg = None
    multishift = None
    clover = None
    if rank == 0 and not args.no_cg_compare:
        g2 = hr.Gauge(lat, U, precs=("f64", "f32", "f16", "bf16", "df64"), stored=True, rebuild=True)
        g2.set_link_mode(hr.LINKS_AUTO)
        cg = {}
        cg_variants = (("fp64", hr.F64, hr.F64), ("mixed_fp32", hr.F32, hr.F64), ("mixed_fp16", hr.F16, hr.F64),
                    ("mixed_bf16", hr.BF16, hr.F64), ("mixed_fp32_df64res", hr.F32, hr.DF64),
                    ("mixed_fp16_df64res", hr.F16, hr.DF64))
        for name, inner, resid in cg_variants:
            g2.cg_solve(hr.EO_PRECOND, phi, tol=1e-3, inner=inner, max_iter=200, check=False)
            torch.cuda.synchronize()
            t0.record(stream)
            # inner tolerances: the fastest of a sweep on this workload
            # (FP32 1e-5: 2 outer steps; F16 3e-4: 3; BF16 1e-3: 4)
            itol = {hr.F32: 1e-5, hr.F16: 3e-4, hr.BF16: 1e-3}[inner] if inner != hr.F64 else 1e-5
            x, r, st = g2.cg_solve(hr.EO_PRECOND, phi, tol=TOL, max_iter=20000, inner=inner,
                                   inner_tol=itol, residual=resid, check=False)
            t1.record(stream)
            torch.cuda.synchronize()
            cg[name] = {"ms": round(t0.elapsed_time(t1), 2), "iters": r[0]["iters"],
                        "outer": r[0]["outer_iters"], "true_rel_residual": r[0]["true_rel_residual"],
                        "status": r[0]["status"]}
        for name, _, _ in cg_variants[1:]:
            cg[name]["speedup_vs_fp64"] = round(cg["fp64"]["ms"] / cg[name]["ms"], 2)
        if not args.no_multishift:
            multishift = multishift_compare(hr, g2, phi, stream, wl.m0)
        if not args.no_clover:
            clover = clover_measure(hr, g2, U, phi, stream)
        g2.close()

    hmc = None
    if rank == 0 and not args.no_hmc:
        hmc = hmc_measure(hr, lat, U, dev, stream)

    batched = None
    if rank == 0 and not args.no_batched:
        g.close()
        torch.cuda.empty_cache()
        # SU(4) 24^3 x 48 + uneven instances: the 2AS in the real basis (real
        # links) and the fundamental with every comparison, the 2AS in the
        # complex basis with the batched mixed solve only
        batched = {"ASYM_REAL": batched_compare(hr, synth, dev, stream, rep="ASYM_REAL"),
                   "FUND": batched_compare(hr, synth, dev, stream, rep="FUND"),
                   "ASYM": batched_compare(hr, synth, dev, stream, rep="ASYM", mixed_only=True)}

    by_rep = None
    if rank == 0 and not args.no_deo_by_rep:
        torch.cuda.empty_cache()
        by_rep = deo_by_rep(hr, synth, dev, stream)

    largen = None
    if rank == 0 and not args.no_largen:
        torch.cuda.empty_cache()
        largen = largen_sweep(hr, synth, dev, stream)

    out = None
    if rank == 0:
        cpu = None if (world > 1 or args.no_cpu_baseline) else cpu_baseline(wl, budget_s=args.cpu_seconds)
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" + ("+df64" if res_prec == hr.DF64 else ""),
            "data": "synthetic (seeded Philox4x32-10 links exp(i 0.4 H) + Haar gauge transform, "
                    "Gaussian pseudofermion)",
            "config": {"workload": WORKLOAD_TEXT,
                       "true_residual_arith": ("float-float intermediate, FP64 final (the reported residual)"
                                               if res_prec == hr.DF64 else "FP64"),
                       "force_arith": "float-float" if res_prec == hr.DF64 else "FP64",
                       "lattice": list(wl.dims), "N": wl.N, "rep": wl.rep, "m0": wl.m0,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (FP32 links 4.8 GB per parity)",
                       "deo_per_step": n_deo, "cg_iters_per_step": res["iters"],
                       "cg_outer_per_step": res["outer_iters"],
                       "true_rel_residual": res["true_rel_residual"]},
            "roofline": {"bound": "hbm", "kernel": f"hopping kernel <3,SYM,F32> variant {variants['store']} (D_eo, stored links)",
                         "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic, "deo_ms": round(deo_ms_avg, 4),
                         "bytes_per_launch": deo_bytes,
                         "effective_GBs": round(hop_bytes(D, real, hr.F32, vh, 8) / (deo_ms_avg * 1e-3) / 1e9, 1),
                         "frac_of_nominal_7900": round(achieved / 7900.0, 4)},
            "step_actual_bytes": {"GBs": round(actual_value, 1), "bytes_per_step": int(actual_bytes),
                                  "note": "the step's hopping launches at the bytes they move (solver "
                                          "launches in their tuned link mode); value charges every "
                                          "launch at stored-link bytes (D_eo-equivalent work)"},
            "hop_variants_f32": variants,
            "solver_links": solver_links,
            "solver_hop_variants_f32": solver_variants,
            "gpu_launches": int(launches),
            "phases_ms": phase_ms,
            "clocks": ck,
            "e2e": e2e,
            "cg": cg,
            "batched": batched,
            "multishift": multishift,
            "hmc": hmc,
            "clover": clover,
            "deo_by_rep": by_rep,
            "large_n_fund_f32_deo": largen,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    g.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def multishift_compare(hr, g, phi, stream, m0):
    """The RHMC's multi-shift inversion (Sec. 4.3.2) on the bench lattice:
    (A + b_k) x_k = phi for the 10 poles b_k of the best relative
    approximation of x^(-1/2) on [0.1, ((4+m)^2 + 16)^2] (hr_rational_approx,
    relative error 1e-7; the upper end
    bounds the spectrum of A = Dhat^dag Dhat), each to a true residual of
    1e-10: multi-shift CG in FP64 and with FP32 iterations + FP64 correction,
    against plain FP64 shifted CG solving one pole after another (the
    definition of the multi-shift inversion); and r(A) phi = a0 phi +
    sum_k a_k x_k, the whole rational application."""
    import torch

    from paper_2503_06721_gb300 import rational
    m4 = 4.0 + m0
    ra = rational.approx(0.5, 10, 0.1, (m4 * m4 + 16.0) ** 2)
    MS_SHIFTS = list(ra.poles)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"approx": f"best x^-1/2 (Remez), degree 10, [0.1, {ra.hi:.1f}], rel. error {ra.max_rel_err:.2e}",
           "shifts": [float(f"{s:.6g}") for s in MS_SHIFTS]}
    for name, inner in (("multishift_fp64", hr.F64), ("multishift_mixed_fp32", hr.F32)):
        g.cg_solve_multishift(hr.EO_PRECOND, phi, MS_SHIFTS, tol=1e-3, inner=inner, check=False)
        torch.cuda.synchronize()
        e0.record(stream)
        x, res, st = g.cg_solve_multishift(hr.EO_PRECOND, phi, MS_SHIFTS, tol=TOL, inner=inner,
                                           inner_tol=1e-5, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms": round(e0.elapsed_time(e1), 2), "status": hr.STATUS.get(st, st),
                     "iters": [r[0]["iters"] for r in res],
                     "outer": [r[0]["outer_iters"] for r in res],
                     "max_true_rel_residual": max(r[0]["true_rel_residual"] for r in res)}
        del x
    torch.cuda.synchronize()
    e0.record(stream)
    worst, its = 0.0, []
    for s in MS_SHIFTS:
        x, res, st = g.cg_solve_multishift(hr.EO_PRECOND, phi, [s], tol=TOL, inner=hr.F64, check=False)
        worst = max(worst, res[0][0]["true_rel_residual"])
        its.append(res[0][0]["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    out["sequential_fp64"] = {"ms": round(e0.elapsed_time(e1), 2), "iters": its,
                              "max_true_rel_residual": worst}
    for name in ("multishift_fp64", "multishift_mixed_fp32"):
        out[f"speedup_{name}_vs_sequential_fp64"] = round(out["sequential_fp64"]["ms"] / out[name]["ms"], 2)
    torch.cuda.synchronize()
    e0.record(stream)
    y, x, res = hr.rational_apply(g, hr.EO_PRECOND, phi, ra, tol=TOL, inner=hr.F32)
    e1.record(stream)
    torch.cuda.synchronize()
    out["rational_apply_mixed_fp32_ms"] = round(e0.elapsed_time(e1), 2)
    del x, y
    return out


def largen_sweep(hr, synth, dev, stream, dims=(48, 24, 24, 24)):
    """D_eo bandwidth of the fundamental representation as N grows (Sec. 8.2,
    the large-N study): SU(3) and SU(4) with the site-parallel kernel (the
    tuned variant), SU(5), SU(6) and SU(8) with the colour-parallel kernel; FP32
    stored links, m0 = -0.1, links exp(i 0.4 H), a 24^3 x 48 lattice (every
    launch moves 0.26-1.5 GB, above L2).  GB/s of compulsory bytes."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"lattice": list(dims)}
    for N in (3, 4, 5, 6, 8):
        lat = hr.Lattice(N, "FUND", dims, (-1, 1, 1, 1), -0.1)
        U = synth.random_links(lat.volume, N, 0.4, 2503067210 + 40 + N, device=dev)
        g = hr.Gauge(lat, U, precs=("f64", "f32"))
        del U
        vh = lat.volume // 2
        x = synth.gaussian_spinor(vh, N, 3, device=dev).to(torch.complex64)
        y = torch.empty_like(x)
        if N <= 4:
            g.tune(hr.F32)
        for _ in range(3):
            g.apply(hr.EVEN, hr.F32, x, out=y)
        torch.cuda.synchronize()
        reps = 20
        e0.record(stream)
        for _ in range(reps):
            g.apply(hr.EVEN, hr.F32, x, out=y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        byts = hop_bytes(N, False, hr.F32, vh)
        out[f"su{N}"] = {"kernel": ("colour-parallel" if N >= 5 else
                                    f"site-parallel variant {g.hop_variant(hr.F32, hr.EPI_STORE, 1)}"),
                         "ms": round(ms, 4), "GBs": round(byts / (ms * 1e-3) / 1e9, 1),
                         "frac_of_hbm": round(byts / (ms * 1e-3) / 1e9 / _peaks()[0], 4)}
        g.close()
        del x, y
        torch.cuda.empty_cache()
    return out


DEO_CASES = [
    # (name, N, rep, dims, m0, eps, precisions, link modes)
    ("su2_adj_8x8x8x8", 2, "ADJ", (8, 8, 8, 8), -0.2, 0.3, ("f32", "f16", "bf16"), ("stored",)),
    ("su3_sym_64x32x32x32", 3, "SYM", (64, 32, 32, 32), -0.3, 0.4, ("f32", "f16", "bf16"),
     ("stored", "rebuild")),
    ("su3_adj_32x32x32x32", 3, "ADJ", (32, 32, 32, 32), -0.35, 0.5, ("f32", "f16", "bf16"), ("stored", "rebuild")),
    ("su3_adj_128x64x64x64", 3, "ADJ", (128, 64, 64, 64), -0.35, 0.5, ("f32", "f16", "bf16"),
     ("stored", "rebuild")),
    ("su4_fund_48x24x24x24", 4, "FUND", (48, 24, 24, 24), -0.25, 0.4, ("f32", "f16", "bf16"), ("stored",)),
    ("su4_asym_48x24x24x24", 4, "ASYM", (48, 24, 24, 24), -0.25, 0.4, ("f32", "f16", "bf16"),
     ("stored", "rebuild")),
    ("su4_asym_real_48x24x24x24", 4, "ASYM_REAL", (48, 24, 24, 24), -0.25, 0.4, ("f32", "f16", "bf16"),
     ("stored", "rebuild")),
    # the colour-parallel kernel (Sec. 8.2's D_R-site-parallel form): D_R = 15 and 10
    ("su4_adj_48x24x24x24", 4, "ADJ", (48, 24, 24, 24), -0.25, 0.4, ("f32",), ("stored",)),
    ("su4_sym_48x24x24x24", 4, "SYM", (48, 24, 24, 24), -0.25, 0.4, ("f32",), ("stored",)),
]


def fp64_peak(dev, stream, n=4096, reps=6):
    """FP64 arithmetic peak of this GPU as a cuBLAS DGEMM measures it
    (2 n^3 flop per product, best of reps, CUDA events)."""
    import torch
    a = torch.randn((n, n), dtype=torch.float64, device=dev)
    b = torch.randn((n, n), dtype=torch.float64, device=dev)
    c = a @ b
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(reps):
        e0.record(stream)
        torch.matmul(a, b, out=c)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def deo_by_rep(hr, synth, dev, stream, reps=20):
    """D_eo (even output, one right-hand side) for every representation and
    storage precision, stored links and, where listed, links rebuilt in the
    kernel from the fundamental ones; each with the tuned kernel variant.
    GB/s of compulsory bytes V/2 (8 L_p + 2 S_p) at the bytes the launch
    reads (L_p of the link mode), and the fraction of the measured HBM copy
    bandwidth.  Plus the FP64 sextet D_eo, whose 0.92 flop per byte makes it
    bound by the FP64 units: GFLOP/s (128 D^2 + 56 D flop per site) against
    the FP64 peak a DGEMM measures on this GPU."""
    import torch
    peak, _ = _peaks()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"unit": "GB/s of compulsory bytes", "peak_GBs": peak, "reps": reps}
    for name, N, rep, dims, m0, eps, precs, modes in DEO_CASES:
        lat = hr.Lattice(N, rep, dims, (-1, 1, 1, 1), m0)
        vh, D = lat.volume // 2, lat.D
        U = synth.random_links(lat.volume, N, eps, 2503067210 + 60, device=dev)
        x64 = synth.gaussian_spinor(vh, D, 3, device=dev)
        row = {"dims": list(dims), "D_R": D}
        for p in precs:
            # one handle per precision: the 64^3 x 128 adjoint's FP32 links alone take 69 GB
            prec = hr.PRECS[p]
            g = hr.Gauge(lat, U, precs=(p,), stored="stored" in modes, rebuild="rebuild" in modes)
            x = x64.to(torch.complex64) if prec == hr.F32 else hr.field_convert(lat, hr.EVEN, x64, hr.F64, prec)
            y = g.apply(hr.EVEN, prec, x)
            for mode in modes:
                g.set_link_mode(hr.LINKS_STORED if mode == "stored" else hr.LINKS_REBUILD)
                g.tune(prec)
                ms = timed(lambda: g.apply(hr.EVEN, prec, x, out=y))
                byts = vh * (8 * link_bytes(N, D, rep, prec, mode == "rebuild") + 2 * spinor_bytes(D, prec))
                gbs = byts / (ms * 1e-3) / 1e9
                row[f"{p}_{mode}"] = {"ms": round(ms, 4), "GBs": round(gbs, 1), "frac": round(gbs / peak, 4),
                                      "variant": g.hop_variant(prec, hr.EPI_STORE, 1)}
            g.close()
            del x, y
            torch.cuda.empty_cache()
        del U, x64
        torch.cuda.empty_cache()
        out[name] = row
    # FP64 sextet D_eo against the FP64 units
    fpk = fp64_peak(dev, stream)
    lat = hr.Lattice(3, "SYM", (64, 32, 32, 32), (-1, 1, 1, 1), -0.3)
    vh, D = lat.volume // 2, lat.D
    g = hr.Gauge(lat, synth.random_links(lat.volume, 3, 0.4, 2503067210 + 61, device=dev), precs=("f64",))
    x = synth.gaussian_spinor(vh, D, 3, device=dev)
    y = g.apply(hr.EVEN, hr.F64, x)
    ms = timed(lambda: g.apply(hr.EVEN, hr.F64, x, out=y))
    flops = vh * (128 * D * D + 56 * D)
    byts = vh * (8 * link_bytes(3, D, "SYM", hr.F64, False) + 2 * spinor_bytes(D, hr.F64))
    out["su3_sym_64x32x32x32_f64"] = {
        "ms": round(ms, 4), "GFLOPs": round(flops / (ms * 1e-3) / 1e9, 1),
        "fp64_peak_dgemm_TFLOPs": round(fpk, 3), "flop_frac": round(flops / (ms * 1e-3) / 1e12 / fpk, 4),
        "GBs": round(byts / (ms * 1e-3) / 1e9, 1), "frac_of_hbm": round(byts / (ms * 1e-3) / 1e9 / peak, 4),
        "bound": "fp64 alu"}
    g.close()
    del x, y
    torch.cuda.empty_cache()
    return out


def clover_measure(hr, g, U, phi, stream, csw=1.0):
    """The clover-improved operator (Sec. 5.1.2) on the bench lattice: the
    build of C and C^-1 (FP64, both parities, FP64 and FP32 records), one Dhat
    = C_ee - D_eo C_oo^-1 D_oe application in FP32 and FP64 against the plain
    Dhat, and a solve of Dhat^dag Dhat x = phi to 1e-10 with FP32 inner
    iterations and FP64 correction."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"csw": csw}
    x32 = phi.to(torch.complex64)
    for name, prec, xin in (("dhat_f32_ms", hr.F32, x32), ("dhat_f64_ms", hr.F64, phi)):
        out["plain_" + name] = round(timed(lambda: g.apply(hr.EO_PRECOND, prec, xin), 10), 3)
    torch.cuda.synchronize()
    e0.record(stream)
    g.set_clover(U, csw, hr.CLOVER_PLAIN)
    e1.record(stream)
    torch.cuda.synchronize()
    out["build_ms"] = round(e0.elapsed_time(e1), 2)
    for name, prec, xin in (("dhat_f32_ms", hr.F32, x32), ("dhat_f64_ms", hr.F64, phi)):
        out["clover_" + name] = round(timed(lambda: g.apply(hr.EO_PRECOND, prec, xin), 10), 3)
    g.cg_solve(hr.EO_PRECOND, phi, tol=1e-3, inner=hr.F32, check=False)
    torch.cuda.synchronize()
    e0.record(stream)
    x, res, st = g.cg_solve(hr.EO_PRECOND, phi, tol=TOL, inner=hr.F32, inner_tol=1e-5, check=False)
    e1.record(stream)
    torch.cuda.synchronize()
    out["cg_mixed_fp32"] = {"ms": round(e0.elapsed_time(e1), 2), "iters": res[0]["iters"],
                            "outer": res[0]["outer_iters"], "true_rel_residual": res[0]["true_rel_residual"],
                            "status": hr.STATUS.get(st, st)}
    g.set_clover(None, 0.0, hr.CLOVER_NONE)
    return out


def hmc_measure(hr, lat, U, dev, stream, beta=5.5, tau=0.5, nsteps=4):
    """One molecular-dynamics trajectory of the two-flavour HMC (Sec. 2.5,
    Sec. 4.2) on the bench lattice: Wilson gauge action at beta, even/odd
    pseudofermion from the heat bath phi = Dhat^dag eta, 2nd-order Omelyan
    integrator, each force solve mixed FP32/FP64 to 1e-10 in the automatic link
    mode.  Momenta and eta are seeded Gaussians."""
    import torch
    U3 = U.clone()
    g3 = hr.Gauge(lat, U3, precs=("f64", "f32"), stored=True, rebuild=True)
    g3.set_link_mode(hr.LINKS_AUTO)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2503067210 + 31)
    ng = lat.N * lat.N - 1
    pi = torch.randn((lat.volume, 4, ng), dtype=torch.float64, device=dev, generator=gen) / (hr.T_FUND ** 0.5)
    eta = torch.randn((lat.volume // 2, 4, lat.D), dtype=torch.complex128, device=dev, generator=gen)
    phi = g3.apply(hr.EO_PRECOND, hr.F64, eta, dagger=True)
    H0 = hr.hamiltonian(g3, U3, pi, phi, beta, tol=1e-11, inner=hr.F32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    st = hr.md_trajectory(g3, U3, pi, phi, beta, tau, nsteps, integrator=hr.MD_OMELYAN2, tol=1e-10,
                          inner=hr.F32, inner_tol=1e-5)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    H1 = hr.hamiltonian(g3, U3, pi, phi, beta, tol=1e-11, inner=hr.F32)
    g3.close()
    return {"workload": f"two-flavour HMC trajectory, beta {beta}, tau {tau}, {nsteps} Omelyan steps, "
                        "FP32-inner / FP64 force solves to 1e-10",
            "trajectory_ms": round(ms, 1), "ms_per_force_eval": round(ms / max(1, st["force_evals"]), 1),
            "force_evals": st["force_evals"], "cg_iters": st["cg_iters"],
            "max_true_rel_residual": st["max_true_rel_residual"],
            "H0": [round(h, 4) for h in H0], "dH": round(sum(H1) - sum(H0), 6)}


def batched_compare(hr, synth, dev, stream, rep="ASYM", mixed_only=False):
    """SU(4) 24^3 x 48 with 12 point sources (4 spins x 3 colour subsets) plus
    8^4, 12^4, 16^3 x 32 instances (4 Gaussian rhs each, m0 = -0.1, -0.25, -0.4):
    one batched FP32-inner / FP64-refined solve to 1e-10 against plain FP64 CG
    solving every right-hand side one after the other."""
    import torch
    wl = synth.WORKLOADS[f"su4_{rep.lower()}_48x24x24x24"]
    specs = [(wl.dims, wl.m0, 12)] + [(d, m, 4) for d, m in synth.UNEVEN_INSTANCES]
    gauges, bs, nr = [], [], []
    for i, (dims, m0, n) in enumerate(specs):
        lat = hr.Lattice(wl.N, rep, dims, wl.bc, m0)
        V = lat.volume
        gauges.append(hr.Gauge(lat, synth.random_links(V, wl.N, wl.eps, wl.seed + i, device=dev),
                               precs=("f64", "f32", "df64")))
        if n == 12:
            b = torch.zeros((12, V // 2, 4, lat.D), dtype=torch.complex128, device=dev)
            for s in range(4):
                for k in range(3):
                    for c in range(lat.D):
                        if c % 3 == k:
                            b[3 * s + k, 0, s, c] = 1.0
        else:
            b = synth.gaussian_spinor(V // 2, lat.D, 700 + i, device=dev, nrhs=n)
        bs.append(b.contiguous())
        nr.append(n)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"SU(4) {rep} 24^3x48 (12 point sources) + 8^4, 12^4, 16^3x32 (4 rhs each)",
           "rhs_total": sum(nr)}
    runs = (("batched_mixed_fp32", hr.F32, hr.F64), ("batched_mixed_fp32_df64res", hr.F32, hr.DF64),
            ("batched_fp64", hr.F64, hr.F64))
    for name, inner, resid in runs[:1] if mixed_only else runs:
        xs = [torch.zeros_like(b) for b in bs]
        hr.cg_solve_batched(gauges, hr.EO_PRECOND, bs, xs, nr, tol=1e-3, inner=inner, residual=resid,
                            check=False)
        xs = [torch.zeros_like(b) for b in bs]
        torch.cuda.synchronize()
        e0.record(stream)
        res, st = hr.cg_solve_batched(gauges, hr.EO_PRECOND, bs, xs, nr, tol=TOL, inner=inner, residual=resid,
                                      check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms": round(e0.elapsed_time(e1), 2), "status": hr.STATUS.get(st, st),
                     "max_true_rel_residual": max(r["true_rel_residual"] for r in res),
                     "max_iters": max(r["iters"] for r in res)}
    # the same mixed solves instance by instance (each instance's right-hand
    # sides together): the gain of batching over per-instance mixed solves
    for g, b, n in zip(gauges, bs, nr):
        g.cg_solve(hr.EO_PRECOND, b, nrhs=n, tol=1e-3, inner=hr.F32, check=False)
    torch.cuda.synchronize()
    e0.record(stream)
    worst = 0.0
    for g, b, n in zip(gauges, bs, nr):
        x, r, st = g.cg_solve(hr.EO_PRECOND, b, nrhs=n, tol=TOL, inner=hr.F32, inner_tol=1e-5, check=False)
        worst = max([worst] + [q["true_rel_residual"] for q in r])
    e1.record(stream)
    torch.cuda.synchronize()
    out["per_instance_mixed_fp32"] = {"ms": round(e0.elapsed_time(e1), 2), "max_true_rel_residual": worst}
    out["speedup_batched_vs_per_instance_mixed"] = round(
        out["per_instance_mixed_fp32"]["ms"] / out["batched_mixed_fp32"]["ms"], 2)
    if mixed_only:
        for g in gauges:
            g.close()
        return out
    # plain FP64 CG, one right-hand side at a time
    torch.cuda.synchronize()
    e0.record(stream)
    worst, its = 0.0, 0
    for g, b, n in zip(gauges, bs, nr):
        for k in range(n):
            x, r, st = g.cg_solve(hr.EO_PRECOND, b[k].contiguous(), tol=TOL, inner=hr.F64, check=False)
            worst = max(worst, r[0]["true_rel_residual"])
            its += r[0]["iters"]
    e1.record(stream)
    torch.cuda.synchronize()
    out["sequential_fp64"] = {"ms": round(e0.elapsed_time(e1), 2), "max_true_rel_residual": worst,
                              "total_iters": its}
    out["speedup_batched_mixed_vs_sequential_fp64"] = round(
        out["sequential_fp64"]["ms"] / out["batched_mixed_fp32"]["ms"], 2)
    out["speedup_batched_mixed_df64res_vs_sequential_fp64"] = round(
        out["sequential_fp64"]["ms"] / out["batched_mixed_fp32_df64res"]["ms"], 2)
    for g in gauges:
        g.close()
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
    byts = hop_bytes(D, wl.rep in REAL_REPS, 0, V // 2)
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
        byts["b"] += (4 * (it + 2) + 2 + 2) * hop_bytes(D, wl.rep in REAL_REPS, 0, V // 2)

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
           "config": {"workload": WORKLOAD_TEXT, "lattice": list(wl.dims), "N": wl.N, "rep": wl.rep,
                      "m0": wl.m0, "sample_lattice": list(dims)},
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
    prec = hr.PRECS[args.prec]
    g = hr.Gauge(lat, wl.links(device=dev), precs=(args.prec,), stored=not args.rebuild,
                 rebuild=args.rebuild)
    vh = lat.volume // 2
    n = args.nrhs
    if args.variant is None:
        g.tune(prec, nrhs=n)
    else:
        g.set_tuning(autotune=False, variant=args.variant)
    variant = g.hop_variant(prec, hr.EPI_STORE, n)
    x = synth.gaussian_spinor(vh, lat.D, 3, device=dev, nrhs=n)
    x = x if prec == hr.F64 else (x.to(torch.complex64) if prec == hr.F32 else
                                  hr.field_convert(lat, hr.EVEN, x, hr.F64, prec, n))
    y = g.apply(hr.EVEN, prec, x, nrhs=n)
    for _ in range(max(args.warmup, 1)):
        g.apply(hr.EVEN, prec, x, out=y, nrhs=n)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("hr_deo")   # profiler captures select this range
    e0.record()
    for _ in range(args.steps):
        g.apply(hr.EVEN, prec, x, out=y, nrhs=n)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    cb = [16, 8, 4, 4, 16][prec]
    sp = 4 * lat.D * cb + (4 if prec in (hr.F16, hr.BF16) else 0)
    lp = link_bytes(wl.N, lat.D, wl.rep, prec, args.rebuild)
    # compulsory bytes: every link once, every input and output spinor once
    byts = vh * (8 * lp + 2 * n * sp)
    print(json.dumps({"mode": "deo", "workload": args.workload, "prec": args.prec, "nrhs": n,
                      "links": "rebuild" if args.rebuild else "stored", "variant": variant,
                      "ms": round(ms, 4),
                      "GBs": round(byts / (ms * 1e-3) / 1e9, 1), "bytes_per_launch": byts}))


def run_force(args, local_rank):
    """Fermion force only (for profiler captures): Y = Dhat X, then W untimed
    and K timed calls of the even/odd force (FP64 or float-float kernel)."""
    import torch
    from paper_2503_06721_gb300 import build, hr, synth
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    build.build()
    wl = synth.WORKLOADS[args.workload]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    arith = hr.PRECS[args.force_arith]
    g = hr.Gauge(lat, wl.links(device=dev), precs=("f64",) + (("df64",) if arith == hr.DF64 else ()))
    X = synth.gaussian_spinor(lat.volume // 2, lat.D, 5, device=dev)
    Y = g.apply(hr.EO_PRECOND, hr.F64, X)
    F = torch.zeros((lat.volume, 4, wl.N ** 2 - 1), dtype=torch.float64, device=dev)
    for _ in range(max(args.warmup, 1)):
        g.force(hr.EO_PRECOND, X, Y, F=F, arith=arith)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("hr_force")
    e0.record()
    for _ in range(args.steps):
        g.force(hr.EO_PRECOND, X, Y, F=F, arith=arith)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "force", "workload": args.workload, "arith": args.force_arith,
                      "ms_per_call": round(e0.elapsed_time(e1) / args.steps, 4),
                      "note": "two force_kernel launches (one per parity) and two FP64 odd-half hops per call"}))


def run_clover(args, local_rank):
    """Clover build only (for profiler captures): W untimed and K timed
    builds of C and C^-1 (FP64 and FP32 records) with c_sw = 1."""
    import torch
    from paper_2503_06721_gb300 import build, hr, synth
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    build.build()
    wl = synth.WORKLOADS[args.workload]
    lat = hr.Lattice(wl.N, wl.rep, wl.dims, wl.bc, wl.m0)
    U = wl.links(device=dev)
    g = hr.Gauge(lat, U, precs=("f64", "f32"))
    for _ in range(max(args.warmup, 1)):
        g.set_clover(U, csw=1.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("hr_clover")
    e0.record()
    for _ in range(args.steps):
        g.set_clover(U, csw=1.0)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "clover", "workload": args.workload,
                      "ms_per_build": round(e0.elapsed_time(e1) / args.steps, 3)}))


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
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-FP64 solve comparison")
    ap.add_argument("--no-hmc", action="store_true", help="skip the HMC trajectory measurement")
    ap.add_argument("--no-clover", action="store_true", help="skip the clover-operator measurement")
    ap.add_argument("--no-largen", action="store_true", help="skip the large-N fundamental D_eo sweep")
    ap.add_argument("--no-deo-by-rep", action="store_true",
                    help="skip the D_eo sweep over representations and precisions")
    ap.add_argument("--no-multishift", action="store_true",
                    help="skip the multi-shift-vs-sequential shifted solve comparison")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--mode", choices=["step", "deo", "force", "clover"], default="step",
                    help="deo: only D_eo applications; force: only the fermion force; clover: only the "
                         "clover build (profiler captures)")
    ap.add_argument("--prec", choices=["f64", "f32", "f16", "bf16", "df64"], default="f32")
    ap.add_argument("--residual", choices=["df64", "f64"], default="df64",
                    help="arithmetic of the defect-correction true residuals (df64: float-float, "
                         "confirmed once in FP64 when it meets the tolerance)")
    ap.add_argument("--force-arith", choices=["f64", "df64"], default="f64",
                    help="force mode: arithmetic of the force kernel")
    ap.add_argument("--rebuild", action="store_true", help="deo mode: rebuild links in-kernel")
    ap.add_argument("--nrhs", type=int, default=1, help="deo mode: right-hand sides per application")
    ap.add_argument("--variant", type=int, default=None, choices=[0, 1, 2, 3, 4],
                    help="deo mode: force a hopping-kernel variant instead of autotuning")
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
    elif args.mode == "force":
        run_force(args, local_rank)
    elif args.mode == "clover":
        run_clover(args, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
