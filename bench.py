#!/usr/bin/env python
"""Benchmark of the GB300 contour-integral Helmholtz solver.

Metric: right-hand sides per second solved to a relative residual of 1e-8 (float64 true
residual), for the 64^3 Gaussian-bump workload (8 bumps, c in [1, 2], 8 points per wavelength
at c_min, 8-cell sponge, one Gaussian source, J = 8 contour nodes, FGMRES(30) with FCI and 4
inner GMRES steps).  One step = one full solve of that right-hand side.  `value` is the chosen
(mixed-precision) form; the plain all-float64 form is reported beside it.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank solves its own copy of the workload (replicas, weak
scaling, no data-path collective); value = all ranks' right-hand sides / max rank time.
--impl reference times the CPU oracle (complex128 numpy) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS/s to rel. residual 1e-8, plain vs chosen form; stencil HBM GB/s"
WORKLOAD = ("gaussian_bumps_64: 64^3 grid (h=1/65), c = 1 + 8 seeded Gaussian bumps (width 0.1, "
            "amplitudes U[0,0.4]) clipped to [1,2], 8 ppw at c_min, 8-cell sponge, Gaussian "
            "source sigma=2h, J=8 contour nodes, FGMRES(30) + FCI with 4 inner GMRES steps, "
            "rtol 1e-8 on the float64 true residual")
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-region", action="store_true",
                    help="bracket only the timed chosen-form steps with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off) and skip the other passes")
    ap.add_argument("--ncu-large", action="store_true",
                    help="run only the 256^3 stencil / polynomial-stage bandwidth measurement, "
                         "bracketed with cudaProfilerStart/Stop")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_counts():
    with open(os.path.join(ROOT, "oracle", "reference_counts.json")) as fh:
        return json.load(fh)


def time_oracle_sample(wl, outer_steps: int):
    """Seconds for `outer_steps` outer FGMRES steps of the oracle on this workload (plus the
    time per step), with the thread count numpy's BLAS uses."""
    from oracle import hz_oracle as O
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    _, nodes = O.setup_nodes(op, wl.J, wl.t, wl.eps)
    t0 = time.perf_counter()
    O.solve(op, op.s * wl.f[0], nodes, wl.restart, wl.k_in, 1e-30, 1, fixed_its=outer_steps)
    return time.perf_counter() - t0


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
        return int(n)
    except Exception:
        return 1


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import workloads as W
    wl = W.gaussian_bumps_64()
    its = oracle_counts()[wl.name]["its"]
    per = 1  # outer FGMRES steps per timed sample
    for _ in range(args.warmup):
        time_oracle_sample(wl, per)
    tt = [time_oracle_sample(wl, per) for _ in range(args.steps)]
    step_s = sum(tt) / len(tt)
    value = 1.0 / (step_s / per * its)
    sample = (f"{per} outer FGMRES step (FCI with {oracle_counts()[wl.name]['poly_matvecs_per_fci']}"
              f" polynomial-sweep matvecs + inner GMRES + CGS2) of the oracle per timed step, "
              f"scaled by the oracle's {its} steps to 1e-8")
    cores = cpu_threads()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": {"workload": WORKLOAD, "form": "oracle complex128"},
        "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def traffic_from_profile(kernel_src_hash: str):
    """DRAM bytes per launch of the polynomial-stage kernel from the committed ncu summary,
    or None if the summary is missing or was taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "poly_stage_gaussian_bumps_64.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256") != kernel_src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def kernel_hash():
    """sha256 over the polynomial-stage kernel's sources (its file and the device header)."""
    h = hashlib.sha256()
    for name in ("hz_kernels.cu", "hz_device.cuh"):
        with open(os.path.join(ROOT, "paper_1811_12378_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def large_grid_bandwidth(hz, torch, dev, N=256, profile_region=False):
    """Complex64 stencil and polynomial stage on an N^3 Gaussian-bump grid (fields >> L2):
    algorithmic GB/s from CUDA events, against the measured copy bandwidth."""
    import workloads as W
    h = 1.0 / (N + 1)
    c = W.medium_gaussian_bumps(1, N, N, N, h)
    P = hz.Problem(c, h, W.omega_for_ppw(c, h, 8.0), 12, 1.0, 1, 1.0, min(1.0, 64.0 / N),
                   nrhs_max=1, restart_max=1, inner_k_max=0)
    n = P.n
    x = torch.randn(1, n, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        P.apply_shifted(x, 0.3 - 1j, out=y)
    torch.cuda.synchronize()
    if profile_region:
        torch.cuda.profiler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record()
    for _ in range(reps):
        P.apply_shifted(x, 0.3 - 1j, out=y)
    e1.record()
    e1.synchronize()
    t_st = e0.elapsed_time(e1) / reps / 1e3
    P.shifted_solve(0, x, out=y)
    P.profile(True)
    P.shifted_solve(0, x, out=y)
    nl, ms, by = P.profile_read(hz.PROF_POLY)
    P.profile(False)
    if profile_region:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    P.close()
    peak, kind = measured_peak_hbm()
    st_gbs = 24.0 * n / t_st / 1e9
    poly_gbs = by / (ms / 1e3) / 1e9
    return {"grid": f"{N}^3", "peak": peak, "peak_kind": f"{kind} copy bandwidth",
            "stencil_c64": {"GB/s": st_gbs, "frac": st_gbs / peak, "us_per_launch": t_st * 1e6,
                            "bytes_per_point": 24},
            "poly_stage_c64_one_node": {"GB/s": poly_gbs, "frac": poly_gbs / peak,
                                        "us_per_launch": ms / nl * 1e3, "launches": nl}}


def batched_uneven(hz, torch, dev, precision):
    """12 instances (4 each of 48^3, 64^3, 96^3; layered media; 4 point sources each) solved
    together by hz_solve_batched, and one after another by hz_solve, to 1e-8."""
    import workloads as W
    wls = W.layered_batch()
    probs = [hz.Problem(w.c, w.h, w.omega, w.layer_cells, w.sigma_max, w.J, w.t, w.eps,
                        nrhs_max=w.nrhs, restart_max=w.restart, inner_k_max=w.k_in) for w in wls]
    fs = [torch.from_numpy(w.f.reshape(w.nrhs, -1).copy()).to(dev) for w in wls]
    kw = dict(restart=30, inner_k=4, rtol=1e-8, max_cycles=30, precision=precision, check=False)
    hz.solve_batched(probs, fs, **kw)  # warm-up: captures each problem's step graphs
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, stats = hz.solve_batched(probs, fs, **kw)
    e1.record()
    e1.synchronize()
    t_b = e0.elapsed_time(e1) / 1e3
    e0.record()
    for P, f in zip(probs, fs):
        P.solve(f, **kw)
    e1.record()
    e1.synchronize()
    t_s = e0.elapsed_time(e1) / 1e3
    flat = [x for st in stats for x in st]
    for P in probs:
        P.close()
    nr = len(flat)
    return {"workload": "12 instances: 4 x 48^3, 4 x 64^3, 4 x 96^3, layered media (5 layers, "
                        "c ~ U[1.5,4.5]), 8 ppw, J=8, 4 point sources each, FGMRES(30)",
            "rhs": nr, "converged": sum(x.converged for x in flat),
            "max_rel_res_true": max(x.rel_res_true for x in flat),
            "its_range": [min(x.its for x in flat), max(x.its for x in flat)],
            "batched_RHS_per_s": nr / t_b, "sequential_RHS_per_s": nr / t_s,
            "batched_s": t_b, "sequential_s": t_s}


def max_over_ranks_of(x: float, world: int, device) -> float:
    """The largest of each rank's x (a time), through the process group when world > 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1811_12378_gb300 as hz
    import workloads as W

    rank, local, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = W.gaussian_bumps_64()
    P = hz.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                   nrhs_max=1, restart_max=wl.restart, inner_k_max=wl.k_in)
    n = P.n
    f_host = torch.from_numpy(wl.f.reshape(1, n).copy()).pin_memory()
    f_dev = f_host.to(dev)
    u_dev = torch.empty_like(f_dev)
    u_host = torch.empty_like(f_host).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    kw = dict(restart=wl.restart, inner_k=wl.k_in, rtol=wl.rtol, max_cycles=20)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def timed(form, k, e2e=False):
        """Device time of k solves (events on the launching stream, L2 flushed between)."""
        total = 0.0
        stats = None
        for _ in range(k):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if e2e:
                f_dev.copy_(f_host, non_blocking=True)
            _, stats = P.solve(f_dev, out=u_dev, precision=form, **kw)
            if e2e:
                u_host.copy_(u_dev, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1) / 1e3
        return total, stats[0]

    def max_over_ranks(x):
        return max_over_ranks_of(x, world, dev)

    chosen = hz.HZ_MIXED_C64_FF
    # warm-up (all forms)
    for _ in range(max(args.warmup, 3)):
        P.solve(f_dev, out=u_dev, precision=chosen, **kw)
    P.solve(f_dev, out=u_dev, precision=hz.HZ_MIXED_C64_FCI32, **kw)
    P.solve(f_dev, out=u_dev, precision=hz.HZ_MIXED_C64, **kw)
    P.solve(f_dev, out=u_dev, precision=hz.HZ_C128, **kw)
    barrier()

    if args.ncu_region:
        torch.cuda.profiler.start()
        timed(chosen, args.steps)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        P.close()
        return

    # timed region: chosen form
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = hz.launch_count()
    barrier()
    t_mixed, st_mixed = timed(chosen, args.steps)
    barrier()
    launches = hz.launch_count() - launches0
    clk = clocks.stop()
    t_mixed = max_over_ranks(t_mixed)

    # the same steps again with CUDA events around every launch of each kernel class, on the
    # launching stream (the events cost host time, so the headline value above is taken
    # without them)
    P.profile(True)
    barrier()
    timed(chosen, args.steps)
    barrier()
    poly = P.profile_read(hz.PROF_POLY)
    sten = P.profile_read(hz.PROF_STENCIL)
    kryl = P.profile_read(hz.PROF_KRYLOV)
    P.profile(False)

    # plain float64 form and the form with float64 FCI internals, same steps
    barrier()
    t_plain, st_plain = timed(hz.HZ_C128, args.steps)
    t_plain = max_over_ranks(t_plain)
    barrier()
    t_m64, st_m64 = timed(hz.HZ_MIXED_C64, args.steps)
    t_m64 = max_over_ranks(t_m64)
    barrier()
    t_f32, st_f32 = timed(hz.HZ_MIXED_C64_FCI32, args.steps)
    t_f32 = max_over_ranks(t_f32)

    # end to end through the public API: pinned host f -> device, solve, u -> pinned host
    barrier()
    t_e2e, _ = timed(chosen, args.steps, e2e=True)
    t_e2e = max_over_ranks(t_e2e)

    # residual check of the last chosen-form solution with an independent float64 stencil
    s = P.info["s"]
    Au = P.apply_shifted(u_dev)
    res = float(torch.linalg.vector_norm(s * f_dev - Au) / torch.linalg.vector_norm(s * f_dev))

    # stencil and polynomial-stage HBM bandwidth on a grid larger than L2 (256^3: every
    # complex64 field is 134 MB), the configuration the HBM figures are meaningful on
    hbm = large_grid_bandwidth(hz, torch, dev)
    uneven = batched_uneven(hz, torch, dev, chosen) if world == 1 else None

    rhs_total = args.steps * world
    value = rhs_total / t_mixed
    peak, peak_kind = measured_peak_hbm()
    nl, ms, by = poly
    achieved = (by / nl) / ((ms / nl) / 1e3) / 1e9 if nl else None
    traffic = traffic_from_profile(kernel_hash())
    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_mixed / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f32pair+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "mixed, FCI in complex64: polynomial sweeps, "
                   "step d and inner GMRES in complex64, quadrature sum accumulated in float pairs "
                   "(~48 bits) and returned in float64; "
                   "outer FGMRES Arnoldi basis and CGS2 in float pairs (two float32, ~48 bits); "
                   "Hessenberg, Givens, solution update and true residual in float64",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "its": st_mixed.its, "matvecs": st_mixed.matvecs,
        "rel_res_true": st_mixed.rel_res_true, "rel_res_check": res,
        "plain": {"value": rhs_total / t_plain, "unit": "RHS/s",
                  "ms_per_step": t_plain / args.steps * 1e3, "dtype": "c128",
                  "its": st_plain.its, "rel_res_true": st_plain.rel_res_true},
        "fci32_f64_outer": {"value": rhs_total / t_f32, "unit": "RHS/s",
                            "ms_per_step": t_f32 / args.steps * 1e3,
                            "form": "FCI in complex64, outer Arnoldi in float64",
                            "its": st_f32.its, "rel_res_true": st_f32.rel_res_true},
        "mixed_f64_fci": {"value": rhs_total / t_m64, "unit": "RHS/s",
                          "ms_per_step": t_m64 / args.steps * 1e3,
                          "form": "complex64 sweeps only; step d, inner GMRES float64",
                          "its": st_m64.its, "rel_res_true": st_m64.rel_res_true},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic, "kernel": "k_poly_stage<float2> (batched sweeps)",
                     "launches": nl, "avg_launch_us": (ms / nl * 1e3) if nl else None,
                     "peak_kind": f"{peak_kind} copy bandwidth"},
        "kernel_classes": {
            "poly_stage": {"launches": poly[0], "ms": poly[1], "GB": poly[2] / 1e9},
            "stencil_f64": {"launches": sten[0], "ms": sten[1], "GB": sten[2] / 1e9},
            "krylov_f64": {"launches": kryl[0], "ms": kryl[1], "GB": kryl[2] / 1e9}},
        "e2e": {"value": rhs_total / t_e2e, "unit": "RHS/s", "h2d_bytes_per_step": n * 16,
                "d2h_bytes_per_step": n * 16},
        "stencil_hbm": hbm,
        "batched_uneven": uneven,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        counts = oracle_counts()[wl.name]
        per = 1
        t_cpu = time_oracle_sample(wl, per)
        line["cpu_baseline"] = {
            "value": 1.0 / (t_cpu / per * counts["its"]), "unit": "RHS/s",
            "cores": cpu_threads(), "kind": "oracle",
            "sample": f"{per} outer FGMRES step of the complex128 oracle on this workload "
                      f"({t_cpu:.2f} s), scaled by the oracle's {counts['its']} steps to 1e-8"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    P.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.ncu_large:
        import torch
        import paper_1811_12378_gb300 as hz
        print(json.dumps(large_grid_bandwidth(hz, torch, torch.device("cuda", 0),
                                              profile_region=True)))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
