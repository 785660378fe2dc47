#!/usr/bin/env python
"""Benchmark of the GB300 contour-integral Helmholtz solver.

Metric: right-hand sides per second solved to a relative residual of 1e-8 (float64 true
residual), for the 64^3 Gaussian-bump workload (8 bumps, c in [1, 2], 8 points per wavelength
at c_min, 8-cell sponge, one Gaussian source, J = 8 contour nodes, FGMRES(30) with FCI and 4
inner GMRES steps).  One step = one full solve of that right-hand side.  `value` is the mixed
form HZ_MIXED_C64 (complex64 polynomial sweeps; quadrature sum, step d, inner and outer CGS2,
Givens and true residual in float64); the plain all-float64 form and two faster forms that
depart from that precision split are reported beside it, each with its solution error against
the float64 oracle.  `large` solves the 256^3 configuration (8 of its 16 sources).

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
    ap.add_argument("--ncu-case", choices=["ilu", "net", "batched128", "spectral128",
                                           "spectral256"], default=None,
                    help="run only one profiling region, bracketed with cudaProfilerStart/Stop: "
                         "ilu = one FCI application with the ILU(0) inner preconditioner on the "
                         "64^3 workload (HZ_MIXED_C64); net = one forward pass and one training "
                         "step of the network on one 64^3 sample; batched128 = one FCI "
                         "application to 8 right-hand sides on a 128^3 Gaussian-bump medium "
                         "(8 nodes x 8 right-hand sides per polynomial stage, fields beyond L2); "
                         "spectral128 / spectral256 = one complex64 spectral operator "
                         "application (five line-FFT passes) on a 128^3 / 256^3 field")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 256^3 sixteen-source configuration's solve")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training and applying the learned preconditioner")
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
# The oracle is timed in processes of its own (spawned before this process touches the GPU),
# one numpy thread each: a full solve to 1e-8 on one core, the float64 reference solution that
# the GPU solutions are compared with (rtol 1e-12), and afterwards one bounded sample per host
# core at the same time (the all-core throughput).

def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def oracle_job(name: str, rtol: float, fixed_its: int = 0, want_u: bool = False):
    """One oracle FGMRES solve of a workload (runs in a worker process).  Returns its step
    count, true residual, wall-clock start/end of the solve and, if asked, the solution."""
    import numpy as np  # noqa: F401  (imported here, after the thread settings)
    import workloads as W
    from oracle import hz_oracle as O
    wl = getattr(W, name)()
    op = O.make_operator(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max)
    _, nodes = O.setup_nodes(op, wl.J, wl.t, wl.eps)
    t0 = time.time()
    res = O.solve(op, op.s * wl.f[0], nodes, wl.restart, wl.k_in, rtol, 60, fixed_its=fixed_its)
    t1 = time.time()
    return {"its": res.its, "rel_res_true": res.rel_res_true, "t0": t0, "t1": t1,
            "u": res.u.ravel() if want_u else None}


def oracle_pool(workers: int):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    _single_thread_env()
    return ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def oracle_counts():
    """The oracle's own step counts to 1e-8 (oracle/reference_counts.json, written by
    oracle/reference_counts.py, which calls only the oracle)."""
    with open(os.path.join(ROOT, "oracle", "reference_counts.json")) as fh:
        return json.load(fh)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    """--impl reference: the oracle (complex128 numpy, one thread) on the benchmark workload.
    Each timed step is a bounded sample: 4 outer FGMRES steps of the solve, scaled by the
    oracle's own step count to 1e-8."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    _single_thread_env()
    counts = oracle_counts()["gaussian_bumps_64"]
    per = 4
    for _ in range(args.warmup):
        oracle_job("gaussian_bumps_64", 1e-30, fixed_its=per)
    tt = []
    for _ in range(args.steps):
        r = oracle_job("gaussian_bumps_64", 1e-30, fixed_its=per)
        tt.append(r["t1"] - r["t0"])
    step_s = sum(tt) / len(tt)
    its = counts["its"]
    value = 1.0 / (step_s / per * its)
    sample = (f"{per} outer FGMRES steps of the oracle per timed step (FCI with "
              f"{counts['poly_matvecs_per_fci']} polynomial-sweep matvecs, 4 inner GMRES steps, "
              f"CGS2), scaled by the oracle's {its} steps to 1e-8; one numpy thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": {"workload": WORKLOAD, "form": "oracle complex128"},
        "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}), flush=True)


# ----------------------------------------------------------------------------- GPU arm
def traffic_from_profile(name: str, kernel_src_hash: str):
    """DRAM bytes per launch of a kernel from a committed ncu summary under profiles/, or None
    if the summary is missing or was taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", name)
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


def measured_peaks():
    """(HBM copy GB/s, kind) from MEASURED_PEAKS.json, else the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Float64 peak of a GB300 from its unit counts: 152 SMs x 2 float64 FMA per clock x 2 flops at
# the 2070 MHz maximum SM clock = 1.259 TFLOP/s (the part's published 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def l2_copy_bandwidth(torch, dev, mib=32, reps=200):
    """Copy bandwidth of a buffer pair that stays in the 126 MB L2 (read + write bytes / time,
    best of several event-timed bursts): the roof of kernels whose fields are L2-resident."""
    n = (mib << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    for _ in range(10):
        b.copy_(a)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        e1.synchronize()
        gbs = 2.0 * a.numel() * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
        best = gbs if best is None else max(best, gbs)
    return best


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
    peak, kind = measured_peaks()
    st_gbs = 24.0 * n / t_st / 1e9
    poly_gbs = by / (ms / 1e3) / 1e9
    return {"grid": f"{N}^3", "peak": peak, "peak_kind": f"{kind} copy bandwidth",
            "stencil_c64": {"GB/s": st_gbs, "frac": st_gbs / peak, "us_per_launch": t_st * 1e6,
                            "bytes_per_point": 24},
            "poly_stage_c64_one_node": {"GB/s": poly_gbs, "frac": poly_gbs / peak,
                                        "us_per_launch": ms / nl * 1e3, "launches": nl}}


def large_solve(hz, torch, dev, nrhs=8, profile_region=False):
    """The large configuration (256^3, 16 Gaussian bumps with c in [1, 3], 12-cell sponge,
    8 ppw, J = 8, FGMRES(40), 4 inner steps): the first nrhs of its 16 point sources solved to
    1e-8 in one call of the float64-outer mixed form (complex64 sweeps and stored directions),
    with per-kernel-class CUDA events (at this size a stage is milliseconds long, so the events
    cost nothing measurable).  The roofline is the batched polynomial stage's (J nodes x nrhs
    right-hand sides per launch, fields far beyond L2) against HBM."""
    import workloads as W
    wl, idx = W.large_bumps_256()
    N = wl.nx
    n = N ** 3
    P = hz.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                   nrhs_max=nrhs, restart_max=wl.restart, inner_k_max=wl.k_in,
                   flags=hz.HZ_LIMIT_SWEEPS_C64 | hz.HZ_LIMIT_Z_C64)
    f = torch.zeros((nrhs, n), dtype=torch.complex128, device=dev)
    for r, (i, j, k) in enumerate(idx[:nrhs]):
        f[r, i + N * (j + N * k)] = 1.0 / wl.h ** 3
    u = torch.empty_like(f)
    torch.cuda.synchronize()
    if profile_region:
        torch.cuda.profiler.start()
    P.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, st = P.solve(f, out=u, restart=wl.restart, inner_k=wl.k_in, rtol=wl.rtol, max_cycles=12,
                    precision=hz.HZ_MIXED_C64, check=False)
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    poly = P.profile_read(hz.PROF_POLY, flops=True)
    sten = P.profile_read(hz.PROF_STENCIL, flops=True)
    kryl = P.profile_read(hz.PROF_KRYLOV, flops=True)
    P.profile(False)
    if profile_region:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    info = P.info
    P.close()
    del f, u
    peak, kind = measured_peaks()
    gbs = poly[2] / (poly[1] / 1e3) / 1e9
    return {"workload": f"large_bumps_256: {N}^3 (h=1/{N + 1}), c = 1 + 16 seeded Gaussian bumps "
                        f"(width 0.1, amplitudes U[0,2]) clipped to [1,3], 8 ppw, 12-cell sponge, "
                        f"J=8, FGMRES(40) + FCI with 4 inner steps, point sources 1..{nrhs} of 16",
            "form": "HZ_MIXED_C64 (complex64 sweeps; float64 quadrature sum, step d, inner and "
                    "outer CGS2, Givens, true residual), sweep workspace and FGMRES directions "
                    "stored in complex64",
            "rhs": nrhs, "seconds": t, "RHS_per_s": nrhs / t,
            "converged": sum(1 for x in st if x.converged),
            "max_rel_res_true": max(x.rel_res_true for x in st),
            "its": [x.its for x in st], "stages_per_fci": info["stages"],
            "kernel_classes": {
                "poly_stage": {"launches": poly[0], "ms": poly[1], "GB": poly[2] / 1e9},
                "stencil": {"launches": sten[0], "ms": sten[1], "GB": sten[2] / 1e9,
                            "fp64_TFLOP": sten[3] / 1e12},
                "krylov": {"launches": kryl[0], "ms": kryl[1], "GB": kryl[2] / 1e9,
                           "fp64_TFLOP": kryl[3] / 1e12}},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": None,
                         "kernel": f"k_poly_stage<float2> ({wl.J} nodes x {nrhs} right-hand "
                                   f"sides per launch, 256^3 fields)",
                         "launches": poly[0], "avg_launch_us": poly[1] / poly[0] * 1e3,
                         "peak_kind": f"{kind} copy bandwidth"}}


def learned_preconditioner(hz, torch, dev, n_media=4, batches=4, nb=8, epochs=40, lr=1e-3,
                           sizes=(64, 128, 192)):
    """The learned right preconditioner: train the U-Net on the GPU (its own BF16 tensor-core
    kernels) from (residual, error) pairs of FCI on n_media random 64^3 Gaussian-bump media
    (r = v - A FCI(v) for smooth random v, e = A^{-1} r by a plain-method solve to 1e-6), then
    solve one fresh medium at each size to 1e-8 with FCI alone (mode 0) and with the network
    followed by FCI on its residual (mode 2).  All on the GPU; the true residual decides."""
    import numpy as np
    import workloads as W
    g = np.random.Generator(np.random.PCG64(11))

    def smooth(k, wl):
        r = g.standard_normal((k, wl.nz, wl.ny, wl.nx)) + 1j * g.standard_normal(
            (k, wl.nz, wl.ny, wl.nx))
        for _ in range(2):
            r = (r + np.roll(r, 1, 1) + np.roll(r, -1, 1) + np.roll(r, 1, 2) + np.roll(r, -1, 2)
                 + np.roll(r, 1, 3) + np.roll(r, -1, 3)) / 7.0
        return torch.from_numpy(r.reshape(k, -1)).to(dev)

    net = hz.Net(64, 64, 64, batch_max=nb)
    net.set_params(hz.flatten_params(hz.init_params(5)))
    data, probs = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for seed in range(1, 1 + n_media):
        wl = W.gaussian_bumps(64, seed)
        P = hz.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                       nrhs_max=nb, restart_max=30, inner_k_max=4)
        probs.append(P)
        s = P.info["s"]
        for _ in range(batches):
            v = smooth(nb, wl)
            z = P.fci(v, inner_k=4, precision=hz.HZ_MIXED_C64)
            t = (v - P.apply_shifted(z)).contiguous()
            e, _ = P.solve(t / s, restart=30, inner_k=4, rtol=1e-6, max_cycles=20,
                           precision=hz.HZ_MIXED_C64, check=False)
            data.append((P, t, e))
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = []
    for ep in range(epochs):
        tot = sum(net.train_fields(P, t, e, lr=lr) for (P, t, e) in data)
        if ep in (0, epochs - 1):
            losses.append(tot / len(data))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    params = net.get_params()
    net.close()
    del data
    for P in probs:
        P.close()
    out = {"training": {"media": n_media, "pairs": n_media * batches * nb, "epochs": epochs,
                        "adam_steps": epochs * n_media * batches, "batch": nb,
                        "pairs_s": t_pairs, "train_s": t_train, "loss_first_last": losses},
           "solves": []}
    for n in sizes:
        wl = W.gaussian_bumps(n, 100 + n)
        P = hz.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                       nrhs_max=1, restart_max=30, inner_k_max=4)
        f = torch.from_numpy(wl.f.reshape(1, -1).copy()).to(dev)
        netn = hz.Net(n, n, n, 1)
        netn.set_params(params)
        row = {"grid": f"{n}^3"}
        for mode in (0, 2):
            P.set_preconditioner(netn if mode else None, mode)
            cyc = 40 if mode == 0 or n < 192 else 3
            kw = dict(restart=30, inner_k=4, rtol=1e-8, max_cycles=cyc, precision=hz.HZ_MIXED_C64,
                      check=False)
            P.solve(f, **kw)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st = P.solve(f, **kw)
            e1.record()
            e1.synchronize()
            row[f"mode{mode}"] = {"its": st[0].its, "max_steps": cyc * 30,
                                  "converged": st[0].converged,
                                  "rel_res_true": st[0].rel_res_true,
                                  "ms": e0.elapsed_time(e1)}
        out["solves"].append(row)
        P.close()
        netn.close()
    return out


def next_rows_block(hz, torch, dev):
    """Case Two (Section 3 eq:mat-2x2, float64) against Case One on the 32^3 point source, and
    FCI with the ILU(0) inner preconditioner (Section 6.3, k_in = 4 and 8) against FCI alone on
    the headline 64^3 workload (HZ_MIXED_C64): one untimed and one event-timed solve each to
    a true relative residual of 1e-8."""
    import workloads as W

    def timed_solve(P, f, **kw):
        P.solve(f, **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, st = P.solve(f, **kw)
        e1.record()
        e1.synchronize()
        return {"its": st[0].its, "converged": st[0].converged,
                "rel_res_true": st[0].rel_res_true, "ms": e0.elapsed_time(e1)}

    def problem(wl, inner_k_max, flags=0):
        return hz.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                          nrhs_max=1, restart_max=wl.restart, inner_k_max=inner_k_max,
                          flags=flags)

    out = {}
    wl = W.point_source_32()
    f = torch.from_numpy(wl.f.reshape(1, -1).copy()).to(dev)
    row = {"workload": "point_source_32: 32^3 (h=1/33), c = 1, 10 ppw, 8-cell sponge, centre "
                       "point source, J=4, FGMRES(30) + FCI with 4 inner steps, float64"}
    for name, flags in (("case_one", 0), ("case_two", hz.HZ_LIMIT_CASE_TWO)):
        P = problem(wl, wl.k_in, flags)
        row[name] = timed_solve(P, f, restart=wl.restart, inner_k=wl.k_in, rtol=1e-8,
                                max_cycles=40)
        P.close()
    out["case_two"] = row
    wl = W.gaussian_bumps_64()
    f = torch.from_numpy(wl.f.reshape(1, -1).copy()).to(dev)
    P = problem(wl, 8)
    row = {"workload": "gaussian_bumps_64 (the headline workload), HZ_MIXED_C64, FGMRES(30)"}
    for name, ilu, kin in (("fci_k4", False, 4), ("ilu0_k4", True, 4), ("ilu0_k8", True, 8)):
        P.set_inner_ilu(ilu)
        row[name] = timed_solve(P, f, restart=wl.restart, inner_k=kin, rtol=1e-8, max_cycles=20,
                                precision=hz.HZ_MIXED_C64)
    P.close()
    out["ilu0"] = row
    return out


def spectral_block(hz, torch, dev, n=64, n_bw=256):
    """The Fourier spectral discretisation (Section 7.1) with the regularised inverse-Laplacian
    inner preconditioner (Section 7.3): one solve to 1e-8 of the n^3 periodic Gaussian-bump
    workload (2.25 points per wavelength in the background, J = 8, FGMRES(30), k_in = 4) per
    precision form, with and without the preconditioner; and the complex64 spectral operator
    (five line-FFT passes) on an n_bw^3 field, beyond L2, against the measured HBM copy rate."""
    import numpy as np
    import workloads as W
    wl = W.spectral_bumps(n, 1)
    P = hz.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                   nrhs_max=1, restart_max=wl.restart, inner_k_max=wl.k_in,
                   discretization=hz.HZ_DISC_SPECTRAL)
    f = torch.from_numpy(wl.f.reshape(1, -1).copy()).to(dev)
    out = {"workload": f"spectral_bumps_{n}: periodic {n}^3 box (h=1/{n}), c = 1 + 8 seeded "
                       f"Gaussian bumps (width 0.1, amplitudes U[0.5,1]) clipped to [1,2], "
                       f"2.25 ppw at c_min, 8-cell sponge, J=8, FGMRES(30) + FCI with 4 inner "
                       f"steps, rtol 1e-8", "solves": {}}
    for invlap in (False, True):
        P.set_inner_invlap(invlap)
        for name, prec in (("plain", hz.HZ_C128), ("mixed_f64", hz.HZ_MIXED_C64)):
            kw = dict(restart=wl.restart, inner_k=wl.k_in, rtol=1e-8, max_cycles=20,
                      precision=prec, check=False)
            P.solve(f, **kw)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st = P.solve(f, **kw)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            out["solves"][f"{name}{'_invlap' if invlap else ''}"] = {
                "RHS_per_s": 1.0 / t, "its": st[0].its, "converged": st[0].converged,
                "rel_res_true": st[0].rel_res_true}
    P.close()
    # the complex64 operator on a field beyond L2
    h = 1.0 / n_bw
    c = np.ones((n_bw, n_bw, n_bw))
    Q = hz.Problem(c, h, 2 * np.pi / (2.25 * h), 8, 1.0, 1, 1.0, 1.0, nrhs_max=1,
                   restart_max=1, inner_k_max=0, flags=hz.HZ_LIMIT_SWEEPS_C64,
                   discretization=hz.HZ_DISC_SPECTRAL)
    x = torch.randn(1, Q.n, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        Q.apply_shifted(x, 0.1, out=y, precision=hz.HZ_MIXED_C64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record()
    for _ in range(reps):
        Q.apply_shifted(x, 0.1, out=y, precision=hz.HZ_MIXED_C64)
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) / reps / 1e3
    Q.close()
    peak, kind = measured_peaks()
    by = 8.0 * Q.n * (10 + 2)  # five passes read and write the field; x and the diagonal again
    out["apply_c64"] = {"grid": f"{n_bw}^3", "us_per_apply": t * 1e6, "GB/s": by / t / 1e9,
                        "frac": by / t / 1e9 / peak, "peak": peak,
                        "peak_kind": f"{kind} copy bandwidth",
                        "bytes_per_point": 96}
    return out


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
    per = []
    for P, f in zip(probs, fs):
        e0.record()
        _, st1 = P.solve(f, **kw)
        e1.record()
        e1.synchronize()
        per.append((e0.elapsed_time(e1) / 1e3, max(x.its for x in st1)))
    t_s = sum(t for t, _ in per)
    flat = [x for st in stats for x in st]
    for P in probs:
        P.close()
    nr = len(flat)
    return {"workload": "12 instances: 4 x 48^3, 4 x 64^3, 4 x 96^3, layered media (5 layers, "
                        "c ~ U[1.5,4.5]), 8 ppw, J=8, 4 point sources each, FGMRES(30)",
            "form": "HZ_MIXED_C64",
            "rhs": nr, "converged": sum(x.converged for x in flat),
            "max_rel_res_true": max(x.rel_res_true for x in flat),
            "its_range": [min(x.its for x in flat), max(x.its for x in flat)],
            "batched_RHS_per_s": nr / t_b, "sequential_RHS_per_s": nr / t_s,
            "batched_s": t_b, "sequential_s": t_s,
            "sequential_per_instance": [{"grid": f"{w.nx}^3", "s": t, "max_its": k}
                                        for w, (t, k) in zip(wls, per)],
            "slowest_instance_s": max(t for t, _ in per)}


def max_over_ranks_of(x: float, world: int, device) -> float:
    """The largest of each rank's x (a time), through the process group when world > 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


FORMS = {  # key: (precision constant name, description)
    "mixed_f64": ("HZ_MIXED_C64", "complex64 stencil sweeps of the polynomial iteration; the "
                  "quadrature-weighted sum, step d, inner and outer CGS2 Arnoldi, Givens least "
                  "squares, solution update and true residual in float64"),
    "plain": ("HZ_C128", "everything complex128 / float64"),
    "fci32_f64_outer": ("HZ_MIXED_C64_FCI32", "departure: the whole FCI preconditioner in "
                        "complex64 (inner GMRES with float32 scalars, quadrature sum in float "
                        "pairs); outer FGMRES CGS2, Givens and true residual in float64"),
    "ff": ("HZ_MIXED_C64_FF", "departure: as fci32_f64_outer with the outer Arnoldi basis and "
           "CGS2 in float pairs (~48 bits); Hessenberg, Givens, update and residual float64"),
}
HEADLINE = "mixed_f64"


def run_ours(args):
    rank, local, world = dist_env()
    cpu_leg = rank == 0 and world == 1 and not args.no_cpu_baseline and not args.ncu_region
    pool = futs = None
    if cpu_leg:
        # the oracle's processes are spawned before this process touches the GPU
        pool = oracle_pool(2)
        futs = {"single": pool.submit(oracle_job, "gaussian_bumps_64", 1e-8),
                "ref": pool.submit(oracle_job, "gaussian_bumps_64", 1e-12, 0, True)}

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1811_12378_gb300 as hz
    import workloads as W

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
    prec = {k: getattr(hz, v[0]) for k, v in FORMS.items()}
    sols = {}

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
            _, stats = P.solve(f_dev, out=u_dev, precision=prec[form], **kw)
            if e2e:
                u_host.copy_(u_dev, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1) / 1e3
        if not e2e:
            sols[form] = u_dev.cpu().numpy()[0].copy()
        return total, stats[0]

    def max_over_ranks(x):
        return max_over_ranks_of(x, world, dev)

    # warm-up (all forms)
    for _ in range(max(args.warmup, 3)):
        P.solve(f_dev, out=u_dev, precision=prec[HEADLINE], **kw)
    for form in FORMS:
        P.solve(f_dev, out=u_dev, precision=prec[form], **kw)
    barrier()

    if args.ncu_region:
        torch.cuda.profiler.start()
        timed(HEADLINE, args.steps)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        P.close()
        return

    # timed region: the headline form
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = hz.launch_count()
    barrier()
    t_head, st_head = timed(HEADLINE, args.steps)
    barrier()
    launches = hz.launch_count() - launches0
    clk = clocks.stop()
    t_head = max_over_ranks(t_head)

    # the same steps again with CUDA events around every launch of each kernel class, on the
    # launching stream (the events cost host time, so the headline value above is taken
    # without them)
    P.profile(True)
    barrier()
    timed(HEADLINE, args.steps)
    barrier()
    cls = {"poly_stage": P.profile_read(hz.PROF_POLY, flops=True),
           "stencil": P.profile_read(hz.PROF_STENCIL, flops=True),
           "krylov": P.profile_read(hz.PROF_KRYLOV, flops=True)}
    P.profile(False)

    # the other forms, same steps
    others = {}
    for form in FORMS:
        if form == HEADLINE:
            continue
        barrier()
        t_f, st_f = timed(form, args.steps)
        others[form] = (max_over_ranks(t_f), st_f)

    # end to end through the public API: pinned host f -> device, solve, u -> pinned host
    barrier()
    t_e2e, _ = timed(HEADLINE, args.steps, e2e=True)
    t_e2e = max_over_ranks(t_e2e)

    # residual check of the headline solution with an independent float64 stencil
    s = P.info["s"]
    u_dev.copy_(torch.from_numpy(sols[HEADLINE][None]).to(dev))
    Au = P.apply_shifted(u_dev)
    res = float(torch.linalg.vector_norm(s * f_dev - Au) / torch.linalg.vector_norm(s * f_dev))

    # the precision floor of every form: solves to a true residual of 1e-11 (untimed)
    sols11 = {}
    for form in FORMS:
        u11, st11 = P.solve(f_dev, restart=wl.restart, inner_k=wl.k_in, rtol=1e-11,
                            max_cycles=40, precision=prec[form], check=False)
        sols11[form] = (u11.cpu().numpy()[0].copy(), st11[0].rel_res_true)
    P.close()

    l2_peak = l2_copy_bandwidth(torch, dev)
    # stencil and polynomial-stage HBM bandwidth on a grid larger than L2 (256^3: every
    # complex64 field is 134 MB), the configuration the HBM figures are meaningful on
    hbm = large_grid_bandwidth(hz, torch, dev)
    large = large_solve(hz, torch, dev) if world == 1 and not args.no_large else None
    uneven = batched_uneven(hz, torch, dev, prec[HEADLINE]) if world == 1 else None
    learned = (learned_preconditioner(hz, torch, dev) if world == 1 and not args.no_learned
               else None)
    spectral = spectral_block(hz, torch, dev) if world == 1 else None
    next_rows = next_rows_block(hz, torch, dev) if world == 1 else None

    rhs_total = args.steps * world
    value = rhs_total / t_head
    peak_hbm, peak_kind = measured_peaks()

    # roofline of the dominant kernel class of the headline solve
    dom = max(cls, key=lambda k: cls[k][1])
    nl, ms, by, fl = cls[dom]
    if dom == "poly_stage":
        achieved = (by / nl) / ((ms / nl) / 1e3) / 1e9
        roof = {"bound": "l2", "achieved": achieved, "peak": l2_peak, "unit": "GB/s",
                "frac": achieved / l2_peak,
                "traffic": traffic_from_profile("poly_stage_gaussian_bumps_64.txt", kernel_hash()),
                "kernel": "k_poly_stage<float2> (batched sweeps of all active contour nodes)",
                "peak_kind": "measured L2-resident copy bandwidth (32 MiB buffers, this run); "
                             "the 64^3 fields stay in L2, so HBM is not the roof here"}
    else:
        achieved = (fl / nl) / ((ms / nl) / 1e3) / 1e12
        traffic = (traffic_from_profile("cgs_f64_gaussian_bumps_64.txt", kernel_hash())
                   if dom == "krylov" else None)
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                "kernel": f"{dom} class (float64 Krylov kernels: CGS2 passes, step d)"
                          if dom == "krylov" else "k_stencil_diag (float64 stencil)",
                "peak_kind": "float64 FMA rate from unit counts (152 SMs x 2 FMA/clk x 2 flops "
                             "x 2.07 GHz)"}
    roof.update({"class": dom, "launches": nl, "avg_launch_us": ms / nl * 1e3})

    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_head / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": f"{FORMS[HEADLINE][0]}: {FORMS[HEADLINE][1]}",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "its": st_head.its, "matvecs": st_head.matvecs,
        "matvecs_per_s": st_head.matvecs * value,
        "rel_res_true": st_head.rel_res_true, "rel_res_check": res,
        "roofline": roof,
        "kernel_classes": {k: {"launches": v[0], "ms": v[1], "GB": v[2] / 1e9,
                               "fp64_TFLOP": v[3] / 1e12} for k, v in cls.items()},
        "e2e": {"value": rhs_total / t_e2e, "unit": "RHS/s", "h2d_bytes_per_step": n * 16,
                "d2h_bytes_per_step": n * 16},
        "l2_copy_GBps": l2_peak,
        "stencil_hbm": hbm,
        "large": large,
        "batched_uneven": uneven,
        "learned_preconditioner": learned,
        "spectral": spectral,
        "next_rows": next_rows,
        "gpu_launches": launches,
        "clocks": clk,
    }
    for form, (t_f, st_f) in others.items():
        line[form] = {"value": rhs_total / t_f, "unit": "RHS/s",
                      "ms_per_step": t_f / args.steps * 1e3, "form": FORMS[form][1],
                      "its": st_f.its, "rel_res_true": st_f.rel_res_true}
    if cpu_leg:
        ref = futs["ref"].result()
        single = futs["single"].result()
        pool.shutdown()
        uref = ref["u"]
        nref = float(np.linalg.norm(uref))
        errs = {}
        for form in FORMS:
            errs[form] = {
                "at_rtol_1e-8": float(np.linalg.norm(sols[form] - uref) / nref),
                "at_rtol_1e-11": float(np.linalg.norm(sols11[form][0] - uref) / nref),
                "rel_res_true_1e-11_solve": sols11[form][1]}
        line["err_vs_oracle"] = {
            "reference": f"oracle float64 solution at a true residual of "
                         f"{ref['rel_res_true']:.2e} ({ref['its']} steps)",
            "forms": errs}
        # all-core sample: one bounded sample per host core at the same time
        cores = host_cores()
        per = 6
        allp = oracle_pool(cores)
        jobs = [allp.submit(oracle_job, "gaussian_bumps_64", 1e-30, per) for _ in range(cores)]
        rs = [j.result() for j in jobs]
        allp.shutdown()
        wall = max(r["t1"] for r in rs) - min(r["t0"] for r in rs)
        its8 = single["its"]
        line["cpu_baseline"] = {
            "value": cores * per / its8 / wall, "unit": "RHS/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{cores} processes (one numpy thread each) each timing {per} outer FGMRES "
                      f"steps of the oracle on this workload at the same time ({wall:.1f} s "
                      f"wall), scaled by the oracle's {its8} steps to 1e-8 measured below"}
        line["cpu_baseline_single_core"] = {
            "value": 1.0 / (single["t1"] - single["t0"]), "unit": "RHS/s", "cores": 1,
            "kind": "oracle",
            "sample": f"one full oracle solve of this workload to 1e-8 ({single['its']} steps, "
                      f"{single['t1'] - single['t0']:.1f} s, true residual "
                      f"{single['rel_res_true']:.2e}), one numpy thread, run beside the GPU part"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def ncu_case(case: str):
    """One small profiling region on the 64^3 workload (cudaProfilerStart/Stop around it, two
    untimed repetitions before)."""
    import torch
    import paper_1811_12378_gb300 as hz
    import workloads as W
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(3)
    if case == "ilu":
        wl = W.gaussian_bumps_64()
        P = hz.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                       nrhs_max=1, restart_max=wl.restart, inner_k_max=wl.k_in)
        P.set_inner_ilu(True)
        r = torch.randn(1, P.n, dtype=torch.complex128, generator=g).to(dev)

        def body():
            P.fci(r, inner_k=wl.k_in, precision=hz.HZ_MIXED_C64)
    elif case in ("spectral128", "spectral256"):
        import numpy as np
        nb = 128 if case == "spectral128" else 256
        h = 1.0 / nb
        P = hz.Problem(np.ones((nb, nb, nb)), h, 2 * np.pi / (2.25 * h), 8, 1.0, 1, 1.0, 1.0,
                       nrhs_max=1, restart_max=1, inner_k_max=0, flags=hz.HZ_LIMIT_SWEEPS_C64,
                       discretization=hz.HZ_DISC_SPECTRAL)
        x = torch.randn(1, P.n, dtype=torch.complex64, generator=g).to(dev)
        y = torch.empty_like(x)

        def body():
            P.apply_shifted(x, 0.1, out=y, precision=hz.HZ_MIXED_C64)
    elif case == "batched128":
        wl = W.gaussian_bumps(128, 7)
        P = hz.Problem(wl.c, wl.h, wl.omega, wl.layer_cells, wl.sigma_max, wl.J, wl.t, wl.eps,
                       nrhs_max=8, restart_max=1, inner_k_max=wl.k_in,
                       flags=hz.HZ_LIMIT_SWEEPS_C64)
        r = torch.randn(8, P.n, dtype=torch.complex128, generator=g).to(dev)

        def body():
            P.fci(r, inner_k=wl.k_in, precision=hz.HZ_MIXED_C64)
    else:
        net = hz.Net(64, 64, 64, batch_max=1)
        net.set_params(hz.flatten_params(hz.init_params(5)))
        x = torch.randn(1, 64, 64, 64, 8, generator=g)
        x[..., 3:] = 0
        x = x.to(dev)
        t = torch.randn(1, 64, 64, 64, 2, generator=g).to(dev)

        def body():
            net.forward(x)
            net.train_step(x, t, lr=1e-4)
    for _ in range(2):
        body()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    body()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"ncu_case": case, "ok": True}))


def main():
    args = parse()
    if args.ncu_case:
        ncu_case(args.ncu_case)
        return
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
