"""Benchmark of the GB300 MRT-Smagorinsky LBM step (one JSON line on stdout).

Workload (headline): the forced-HIT DNS shape, an 800^3 periodic lattice
(5.12e8 cells) with FP32 storage, seeded random solenoidal initial field
(k^4 exp(-2 (k/4)^2), u_rms = 0.05, generated on the device by the library),
the paper's sinusoidal forcing with U0 = 0.043, Cf = 0.2 (F0 = 4.6225e-7),
C = 0 and nu0 from Re = 2e4 (nu0 = 0.00172).  A step is one launch of the
fused stream + collide kernel over all cells; MLUPS = cells x steps / time.
Extra entries: the same lattice with FP16 and BF16 weight-shifted storage;
the 100^3 LES (C = 0.13, nu0 = 2.15e-4, FP32) against an L2-resident copy
rate measured beside it; the 100^3 LES run of 20,000 steps with the
statistics cadence of the paper (every 500 steps); the 48-instance batch
over 5,000 steps; the 800^3 storage study over 2,000 steps; the
Smagorinsky-constant sweep at 128^3 with its ESS exponents.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs as torchrun ranks, one independent lattice per GPU (replicas: the
method has no exchange step on one box), value = total cell updates of all
ranks / max rank time.  --impl reference times the FP64 CPU oracle on a
bounded 128^3 sample of the same setup on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = {0: 152, 1: 76, 2: 76}  # 19 loads + 19 stores of one stored population
DTYPE_NAME = {0: "f32", 1: "f32 (f16 storage)", 2: "f32 (bf16 storage)"}
U0, CF, RE = 0.043, 0.2, 2.0e4


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# Nominal HBM3e bandwidth of one GB300 (~8 TB/s), the second denominator the
# roofline fractions are quoted against beside the measured copy bandwidth.
NOMINAL_HBM_GBS = 8000.0


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6750.0)), "measured"
    return 6800.0, "fallback"


def traffic_per_update(kernel_digest: str, storage: str = "fp32"):
    """DRAM bytes per cell update of the step kernel (FP32 or FP16 storage) from
    the committed ncu summary, or None when the kernel source changed since the
    capture."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for ln in fh:
            if ":" in ln and not ln.startswith("#"):
                k, v = ln.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_digest") != kernel_digest:
        return None
    key = f"dram_bytes_per_update_{storage}"
    return float(vals[key]) if key in vals else None


# Sources that define the step kernel k_step_tma and what it computes per cell.
STEP_KERNEL_SOURCES = ("lbm_device.cuh", "lbm_internal.h", "lbm_kernels.h", "lbm_reduce.cuh",
                       "lbm_step_tma.cu")


def _code_only(text: str) -> str:
    """C++ source without comments, blank lines and trailing blanks."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_digest(csrc: str = "") -> str:
    """Hash of the step kernel's code (comments excluded): a committed ncu
    traffic figure is only reported while it matches."""
    import hashlib
    h = hashlib.sha256()
    csrc = csrc or os.path.join(ROOT, "paper_2512_23116_gb300", "csrc")
    for f in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, f)) as fh:
            h.update(f.encode())
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"lbm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for ln in fh:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_mlups(n: int, seconds: float, nu0: float, C: float, threads: int = 0):
    """The FP64 CPU oracle as it stands, on an n^3 sample, for ~`seconds`
    (threads = 0: every host thread, OpenMP)."""
    import oracle
    import synthetic
    oracle.build()
    u = synthetic.random_solenoidal(n, seed=1, urms=0.05)
    F0 = oracle.forcing_amplitude(CF, U0, n)
    L = oracle.OracleLBM(n, n, n, nu0, C, oracle.FORCE_PAPER_SIN, F0=F0)
    L.init_equilibrium(u)
    L.step(1, threads)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        L.step(1, threads)
        steps += 1
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt / 1e6, steps, dt


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = 128
    nu0 = U0 * n / RE
    import oracle
    import synthetic
    oracle.build()
    u = synthetic.random_solenoidal(n, seed=1, urms=0.05)
    L = oracle.OracleLBM(n, n, n, nu0, 0.0, oracle.FORCE_PAPER_SIN, F0=oracle.forcing_amplitude(CF, U0, n))
    L.init_equilibrium(u)
    L.step(args.warmup)
    t0 = time.perf_counter()
    L.step(args.steps)
    dt = time.perf_counter() - t0
    value = n ** 3 * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": "MLUPS (stream+collide, D3Q19 MRT-Smagorinsky-Guo)",
        "value": value, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"forced-HIT DNS shape (800^3 setup), bounded {n}^3 sample for the FP64 CPU oracle",
                   "cells": n ** 3, "C": 0.0, "nu0": nu0, "Re": RE},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": host_cores(), "kind": "oracle",
                         "sample": f"{n}^3, {args.steps} steps after {args.warmup} warm-up"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def aggregate_ranks(ms: float, e2e_ms: float, cells_per_rank: int, steps: int, world: int,
                    device=None):
    """Whole-job numbers of a replicas run: the slowest rank's times (MAX over
    ranks) and the cell updates of all ranks.  Returns (value MLUPS, e2e MLUPS,
    max ms, max e2e ms).  With world == 1 no collective is called."""
    import torch
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max, e2e_max = float(t[0]), float(t[1])
    total = world * cells_per_rank * steps
    return total / (ms_max * 1e-3) / 1e6, total / (e2e_max * 1e-3) / 1e6, ms_max, e2e_max


SEED, URMS, K0 = 1, 0.05, 4.0  # the seeded random field of every workload


def time_steps(lbm, lat, stream, steps, warmup, dist):
    import torch
    lat.step(warmup)
    lat.sync()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    lat.step(steps)
    stop.record(stream)
    stop.synchronize()
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    ms = start.elapsed_time(stop)
    return ms


def config_of(cfg: dict) -> str:
    """The --config string (kind, tile rows, stages, threads, tma_slots) that
    reproduces a handle's kernel configuration (lbm_kernel_config)."""
    slots = {0: 1, 2880: 2}.get(cfg["slot_bytes"], 0) if cfg["kind"] == 2 else 0
    return f"{cfg['kind']},{cfg['tile_rows']},{cfg['stages']},{cfg['threads']},{slots}"


def run_case(lbm, n, precision, C, nu0, steps, warmup, device, stream, dist, clocks=None,
             config="", shape=None, row_align=0, layout=0, u_out=None, strain_mode=0):
    """Create, initialise from the library's seeded random field (u_out, when
    given, receives its FP32 velocity), time `steps` steps."""
    kind = rows = stages = threads = slots = 0
    if config:
        vals = [int(v) for v in config.split(",")]
        kind, rows, stages, threads = vals[:4]
        slots = vals[4] if len(vals) > 4 else 0
    nx, ny, nz = shape if shape else (n, n, n)
    p = lbm.make_params(nx, ny, nz, precision=precision, nu0=nu0, cs=C, f0=CF * U0 * U0 / nx,
                        force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device, stream=stream.cuda_stream,
                        kernel=kind, tile_rows=rows, stages=stages, threads=threads, row_align=row_align,
                        layout=layout, tma_slots=slots, strain_mode=strain_mode)
    lat = lbm.Lattice(p)
    lat.init_random(seed=SEED, urms=URMS, k0=K0, u_out=u_out)
    if clocks is not None:
        with clocks:
            ms = time_steps(lbm, lat, stream, steps, warmup, dist)
    else:
        ms = time_steps(lbm, lat, stream, steps, warmup, dist)
    cfg = lat.config()
    st = lat.stats()
    return lat, ms, cfg, st


def batch_case(lbm, device, stream, steps, warmup):
    """48 independent LES instances (12 each of 64^3, 96^3, 100^3, 128^3, seeds
    1..48, C = 0.13, nu0 from Re = 2e4 at each N, the paper's forcing) in one
    handle (one launch per step over all instances) against the same 48
    instances run one after the other as single-instance handles."""
    import torch
    sizes = [64] * 12 + [96] * 12 + [100] * 12 + [128] * 12

    def params(n):
        return lbm.make_params(n, nu0=U0 * n / RE, cs=0.13, f0=CF * U0 * U0 / n,
                               force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device,
                               stream=stream.cuda_stream)

    cells = sum(n ** 3 for n in sizes)
    lat = lbm.Lattice([params(n) for n in sizes])
    for i, n in enumerate(sizes):
        lat.init_random(seed=i + 1, urms=URMS, k0=K0, inst=i)
    ms_batch = time_steps(lbm, lat, stream, steps, warmup, False)
    cfg = lat.config()
    lat.close()
    # the same 48 instances as 48 single-instance handles: (a) each run to
    # completion one after the other (each small lattice then lives in L2),
    # (b) round robin, one step of every instance per ensemble step
    ms_seq = 0.0
    singles = []
    for i, n in enumerate(sizes):
        one = lbm.Lattice(params(n))
        one.init_random(seed=i + 1, urms=URMS, k0=K0)
        ms_seq += time_steps(lbm, one, stream, steps, warmup, False)
        singles.append(one)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        for one in singles:
            one.step(1)
    stop.record(stream)
    stop.synchronize()
    ms_rr = start.elapsed_time(stop)
    for one in singles:
        one.close()
    return {"instances": len(sizes), "sizes": "12 each of 64^3, 96^3, 100^3, 128^3", "cells": cells,
            "steps": steps, "MLUPS_batched": cells * steps / (ms_batch * 1e-3) / 1e6,
            "MLUPS_sequential_to_completion": cells * steps / (ms_seq * 1e-3) / 1e6,
            "MLUPS_sequential_round_robin": cells * steps / (ms_rr * 1e-3) / 1e6,
            "speedup_vs_round_robin": ms_rr / ms_batch, "speedup_vs_to_completion": ms_seq / ms_batch,
            "ms_per_step_batched": ms_batch / steps, "kernel": cfg,
            "note": "5.09e7 cells, 3.9 GB FP32 batched (HBM); a single instance of 64^3-100^3 "
                    "fits in L2 when run to completion"}


def max_shell(nx, ny, nz):
    """Largest integer shell s (s - 1/2 <= |k| < s + 1/2) holding a mode of an
    nx x ny x nz box (the shells lbm_spectrum bins into)."""
    K = (nx // 2) ** 2 + (ny // 2) ** 2 + (nz // 2) ** 2
    r = math.isqrt(K)
    return r + 1 if K > r * r + r else r


def _dissipation_shell(E, n):
    """Last shell before E falls below 1e-3 of its peak (bounded by N/3)."""
    peak = float(np.max(E[1:]))
    kd = 1
    for s_ in range(1, min(len(E), n // 3 + 1)):
        if E[s_] < 1e-3 * peak:
            break
        kd = s_
    return kd


def _spectral_error(E, E_ref, n):
    kd = _dissipation_shell(E_ref, n)
    rel = np.abs(E[1:kd + 1] - E_ref[1:kd + 1]) / E_ref[1:kd + 1]
    return {"max_rel_error_shells_1_to_kd": float(rel.max()), "mean_rel_error": float(rel.mean()),
            "kd": kd}


def precision_study(lbm, device, stream, n=800, steps=2000, every=100):
    """The DNS-shape storage study (C = 0, nu0 from Re = 2e4, the paper's
    forcing, seeded random field, `steps` steps, a spectrum every `every`
    steps) with FP32, FP16-shifted and BF16-shifted storage, for two readings
    of the initial u_rms = 0.05: per component (sqrt(<u.u>/3), the definition
    of Eq. rms_velocity; peaks near Mach 0.4) and as the magnitude
    (sqrt(<u.u>) = 0.05, per component 0.05/sqrt(3)).  Per storage: the steps
    it ran with finite statistics, its throughput including the spectra, E_k
    at the end; for FP16 / BF16 the per-shell error of the time-averaged
    spectrum against FP32 storage (shells 1..kd, kd where E falls below 1e-3
    of its peak, at most N/3) over the records every storage has, and over
    their second half.  (The errors against the FP64 oracle are GPU tests at
    64^3 and 128^3.)"""
    import torch
    kmax = max_shell(n, n, n)
    nu0 = U0 * n / RE
    out = {"n": n, "steps": steps, "spectrum_every": every, "C": 0.0, "nu0": nu0}
    for reading, urms in (("u_rms_per_component_0.05", URMS), ("u_rms_magnitude_0.05", URMS / math.sqrt(3.0))):
        spectra, rows = {}, {}
        for prec, name in ((0, "fp32"), (1, "fp16_shifted"), (2, "bf16_shifted")):
            p = lbm.make_params(n, precision=prec, nu0=nu0, cs=0.0, f0=CF * U0 * U0 / n,
                                force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device, stream=stream.cuda_stream)
            row, Es = {}, []
            with lbm.Lattice(p) as L:
                L.init_random(seed=SEED, urms=urms, k0=K0)
                L.sync()
                t0 = time.perf_counter()
                try:
                    while L.time < steps:
                        L.step(every)
                        Es.append(L.spectrum(kmax))
                    row["steps_finite"] = L.time
                    row["E_k_end"] = L.stats()["E_k"]
                except lbm.LbmError as exc:
                    if exc.code != lbm.LBM_ERR_UNSTABLE:
                        raise
                    row["steps_finite"] = L.time - every
                    row["unstable_by_step"] = L.time
                wall = time.perf_counter() - t0
            row["MLUPS_incl_spectra"] = n ** 3 * row["steps_finite"] / wall / 1e6
            rows[name], spectra[name] = row, Es
        common = min(len(v) for v in spectra.values())
        for name in ("fp16_shifted", "bf16_shifted"):
            if common >= 2:
                ref = np.array(spectra["fp32"][:common])
                mine = np.array(spectra[name][:common])
                half = common // 2
                rows[name]["vs_fp32_records"] = common
                rows[name]["vs_fp32_window_steps"] = common * every
                rows[name]["vs_fp32_window"] = _spectral_error(mine.mean(axis=0), ref.mean(axis=0), n)
                rows[name]["vs_fp32_second_half_of_window"] = _spectral_error(mine[half:].mean(axis=0),
                                                                              ref[half:].mean(axis=0), n)
            if "E_k_end" in rows[name] and "E_k_end" in rows["fp32"]:
                rows[name]["E_k_end_rel_diff_vs_fp32"] = abs(rows[name]["E_k_end"] - rows["fp32"]["E_k_end"]) / \
                    rows["fp32"]["E_k_end"]
        out[reading] = {"u_rms_per_component": urms, "storage": rows}
        torch.cuda.empty_cache()
    return out


def sweep(lbm, device, stream, sizes=(128, 256, 512, 1024), steps=500, warmup=5):
    """Roofline sweep: N^3 for each N, FP32 and FP16-shifted storage, the LES
    setting (C = 0.13, nu0 from Re = 2e4 at each N, the paper's forcing).  (The
    spectral error of both storages against the FP64 oracle at N = 128 is a GPU
    test.)"""
    import torch
    hbm_peak, _ = measured_peaks()
    rows = []
    for n in sizes:
        for prec in (0, 1):
            p = lbm.make_params(n, precision=prec, nu0=U0 * n / RE, cs=0.13, f0=CF * U0 * U0 / n,
                                force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device, stream=stream.cuda_stream)
            with lbm.Lattice(p) as L:
                L.init_random(seed=SEED, urms=URMS, k0=K0)
                ms = time_steps(lbm, L, stream, steps, warmup, False)
                cfg = L.config()
            gbs = n ** 3 * BYTES_PER_UPDATE[prec] * steps / (ms * 1e-3) / 1e9
            rows.append({"N": n, "storage": ["fp32", "fp16_shifted"][prec], "steps": steps,
                         "MLUPS": n ** 3 * steps / (ms * 1e-3) / 1e6, "GB_s": gbs, "frac_hbm": gbs / hbm_peak,
                         "frac_of_nominal": gbs / NOMINAL_HBM_GBS, "kernel": cfg})
        torch.cuda.empty_cache()
    return {"rows": rows}


def ess_exponents(st, lo=2, hi=16):
    """Extended self-similarity (Sec. 3.4): slopes zeta_p / zeta_3 of log S_p
    against log |S_3| over lo <= r <= hi, p = 2, 4, 6, from the structure
    functions of an lbm_stats result."""
    r = np.array(st["r"], dtype=float)
    Sp = st["Sp"]
    sel = (r >= lo) & (r <= hi)
    s3 = np.log(np.abs(Sp[sel, 2]))
    return {p_: float(np.polyfit(s3, np.log(np.abs(Sp[sel, p_ - 1])), 1)[0]) for p_ in (2, 4, 6)}


def c_sweep(lbm, device, stream, n=128, re=5000.0, cs=(0.0, 0.1, 0.16, 0.25), steps=4000,
            every=250):
    """The Smagorinsky-constant sweep of Sec. 3.3 (Fig. c_variation): n^3, Re = 5000,
    C in {0, 0.1, 0.16, 0.25}, the paper's forcing, from the seeded random field.
    Reports the spectrum time-averaged over the second half of the run, the
    high-k pile-up indicator E(n/3)/E(peak), and the ESS exponents zeta_p/zeta_3
    (slopes of log S_p against log |S_3| over r = 2..16, Sec. 3.4) from the
    structure functions of the last state."""
    import torch
    kmax = max_shell(n, n, n)
    out = {}
    for C in cs:
        nu0 = U0 * n / re
        p = lbm.make_params(n, nu0=nu0, cs=C, f0=CF * U0 * U0 / n, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                            device=device, stream=stream.cuda_stream)
        row = {"C": C, "nu0": nu0}
        try:
            with lbm.Lattice(p) as L:
                L.init_random(seed=SEED, urms=URMS, k0=K0)
                E = np.zeros(kmax + 1)
                navg = 0
                while L.time < steps:
                    L.step(every)
                    L.sync()
                    if L.time > steps // 2:
                        E += L.spectrum(kmax)
                        navg += 1
                st = L.stats(what=lbm.LBM_STATS_STRUCTURE)
            E /= max(1, navg)
            peak = int(np.argmax(E[1:])) + 1
            row["E"] = [float(f"{v:.4e}") for v in E[:n // 2 + 1]]
            row["pileup_E(n/3)/E(peak)"] = float(E[n // 3] / E[peak])
            row["ESS_zeta_p_over_zeta_3"] = ess_exponents(st)
            row["F4_r1"] = float(st["F4"][0])
            row["theta_mean"] = st["theta_mean"]
        except lbm.LbmError as exc:
            if exc.code != lbm.LBM_ERR_UNSTABLE:
                raise
            row["unstable"] = True
        out[f"C={C}"] = row
    return {"n": n, "Re": re, "steps": steps, "c_sweep": out}


def les_c2_run(lbm, device, stream, n=100, steps=20000, every=500, plane=50, spread_seeds=(2, 3)):
    """The paper's LES workload as one job (Sec. 3.1, Sec. 4.1): n^3, C = 0.13,
    nu0 from Re = 2e4, the paper's forcing, from the seeded random field,
    `steps` steps with the statistics cadence of the paper's post-processing
    ("computed on the fly at set intervals"): every `every` steps the library's
    statistics time series (paper_2512_23116_gb300.series: the domain
    statistics with the derived scales and S_p / F4 by separation, the shell
    spectrum, and a theta = tau_e - 1/2 slice at z = `plane`, the K_t map)
    written as JSON lines, with the fused in-step records
    (lbm_params.stats_every) besides.  Wall time of the whole job with that
    cadence against the same steps without it (the first statistics call's
    one-time FFT setup timed on its own); late-time theta statistics
    (t >= steps / 2) beside the values the paper prints for its 100^3 LES
    (Sec. 4.1: mean ~1.34e-3, 5th percentile > 1.0e-3, 95th <~ 1.82e-3, maxima
    up to ~3.7e-3), context only: the paper's statistics are over t/t0 in
    [200, 600] of a stationary state, this run starts from the synthetic
    field.  The same job from the seeds `spread_seeds` (untimed) gives the
    seed-to-seed spread of those late-time statistics."""
    import tempfile

    import torch
    from paper_2512_23116_gb300 import series
    nu0 = U0 * n / RE

    def params(stats_every):
        return lbm.make_params(n, nu0=nu0, cs=0.13, f0=CF * U0 * U0 / n, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                               device=device, stream=stream.cuda_stream, stats_every=stats_every)

    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "c2_series.jsonl")
        with lbm.Lattice(params(every)) as L:
            L.init_random(seed=SEED, urms=URMS, k0=K0)
            L.sync()
            # one-time setup of the first statistics call, timed on its own: the
            # FFT plan and the loading of its kernels (once per process and size)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lbm.lbm_stats(L.h, 0, lbm.LBM_STATS_SPECTRUM | lbm.LBM_STATS_STRUCTURE)
            lbm.lbm_get_theta_slice(L.h, 0, 2, plane, L.shapes[0])
            first_call = time.perf_counter() - t0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            recs = series.run_with_statistics(L, steps, every, path, theta_slice=(2, plane))
            fused = L.series()
            wall_cadence = time.perf_counter() - t0
        lines = len(series.read_series(path))

        def late_rows(records):
            rows = []
            for r in records:
                if r["step"] >= steps // 2:
                    sl = np.load(os.path.join(tmp, r["theta_slice"]["file"]))
                    rows.append((r["theta_mean"], r["theta_p05"], r["theta_p50"], r["theta_p95"],
                                 r["theta_p99"], r["theta_max"], float(sl.mean()), float(sl.max()), r["F4"][0],
                                 r["Re_lambda"], r["E_k"]))
            return np.array(rows)

        late = late_rows(recs)
        per_seed = [late.mean(axis=0)]
        for seed in spread_seeds:
            with lbm.Lattice(params(every)) as L:
                L.init_random(seed=seed, urms=URMS, k0=K0)
                sp = os.path.join(tmp, f"c2_series_seed{seed}.jsonl")
                per_seed.append(late_rows(series.run_with_statistics(L, steps, every, sp,
                                                                     theta_slice=(2, plane))).mean(axis=0))
        per_seed = np.array(per_seed)
    with lbm.Lattice(params(0)) as L:
        L.init_random(seed=SEED, urms=URMS, k0=K0)
        L.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.step(steps)
        L.sync()
        wall_plain = time.perf_counter() - t0
        cfg = L.config()
    last = recs[-1]
    a = late
    names = ("theta_mean", "theta_p05", "theta_p50", "theta_p95", "theta_p99", "theta_max",
             "slice_theta_mean", "slice_theta_max", "F4_r1", "Re_lambda", "E_k")
    seeds = (SEED,) + tuple(spread_seeds)
    return {"n": n, "steps": steps, "every": every, "C": 0.13, "nu0": nu0, "theta_molecular_3nu0": 3 * nu0,
            "records": len(recs), "jsonl_lines": lines, "fused_records": len(fused),
            "wall_s_with_statistics_cadence": wall_cadence, "wall_s_steps_only": wall_plain,
            "MLUPS_with_cadence": n ** 3 * steps / wall_cadence / 1e6,
            "MLUPS_steps_only": n ** 3 * steps / wall_plain / 1e6,
            "statistics_overhead": wall_cadence / wall_plain - 1.0,
            "first_statistics_call_s": first_call,
            "statistics_overhead_with_first_call": (wall_cadence + first_call) / wall_plain - 1.0,
            "late_time_mean": {k: float(v) for k, v in zip(names, a.mean(axis=0))},
            "late_time_max_theta": float(a[:, 5].max()),
            "seed_spread": {"seeds": list(seeds),
                            "late_time_mean_by_seed": {k: [float(v) for v in per_seed[:, j]]
                                                       for j, k in enumerate(names)},
                            "relative_std": {k: float(per_seed[:, j].std(ddof=1) / abs(per_seed[:, j].mean()))
                                             for j, k in enumerate(names) if len(seeds) > 1}},
            "paper_context_sec_4_1": {"theta_mean": 1.34e-3, "theta_p05_above": 1.0e-3,
                                      "theta_p95_below": 1.82e-3, "theta_max_up_to": 3.68e-3},
            "final": {"E_k": last["E_k"], "Re_lambda": last["Re_lambda"], "eta": last["eta"], "L": last["L"],
                      "F4_r1": last["F4"][0], "E": [float(f"{v:.4e}") for v in last["E"]]},
            "kernel": cfg}


def les_stationary(lbm, device, stream, n=100, t0=1000, t_end=600, window=(200, 600), every=10, plane=50):
    """The paper's 100^3 LES run to its statistically stationary state (Sec.
    3.1, Sec. 4.1): Re = 2e4 (nu0 = U0 n / Re), C = 0.13, the paper's forcing
    (U0 = 0.043, Cf = 0.2), from the Taylor-Green field of amplitude U0, t0 =
    1000 steps, t_end t0 steps; every `every` t0 the domain statistics and a
    theta slice at z = `plane`.  Reported: theta = tau_e - 1/2 over t / t0 in
    `window` (the paper's interval) -- domain mean, 5th / 95th percentiles,
    maximum, the slice's mean and maximum, each also over 3 nu0 -- beside the
    values the paper prints for this run (context: the paper's numbers, not
    a parity bar); the flow's window means (E_k, u_rms, K_t, the injection
    <F.u> against the resolved and subgrid dissipation, Re_lambda, eta, L)
    and the series over time."""
    import torch
    nu0 = U0 * n / RE
    p = lbm.make_params(n, nu0=nu0, cs=0.13, f0=CF * U0 * U0 / n, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                        device=device, stream=stream.cuda_stream)
    recs = []
    with lbm.Lattice(p) as L:
        L.init(lbm.LBM_INIT_TGV3D, amplitude=U0)
        cfg = L.config()
        torch.cuda.synchronize()
        t_start = time.perf_counter()
        for k in range(every, t_end + 1, every):
            L.step(every * t0)
            st = L.stats(what=lbm.LBM_STATS_SPECTRUM)
            sl = L.theta_slice(2, plane)
            recs.append({"t_over_t0": k, "theta_mean": st["theta_mean"], "theta_p05": st["theta_p05"],
                         "theta_p50": st["theta_p50"], "theta_p95": st["theta_p95"],
                         "theta_max": st["theta_max"], "slice_mean": float(sl.mean()),
                         "slice_p95": float(np.quantile(sl, 0.95)), "slice_max": float(sl.max()),
                         "E_k": st["E_k"], "u_rms": st["u_rms"], "Kt_mean": st["Kt_mean"],
                         "inj": st["inj"], "eps0": st["eps0"], "eps_sgs": st["eps_sgs"],
                         "Re_lambda": st["Re_lambda"], "eta": st["eta"], "L": st["L"]})
        wall = time.perf_counter() - t_start
    win = [r for r in recs if window[0] <= r["t_over_t0"] <= window[1]]
    keys = ("theta_mean", "theta_p05", "theta_p50", "theta_p95", "theta_max", "slice_mean", "slice_p95",
            "slice_max")
    flow = {k: float(np.mean([r[k] for r in win]))
            for k in ("E_k", "u_rms", "Kt_mean", "inj", "eps0", "eps_sgs", "Re_lambda", "eta", "L")}
    flow["injection_over_dissipation"] = flow["inj"] / (flow["eps0"] + flow["eps_sgs"])
    mean = {k: float(np.mean([r[k] for r in win])) for k in keys}
    th0 = 3 * nu0
    return {"n": n, "steps": t_end * t0, "t0_steps": t0, "window_t_over_t0": list(window), "C": 0.13,
            "nu0": nu0, "theta_molecular_3nu0": th0, "wall_s": wall,
            "MLUPS": n ** 3 * t_end * t0 / wall / 1e6, "kernel": cfg,
            "window_mean": mean, "window_mean_over_3nu0": {k: v / th0 for k, v in mean.items()},
            "window_mean_flow": flow,
            "window_min_theta_p05": float(min(r["theta_p05"] for r in win)),
            "window_max_theta_p95": float(max(r["theta_p95"] for r in win)),
            "window_max_theta": float(max(r["theta_max"] for r in win)),
            "paper_sec_4_1": {"theta_mean": 1.34e-3, "theta_mean_over_3nu0": 2.08, "theta_p05_above": 1.0e-3,
                              "theta_p95_below": 1.82e-3, "slice_peaks_up_to": 3.7e-3},
            "series": [{k: (float(f"{v:.6g}") if isinstance(v, float) else v) for k, v in r.items()} for r in recs]}


def strain_mode_cost(lbm, device, stream, m, cfg_les, n, cfg_fp16, les_steps=2000, steps=40):
    """The self-consistent strain evaluation (lbm_params.strain_mode = 1: the
    local s_nu(|S|) in the strain formula, a closed form plus two Newton steps
    per cell) against the explicit one (0), same kernel configuration: the
    m^3 LES in FP32 (L2-resident, where per-cell arithmetic shows) and the
    n^3 lattice with C = 0.13 in FP16 storage (HBM-bound)."""
    out = {}
    for tag, size, prec, cfg, k, w in ((f"{m}^3_les_fp32", m, 0, cfg_les, les_steps, 20),
                                       (f"{n}^3_les_fp16_shifted", n, 1, cfg_fp16, steps, 3)):
        ms = {}
        for mode in (0, 1):
            lat, t, _, st = run_case(lbm, size, prec, 0.13, U0 * size / RE, k, w, device, stream, False,
                                     config=config_of(cfg), layout=cfg["layout"], strain_mode=mode)
            lat.close()
            ms[mode] = t
            assert math.isfinite(st["E_k"])
        out[tag] = {"MLUPS_strain_mode_0": size ** 3 * k / (ms[0] * 1e-3) / 1e6,
                    "MLUPS_strain_mode_1": size ** 3 * k / (ms[1] * 1e-3) / 1e6,
                    "time_ratio_1_over_0": ms[1] / ms[0], "steps": k, "kernel": cfg}
    return out


def stats_cost(lbm, device, stream, n, precision, C, config="", layout=0, reps=3):
    """Cost of each statistics call on the n^3 lattice from the seeded random
    field (the paper's forcing, nu0 from Re = 2e4, Smagorinsky constant C):
    milliseconds of host wall time around each synchronous call, after one
    step that makes the cached velocity stale, minus that step; the first
    call with the spectrum (the FFT's one-time setup) timed on its own."""
    import torch
    nu0 = U0 * n / RE
    lat, _, cfg, _ = run_case(lbm, n, precision, C, nu0, 1, 1, device, stream, False, config=config,
                              layout=layout)
    W = {"plain": 0, "spectrum": lbm.LBM_STATS_SPECTRUM, "structure": lbm.LBM_STATS_STRUCTURE,
         "spectrum_and_structure": lbm.LBM_STATS_SPECTRUM | lbm.LBM_STATS_STRUCTURE}

    def wall(f, k=1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            f()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / k * 1e3

    out = {"n": n, "precision": precision, "C": C, "kernel": cfg,
           "first_spectrum_call_ms": wall(lambda: lbm.lbm_stats(lat.h, 0, W["spectrum"]))}
    step_ms = wall(lambda: (lbm.lbm_step(lat.h, 1), lat.sync()), reps)
    out["step_ms"] = step_ms
    for name, what in W.items():
        out[f"{name}_ms"] = wall(lambda: (lbm.lbm_step(lat.h, 1), lbm.lbm_stats(lat.h, 0, what)), reps) - step_ms
    out["theta_slice_ms"] = wall(lambda: lbm.lbm_get_theta_slice(lat.h, 0, 2, n // 2, lat.shapes[0]), reps)
    lat.close()
    return out


def l2_copy_rate(device, stream, mbytes=76, reps=50, rounds=4):
    """GB/s (read + write bytes) of an in-place FP32 multiply over an
    L2-resident buffer of `mbytes` MB, graph-replayed, CUDA events on the
    stream: the denominator of the L2-resident 100^3 line."""
    import torch
    x = torch.ones(mbytes * 1000 * 1000 // 4, dtype=torch.float32, device=torch.device("cuda", device))
    with torch.cuda.stream(stream):
        for _ in range(5):
            x.mul_(1.0)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(reps):
                x.mul_(1.0)
        g.replay()
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(rounds):
            g.replay()
        b.record(stream)
        b.synchronize()
    ms = a.elapsed_time(b) / (reps * rounds)
    nbytes = 2 * x.numel() * 4
    del g, x
    return nbytes / (ms * 1e-3) / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=800)
    ap.add_argument("--les-n", type=int, default=100)
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--row-align", type=int, default=0, help="x-line alignment in bytes (lbm_params.row_align)")
    ap.add_argument("--cs", type=float, default=0.0,
                    help="Smagorinsky constant of an --only-step run (the DNS shape uses 0)")
    ap.add_argument("--only-step", action="store_true",
                    help="time the step kernel only (no e2e, extras or CPU baseline): profiling runs")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--c-sweep", action="store_true",
                    help="Smagorinsky-constant sweep at 128^3, Re = 5000 (Sec. 3.3): spectra and ESS exponents")
    ap.add_argument("--sweep", action="store_true",
                    help="roofline sweep N in {128, 256, 512, 1024}, FP32 and FP16, with spectral error at 128^3")
    ap.add_argument("--precision-study", action="store_true",
                    help="FP16/BF16 storage against FP32 at 800^3 over 2000 steps (spectral error, stability)")
    ap.add_argument("--les-stationary", action="store_true",
                    help="the paper's 100^3 LES from the Taylor-Green field to t/t0 = 600 (t0 = 1000 steps)")
    ap.add_argument("--stats-cost", action="store_true",
                    help="cost of each statistics call at --n (--precision, --cs, --config, --layout)")
    ap.add_argument("--shape", default="",
                    help="nx,ny,nz of a non-cubic box for --only-step profiling runs")
    ap.add_argument("--layout", type=int, default=0, choices=[0, 1, 2],
                    help="population array of an --only-step run: 1 population-major, 2 row-interleaved, 0 autotuned")
    ap.add_argument("--config", default="",
                    help="kind,tile_rows,stages,threads[,tma_slots]: a fixed kernel configuration (no autotuning)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_env()
    dist = world > 1
    if dist:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_23116_gb300 as lbm
    lbm.load()

    if args.c_sweep:
        stream = torch.cuda.Stream(device=dev)
        res = c_sweep(lbm, local, stream)
        if rank == 0:
            print(json.dumps(res), flush=True)
        return 0
    if args.sweep:
        stream = torch.cuda.Stream(device=dev)
        res = sweep(lbm, local, stream)
        if rank == 0:
            print(json.dumps({"sweep": res}), flush=True)
        return 0
    if args.les_stationary:
        stream = torch.cuda.Stream(device=dev)
        res = les_stationary(lbm, local, stream)
        if rank == 0:
            print(json.dumps({"les_stationary": res}), flush=True)
        return 0
    if args.stats_cost:
        stream = torch.cuda.Stream(device=dev)
        res = stats_cost(lbm, local, stream, args.n, args.precision, args.cs, config=args.config,
                         layout=args.layout)
        if rank == 0:
            print(json.dumps({"stats_cost": res}), flush=True)
        return 0
    if args.precision_study:
        stream = torch.cuda.Stream(device=dev)
        res = precision_study(lbm, local, stream, n=args.n)
        if rank == 0:
            print(json.dumps({"precision_study": res}), flush=True)
        return 0

    n = args.n
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
    if shape and not args.only_step:
        raise SystemExit("--shape is for --only-step profiling runs")
    nu0 = U0 * (shape[0] if shape else n) / RE
    stream = torch.cuda.Stream(device=dev)
    cells = shape[0] * shape[1] * shape[2] if shape else n ** 3
    # host copy of the initial field for the end-to-end run: the FP32 velocity
    # the library generates (the kernels build the equilibrium from FP32)
    u_host = None
    if not args.only_step:
        u_host = torch.empty((3, n, n, n), dtype=torch.float32, pin_memory=True)
    clocks = ClockSampler(local)
    lat, ms, cfg, st = run_case(lbm, n, args.precision, args.cs if args.only_step else 0.0, nu0,
                                args.steps, args.warmup, local,
                                stream, dist, clocks, config=args.config, shape=shape,
                                row_align=args.row_align, layout=args.layout, u_out=u_host)
    assert math.isfinite(st["E_k"]) and st["cells"] == cells, st
    if args.only_step:
        if rank == 0:
            print(json.dumps({"only_step": True, "n": n, "shape": shape, "cells": cells,
                              "precision": args.precision, "steps": args.steps,
                              "ms_per_step": ms / args.steps,
                              "MLUPS": cells * args.steps / (ms * 1e-3) / 1e6,
                              "GB_s": cells * BYTES_PER_UPDATE[args.precision] * args.steps / (ms * 1e-3) / 1e9,
                              "kernel": cfg}), flush=True)
        lat.close()
        return 0
    # e2e: the public API with host buffers: H2D of the initial field from pinned
    # memory, the K steps, and the D2H statistics read, all inside the timed
    # region.  The page-locked buffer is read once before (untimed, like the
    # warm-up steps): the GPU's first read of freshly page-locked memory runs
    # at ~120-150 GB/s, later reads at ~210 GB/s.
    lbm.lbm_init_field(lat.h, 0, lbm.LBM_INIT_VELOCITY, 0.0, u_host)
    lat.sync()
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    lbm.lbm_init_field(lat.h, 0, lbm.LBM_INIT_VELOCITY, 0.0, u_host)  # FP32, read in place (page-locked)
    lat.step(args.steps)
    st2 = lat.stats()
    t_e2e = time.perf_counter() - t0
    if dist:
        torch.distributed.barrier()
    assert math.isfinite(st2["E_k"])
    lat.close()
    del u_host

    value, e2e_value, ms_max, e2e_ms = aggregate_ranks(ms, t_e2e * 1e3, cells, args.steps, world, dev)

    hbm_peak, peak_kind = measured_peaks()
    achieved = cells * BYTES_PER_UPDATE[0] * args.steps / (ms * 1e-3) / 1e9  # this rank's kernel
    digest = kernel_digest()
    tpu = traffic_per_update(digest)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_gbs": NOMINAL_HBM_GBS,
                "traffic": None if tpu is None else tpu * cells,
                "algorithmic_bytes_per_launch": cells * BYTES_PER_UPDATE[0]}

    extra = {}
    # the extra workloads and studies run in single-GPU runs only (a replicas
    # run measures the headline workload on every rank)
    if not args.no_extra and not dist:
        def guarded(name, fn):
            # one failing study is recorded in the line, not fatal to it
            try:
                extra[name] = fn()
            except Exception as exc:  # noqa: BLE001
                extra[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()

        for prec, name in ((1, "fp16_shifted"), (2, "bf16_shifted")):
            lat2, ms2, cfg2, st3 = run_case(lbm, n, prec, 0.0, nu0, args.steps, args.warmup, local,
                                            stream, dist)
            lat2.close()
            extra[f"{n}^3_{name}"] = {
                "MLUPS": cells * args.steps / (ms2 * 1e-3) / 1e6, "ms_per_step": ms2 / args.steps,
                "GB_s": cells * BYTES_PER_UPDATE[prec] * args.steps / (ms2 * 1e-3) / 1e9,
                "frac_hbm": cells * BYTES_PER_UPDATE[prec] * args.steps / (ms2 * 1e-3) / 1e9 / hbm_peak,
                "frac_of_nominal": cells * BYTES_PER_UPDATE[prec] * args.steps / (ms2 * 1e-3) / 1e9
                / NOMINAL_HBM_GBS,
                "speedup_vs_fp32": ms / ms2, "kernel": cfg2}
            if prec == 1:
                extra[f"{n}^3_{name}"]["dram_bytes_per_update"] = traffic_per_update(digest, "fp16")
        torch.cuda.empty_cache()
        m = args.les_n
        nu_les = U0 * m / RE
        les_steps = 2000
        lat3, ms3, cfg3, st4 = run_case(lbm, m, 0, 0.13, nu_les, les_steps, 20, local, stream, dist)
        lat3.close()
        gbs_les = m ** 3 * BYTES_PER_UPDATE[0] * les_steps / (ms3 * 1e-3) / 1e9
        l2_mb = (19 * m ** 3 * 4) // 1000000
        l2_gbs = l2_copy_rate(local, stream, mbytes=l2_mb)
        extra[f"{m}^3_les_fp32"] = {
            "MLUPS": m ** 3 * les_steps / (ms3 * 1e-3) / 1e6, "ms_per_step": ms3 / les_steps,
            "GB_s": gbs_les, "steps": les_steps, "C": 0.13, "nu0": nu_les,
            "roofline": {"bound": "l2", "achieved": gbs_les, "peak": l2_gbs, "unit": "GB/s",
                         "frac": gbs_les / l2_gbs,
                         "peak_kind": "measured in this run: in-place FP32 multiply over an "
                                      f"L2-resident {l2_mb} MB buffer (read + write bytes)"},
            "frac_of_hbm_copy_peak": gbs_les / hbm_peak,
            "note": f"{l2_mb} MB lattice: L2-resident (129 MB L2); the roofline fraction is of the "
                    "L2-resident copy rate measured beside it",
            "kernel": cfg3, "theta_mean": st4["theta_mean"]}
        guarded("NEXT4_strain_mode_cost", lambda: strain_mode_cost(lbm, local, stream, m, cfg3, n,
                                                                    extra[f"{n}^3_fp16_shifted"]["kernel"]))
        guarded("C2_100^3_les_20000_steps_statistics_every_500", lambda: les_c2_run(lbm, local, stream))
        guarded("C2_stationary_100^3_les_tgv_600k_steps", lambda: les_stationary(lbm, local, stream))
        guarded("C4_batch48_les_fp32_5000_steps", lambda: batch_case(lbm, local, stream, 5000, 10))
        guarded("C3_800^3_storage_precision_2000_steps", lambda: precision_study(lbm, local, stream, n=n))
        guarded("NEXT3_c_sweep_128^3_Re5000", lambda: c_sweep(lbm, local, stream))

    cpu = None
    if rank == 0:
        mlups, csteps, cdt = oracle_mlups(64, args.cpu_seconds, U0 * 64 / RE, 0.0)
        mlups1, csteps1, cdt1 = oracle_mlups(64, args.cpu_seconds, U0 * 64 / RE, 0.0, threads=1)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": host_cores(), "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"64^3 sample of the same setup (Re = 2e4 at N = 64), {csteps} steps, {cdt:.1f} s, "
                         f"all {host_cores()} host threads (OpenMP)",
               "single_thread": {"value": mlups1, "unit": "MLUPS", "cores": 1,
                                 "sample": f"64^3, {csteps1} steps, {cdt1:.1f} s"}}

    if rank == 0:
        h2d = 3 * cells * 4
        line = {
            "metric": "MLUPS (stream+collide, D3Q19 MRT-Smagorinsky-Guo)",
            "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"forced-HIT DNS shape {n}^3 FP32 storage, C = 0, Re = 2e4",
                       "cells_per_gpu": cells, "nu0": nu0, "F0": CF * U0 * U0 / n,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (38.9 GB lattice), no flush",
                       "kernel": cfg},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": 1024.0 / args.steps,
                    "note": "initial velocity from page-locked host FP32 memory read in place "
                            "(lbm_init_velocity_f32) + lbm_step(K) + lbm_stats"},
            "gpu_launches": args.steps,
            "clocks": clocks.summary(),
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
