"""Benchmark of the GB300 MRT-Smagorinsky LBM step (one JSON line on stdout).

Workload (headline): the forced-HIT DNS shape, an 800^3 periodic lattice
(5.12e8 cells) with FP32 storage, seeded random solenoidal initial field
(k^4 exp(-2 (k/4)^2), u_rms = 0.05), the paper's sinusoidal forcing with
U0 = 0.043, Cf = 0.2 (F0 = 4.6225e-7), C = 0 and nu0 from Re = 2e4
(nu0 = 0.00172).  A step is one launch of the fused stream + collide kernel
over all cells; MLUPS = cells x steps / time.  Extra entries: the same lattice
with FP16 and BF16 weight-shifted storage, and the 100^3 LES (C = 0.13,
nu0 = 2.15e-4, FP32).

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


def oracle_mlups(n: int, seconds: float, nu0: float, C: float):
    """The FP64 CPU oracle as it stands, on an n^3 sample, for ~`seconds`."""
    import oracle
    import synthetic
    oracle.build()
    u = synthetic.random_solenoidal(n, seed=1, urms=0.05)
    F0 = oracle.forcing_amplitude(CF, U0, n)
    L = oracle.OracleLBM(n, n, n, nu0, C, oracle.FORCE_PAPER_SIN, F0=F0)
    L.init_equilibrium(u)
    L.step(1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        L.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt / 1e6, steps, dt


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


def make_velocity(n, device, shape=None):
    import synthetic
    nx, ny, nz = shape if shape else (n, n, n)
    k, a = synthetic.spectrum_coefficients(nx, ny, nz, seed=1, k0=4.0, urms=0.05)
    return synthetic.synthesize_torch(k, a, nx, ny, nz, device, zchunk=32)


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


def run_case(lbm, n, precision, C, nu0, steps, warmup, device, stream, u_dev, dist, clocks=None,
             config="", shape=None, row_align=0, layout=0):
    """Create, initialise from the device velocity, time `steps` steps."""
    kind = rows = stages = threads = slots = 0
    if config:
        vals = [int(v) for v in config.split(",")]
        kind, rows, stages, threads = vals[:4]
        slots = vals[4] if len(vals) > 4 else 0
    nx, ny, nz = shape if shape else (n, n, n)
    p = lbm.make_params(nx, ny, nz, precision=precision, nu0=nu0, cs=C, f0=CF * U0 * U0 / nx,
                        force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device, stream=stream.cuda_stream,
                        kernel=kind, tile_rows=rows, stages=stages, threads=threads, row_align=row_align,
                        layout=layout, tma_slots=slots)
    lat = lbm.Lattice(p)
    lat.init(lbm.LBM_INIT_VELOCITY, u=u_dev)
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
    dev = torch.device("cuda", device)

    def params(n):
        return lbm.make_params(n, nu0=U0 * n / RE, cs=0.13, f0=CF * U0 * U0 / n,
                               force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device,
                               stream=stream.cuda_stream)

    def velocity(n, seed):
        import synthetic
        k, a = synthetic.spectrum_coefficients(n, n, n, seed=seed, k0=4.0, urms=0.05)
        return synthetic.synthesize_torch(k, a, n, n, n, dev, zchunk=32)

    cells = sum(n ** 3 for n in sizes)
    lat = lbm.Lattice([params(n) for n in sizes])
    for i, n in enumerate(sizes):
        lat.init(lbm.LBM_INIT_VELOCITY, u=velocity(n, i + 1), inst=i)
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
        one.init(lbm.LBM_INIT_VELOCITY, u=velocity(n, i + 1))
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


def precision_study(lbm, device, stream, n_small=64, steps_small=500, every_small=50, n_big=800,
                    steps_big=600, every_big=60):
    """Spectral error of each storage precision (reading: time-averaged shell
    spectra, per-shell relative error for shells 1..kd, kd = where E drops below
    1e-3 of its peak, <= N/3): against the FP64 oracle on an n_small^3 rerun of
    the setup (C = 0 with nu0 from Re = 2e4, and the LES C = 0.13), and against
    FP32 storage at n_big^3 (C = 0) over the first 600 steps: from the synthetic
    initial field (u_rms = 0.05 per component, peaks near 0.3) the C = 0 run at
    tau - 1/2 = 0.00516 turns unstable at its fastest spot after ~1300 steps in
    FP32 (earlier with the noisier low-precision storage)."""
    import torch
    import oracle
    import synthetic
    from oracle import diagnostics as dg
    out = {}
    dev = torch.device("cuda", device)
    m = n_small
    nu0 = U0 * m / RE
    F0 = CF * U0 * U0 / m
    u = synthetic.random_solenoidal(m, seed=1, urms=0.05)
    kmax = dg.max_shell(m, m, m)
    for C in (0.0, 0.13):
        ref = oracle.OracleLBM(m, m, m, nu0, C, oracle.FORCE_PAPER_SIN, F0=F0)
        ref.init_equilibrium(u)
        E_ref = np.zeros(kmax + 1)
        kt_ref = []
        for _ in range(steps_small // every_small):
            ref.step(every_small)
            fl = ref.fields()
            E_ref += dg.spectrum(fl["u"], kmax)
            kt_ref.append((np.sqrt(3) * fl["theta"].mean(), 3 * fl["theta"].var()))
        E_ref /= steps_small // every_small
        case = {}
        for prec, name in ((0, "fp32"), (1, "fp16_shifted"), (2, "bf16_shifted")):
            p = lbm.make_params(m, precision=prec, nu0=nu0, cs=C, f0=F0, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                                device=device, stream=stream.cuda_stream)
            try:
                with lbm.Lattice(p) as L:
                    L.init(lbm.LBM_INIT_VELOCITY, u=u)
                    E = np.zeros(kmax + 1)
                    kt = []
                    for _ in range(steps_small // every_small):
                        L.step(every_small)
                        E += L.spectrum(kmax)
                        st = L.stats()
                        kt.append((st["Kt_mean"], st["Kt_var"]))
                    E /= steps_small // every_small
            except lbm.LbmError as exc:
                if exc.code != lbm.LBM_ERR_UNSTABLE:
                    raise
                case[name] = {"unstable": True, "non_finite_by_step": (len(kt) + 1) * every_small}
                continue
            r = _spectral_error(E, E_ref, m)
            km, kv = np.mean(kt, axis=0)
            kmr, kvr = np.mean(kt_ref, axis=0)
            r["Kt_mean_rel_error"] = float(abs(km - kmr) / kmr)
            r["Kt_var_rel_error"] = float(abs(kv - kvr) / kvr) if kvr > 0 else None
            case[name] = r
        out[f"{m}^3_C{C}_vs_fp64_oracle_{steps_small}_steps"] = case
    if n_big:
        nb = n_big
        nu0b = U0 * nb / RE
        k, a = synthetic.spectrum_coefficients(nb, nb, nb, seed=1, k0=4.0, urms=0.05)
        ub = synthetic.synthesize_torch(k, a, nb, nb, nb, dev, zchunk=32)
        kmax_b = dg.max_shell(nb, nb, nb)
        spectra = {}
        for prec, name in ((0, "fp32"), (1, "fp16_shifted"), (2, "bf16_shifted")):
            p = lbm.make_params(nb, precision=prec, nu0=nu0b, cs=0.0, f0=CF * U0 * U0 / nb,
                                force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device, stream=stream.cuda_stream)
            done = 0
            try:
                with lbm.Lattice(p) as L:
                    L.init(lbm.LBM_INIT_VELOCITY, u=ub)
                    E = np.zeros(kmax_b + 1)
                    for _ in range(steps_big // every_big):
                        L.step(every_big)
                        E += L.spectrum(kmax_b)
                        L.stats()
                        done += every_big
                    spectra[name] = E / (steps_big // every_big)
            except lbm.LbmError as exc:
                if exc.code != lbm.LBM_ERR_UNSTABLE:
                    raise
                spectra[name] = {"unstable": True, "non_finite_by_step": done + every_big}
        del ub
        torch.cuda.empty_cache()
        res = {}
        for name in ("fp16_shifted", "bf16_shifted"):
            if isinstance(spectra["fp32"], dict):
                res[name] = {"reference": spectra["fp32"], "this": spectra[name] if isinstance(spectra[name], dict) else "finite"}
            elif isinstance(spectra[name], dict):
                res[name] = spectra[name]
            else:
                res[name] = _spectral_error(spectra[name], spectra["fp32"], nb)
        out[f"{nb}^3_C0_vs_fp32_{steps_big}_steps"] = res
    return out


def sweep(lbm, device, stream, sizes=(128, 256, 512, 1024), steps=500, warmup=5, err_steps=200):
    """Roofline sweep: N^3 for each N, FP32 and FP16-shifted storage, the LES
    setting (C = 0.13, nu0 from Re = 2e4 at each N, the paper's forcing); and
    the spectral error of both storages against the FP64 oracle at N = 128
    after err_steps steps."""
    import torch
    import oracle
    from oracle import diagnostics as dg
    hbm_peak, _ = measured_peaks()
    rows = []
    dev = torch.device("cuda", device)
    for n in sizes:
        u = make_velocity(n, dev)
        for prec in (0, 1):
            p = lbm.make_params(n, precision=prec, nu0=U0 * n / RE, cs=0.13, f0=CF * U0 * U0 / n,
                                force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device, stream=stream.cuda_stream)
            with lbm.Lattice(p) as L:
                L.init(lbm.LBM_INIT_VELOCITY, u=u)
                ms = time_steps(lbm, L, stream, steps, warmup, False)
                cfg = L.config()
            gbs = n ** 3 * BYTES_PER_UPDATE[prec] * steps / (ms * 1e-3) / 1e9
            rows.append({"N": n, "storage": ["fp32", "fp16_shifted"][prec], "steps": steps,
                         "MLUPS": n ** 3 * steps / (ms * 1e-3) / 1e6, "GB_s": gbs, "frac_hbm": gbs / hbm_peak,
                         "frac_of_nominal": gbs / NOMINAL_HBM_GBS, "kernel": cfg})
        del u
        torch.cuda.empty_cache()
    n = 128
    u = make_velocity(n, dev).cpu().numpy()
    ref = oracle.OracleLBM(n, n, n, U0 * n / RE, 0.13, oracle.FORCE_PAPER_SIN, F0=CF * U0 * U0 / n)
    ref.init_equilibrium(u)
    ref.step(err_steps)
    kmax = dg.max_shell(n, n, n)
    E_ref = dg.spectrum(ref.fields()["u"], kmax)
    errs = {}
    for prec in (0, 1):
        p = lbm.make_params(n, precision=prec, nu0=U0 * n / RE, cs=0.13, f0=CF * U0 * U0 / n,
                            force_mode=lbm.LBM_FORCE_PAPER_SIN, device=device, stream=stream.cuda_stream)
        with lbm.Lattice(p) as L:
            L.init(lbm.LBM_INIT_VELOCITY, u=u)
            L.step(err_steps)
            E = L.spectrum(kmax)
        errs[["fp32", "fp16_shifted"][prec]] = _spectral_error(E, E_ref, n)
    return {"rows": rows, f"spectral_error_vs_fp64_oracle_128^3_{err_steps}_steps": errs}


def c_sweep(lbm, device, stream, n=128, re=5000.0, cs=(0.0, 0.1, 0.16, 0.25), steps=4000,
            every=250):
    """The Smagorinsky-constant sweep of Sec. 3.3 (Fig. c_variation): n^3, Re = 5000,
    C in {0, 0.1, 0.16, 0.25}, the paper's forcing, from the seeded random field.
    Reports the spectrum time-averaged over the second half of the run, the
    high-k pile-up indicator E(n/3)/E(peak), and the ESS exponents zeta_p/zeta_3
    (slopes of log S_p against log |S_3| over r = 2..16, Sec. 3.4) from the
    structure functions of the last state."""
    import torch
    from oracle import diagnostics as dg  # shell count only
    dev = torch.device("cuda", device)
    u = make_velocity(n, dev)
    kmax = dg.max_shell(n, n, n)
    out = {}
    for C in cs:
        nu0 = U0 * n / re
        p = lbm.make_params(n, nu0=nu0, cs=C, f0=CF * U0 * U0 / n, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                            device=device, stream=stream.cuda_stream)
        row = {"C": C, "nu0": nu0}
        try:
            with lbm.Lattice(p) as L:
                L.init(lbm.LBM_INIT_VELOCITY, u=u)
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
            row["E"] = [float(v) for v in E[:n // 2 + 1]]
            row["pileup_E(n/3)/E(peak)"] = float(E[n // 3] / E[peak])
            r = np.array(st["r"], dtype=float)
            Sp = st["Sp"]
            sel = (r >= 2) & (r <= 16)
            s3 = np.log(np.abs(Sp[sel, 2]))
            row["ESS_zeta_p_over_zeta_3"] = {
                p_: float(np.polyfit(s3, np.log(np.abs(Sp[sel, p_ - 1])), 1)[0]) for p_ in (2, 4, 6)}
            row["F4_r1"] = float(st["F4"][0])
            row["theta_mean"] = st["theta_mean"]
        except lbm.LbmError as exc:
            if exc.code != lbm.LBM_ERR_UNSTABLE:
                raise
            row["unstable"] = True
        out[f"C={C}"] = row
    return {"n": n, "Re": re, "steps": steps, "c_sweep": out}


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
                    help="spectral error of FP32/FP16/BF16 storage vs the FP64 oracle (64^3) and vs FP32 (800^3)")
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
    if args.precision_study:
        stream = torch.cuda.Stream(device=dev)
        res = precision_study(lbm, local, stream, n_big=args.n)
        if rank == 0:
            print(json.dumps({"precision_study": res}), flush=True)
        return 0

    n = args.n
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
    if shape and not args.only_step:
        raise SystemExit("--shape is for --only-step profiling runs")
    nu0 = U0 * (shape[0] if shape else n) / RE
    stream = torch.cuda.Stream(device=dev)
    u_dev = make_velocity(n, dev, shape)
    torch.cuda.synchronize()
    cells = shape[0] * shape[1] * shape[2] if shape else n ** 3
    clocks = ClockSampler(local)
    lat, ms, cfg, st = run_case(lbm, n, args.precision, args.cs if args.only_step else 0.0, nu0,
                                args.steps, args.warmup, local,
                                stream, u_dev, dist, clocks, config=args.config, shape=shape,
                                row_align=args.row_align, layout=args.layout)
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
    # memory, the K steps, and the D2H statistics read, all inside the timed region
    u_host = u_dev.float().cpu().pin_memory()  # FP32: the kernels round the velocity to FP32
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
    if not args.no_extra:
        for prec, name in ((1, "fp16_shifted"), (2, "bf16_shifted")):
            lat2, ms2, cfg2, st3 = run_case(lbm, n, prec, 0.0, nu0, args.steps, args.warmup, local,
                                            stream, u_dev, dist)
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
        del u_dev
        torch.cuda.empty_cache()
        m = args.les_n
        u_les = make_velocity(m, dev)
        nu_les = U0 * m / RE
        lat3, ms3, cfg3, st4 = run_case(lbm, m, 0, 0.13, nu_les, 400, 20, local, stream, u_les, dist)
        lat3.close()
        gbs_les = m ** 3 * BYTES_PER_UPDATE[0] * 400 / (ms3 * 1e-3) / 1e9
        extra[f"{m}^3_les_fp32"] = {
            "MLUPS": m ** 3 * 400 / (ms3 * 1e-3) / 1e6, "ms_per_step": ms3 / 400,
            "GB_s": gbs_les, "frac_hbm": gbs_les / hbm_peak, "frac_of_nominal": gbs_les / NOMINAL_HBM_GBS,
            "steps": 400, "C": 0.13, "nu0": nu_les,
            "note": "76 MB lattice: L2-resident (129 MB L2); the fractions are of HBM bandwidths, "
                    "which an L2-resident lattice can exceed",
            "kernel": cfg3, "theta_mean": st4["theta_mean"]}

        extra["batch48_les_fp32"] = batch_case(lbm, local, stream, 200, 10)

    cpu = None
    if rank == 0:
        mlups, csteps, cdt = oracle_mlups(64, args.cpu_seconds, U0 * 64 / RE, 0.0)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": host_cores(), "kind": "oracle",
               "sample": f"64^3 sample of the same setup (Re = 2e4 at N = 64), {csteps} steps, {cdt:.1f} s"}

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
