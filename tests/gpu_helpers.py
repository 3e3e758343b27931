"""Shared helpers of the GPU parity tests: run the same seeded case through the
CUDA library (C ABI via the binding) and through the FP64 oracle."""
from __future__ import annotations

import numpy as np

import oracle

KINDS = [1, 2]  # direct-load kernel, TMA bulk-copy kernel
LAYOUTS = [1, 2]  # population-major, row-interleaved population array


def oracle_force_mode(lbm, mode):
    return {lbm.LBM_FORCE_NONE: oracle.FORCE_NONE, lbm.LBM_FORCE_PAPER_SIN: oracle.FORCE_PAPER_SIN,
            lbm.LBM_FORCE_CONST: oracle.FORCE_CONST,
            lbm.LBM_FORCE_KOLMOGOROV: oracle.FORCE_KOLMOGOROV}[mode]


def make_pair(lbm, shape, *, nu0, C, force_mode=0, F0=0.0, body=(0.0, 0.0, 0.0), kind=0,
              precision=0, stats_every=0, hist_bins=0, hist_max=0.0, tile_rows=0, layout=0):
    nz, ny, nx = shape
    p = lbm.make_params(nx, ny, nz, precision=precision, nu0=nu0, cs=C, f0=F0, body_force=body,
                        force_mode=force_mode, kernel=kind, stats_every=stats_every,
                        hist_bins=hist_bins, hist_max=hist_max, tile_rows=tile_rows, layout=layout)
    gpu = lbm.Lattice(p)
    ref = oracle.OracleLBM(nx, ny, nz, nu0, C, oracle_force_mode(lbm, force_mode), F0=F0, body=body)
    return gpu, ref


def random_populations(shape, seed, u_scale=0.03, neq=1e-3):
    """Equilibrium of a random velocity field plus a random non-equilibrium part
    (weight-shifted populations), built by the oracle."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    u = rng.normal(scale=u_scale, size=(3, nz, ny, nx))
    L = oracle.OracleLBM(nx, ny, nz, 0.02, 0.0)
    L.init_equilibrium(u)
    return L.populations() + rng.normal(scale=neq, size=(19, nz, ny, nx))


def full_f_rel_error(gpu_shifted, ref_shifted):
    _, w = oracle.lattice()
    wf = w[:, None, None, None]
    return float(np.max(np.abs(gpu_shifted - ref_shifted) / (ref_shifted + wf)))


def ulp(x: float, mant_bits: int) -> float:
    return 2.0 ** (np.floor(np.log2(x)) - mant_bits)


def fp32_mass_tolerance(ncell: int, steps: int, fmax: float) -> float:
    """Round-off bound on the drift of sum f' with FP32 arithmetic and storage.

    Random part: every step rounds 19 ncell stored values by up to ulp/2 with
    random sign, 6 sigma of that random walk.  Systematic part: round to nearest
    inside the collision's arithmetic leaves a small bias in sum f*, measured at
    about 1 % of a half ulp per cell and step on the 800^3 DNS-shape field; the
    bound allows 5 %.  (A mass error of the method itself would be of order
    |f'| per cell and step, 10^7 times larger.)  ulp of the largest |f'|."""
    half_ulp = 0.5 * ulp(fmax, 23)
    return 6.0 * np.sqrt(19.0 * ncell * (steps + 1)) * half_ulp + 0.05 * half_ulp * ncell * (steps + 1)
