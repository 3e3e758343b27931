"""Diagnostics of the oracle in numpy FP64 (TEST INFRASTRUCTURE ONLY).

Written from the paper's definitions, one function per quantity:

* ``spectrum``            E(k) of Eq. (integral_length_scale): half the sum of
                          |u_hat|^2 over the integer shell k - 1/2 <= |k| < k + 1/2,
                          u_hat = N^-3 sum_x u e^{-2 pi i k.x/N} (the paper prints
                          |u_hat|; the energy reading |u_hat|^2 makes sum_k E = E_k).
* ``structure_functions`` S_p(r) of Eqs. (velocity_increment)-(structure_function)
                          for axis-aligned separations, longitudinal component,
                          the three axes pooled; F4 of Eq. (flatness).
* ``domain_stats``        E_k = <u.u>/2, injection <F.u>, eps0 = 2 nu0 <S_ij S_ij>
                          (Eq. energy_balance), eps_sgs = 2 <nu_t S_ij S_ij>, and the
                          statistics of theta = tau_e - 1/2 and K_t (Eq. Kt_definition).
* ``derived_scales``      L, eta, lambda, u_rms, eps (Eqs. integral_length_scale -
                          dissipation_rate) and Re_lambda (Sec. 3.1), with the
                          lattice wavenumber k_s = 2 pi s / N.
* ``isotropy``            directional energy fractions E_i/E, the Reynolds-stress
                          anisotropy b_ij = <u_i u_j>/<u_k u_k> - delta_ij/3, its
                          invariants II_b = -b_ij b_ji/2, III_b = b_ij b_jk b_ki/3 and
                          the Lumley coordinates xi = (III_b/2)^(1/3),
                          eta = (-II_b/3)^(1/2) (Sec. 3.2, Fig. isotropy_validation).
* ``energy_balance``      residual of Eq. (energy_balance), eps = -dE_k/dt + <F.u>,
                          from a time series (central differences).

numpy's FFT is used as a library primitive; a brute-force DFT pins it in
tests/test_oracle_diagnostics.py.
"""
from __future__ import annotations

import math

import numpy as np


def wavenumbers(n: int) -> np.ndarray:
    """Signed integer wavenumbers of an n-point DFT: 0, 1, ..., -1."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def shell_index(K2: np.ndarray) -> np.ndarray:
    """Shell s with s - 1/2 <= sqrt(K2) < s + 1/2 for integer K2 >= 0, exactly:
    s = r or r + 1 with r = isqrt(K2); K2 lies in shell s iff
    s^2 - s + 1 <= K2 <= s^2 + s (K2 integer, so no ties)."""
    K2 = np.asarray(K2, dtype=np.int64)
    r = np.floor(np.sqrt(K2.astype(np.float64))).astype(np.int64)
    r = np.where(r * r > K2, r - 1, r)
    r = np.where((r + 1) * (r + 1) <= K2, r + 1, r)
    return np.where(K2 > r * r + r, r + 1, r)


def max_shell(nx: int, ny: int, nz: int) -> int:
    kx, ky, kz = nx // 2, ny // 2, nz // 2
    return int(shell_index(np.array([kx * kx + ky * ky + kz * kz]))[0])


def spectrum(u: np.ndarray, kmax: int | None = None) -> np.ndarray:
    """E(s), s = 0..kmax, of a velocity field u of shape (3, nz, ny, nx)."""
    _, nz, ny, nx = u.shape
    ncell = nx * ny * nz
    kz = wavenumbers(nz)[:, None, None]
    ky = wavenumbers(ny)[None, :, None]
    kx = wavenumbers(nx)[None, None, :]
    K2 = kx * kx + ky * ky + kz * kz
    s = shell_index(K2)
    if kmax is None:
        kmax = max_shell(nx, ny, nz)
    energy = np.zeros(s.shape)
    for d in range(3):
        uh = np.fft.fftn(u[d]) / ncell
        energy += 0.5 * (uh.real ** 2 + uh.imag ** 2)
    E = np.zeros(kmax + 1)
    mask = s <= kmax
    np.add.at(E, s[mask], energy[mask])
    return E


def separations(n: int) -> list[int]:
    """Separations r = 1, 2, 3, 4, 6, 8, 12, 16, ... (2^k and 3 * 2^k) up to n/2."""
    out = set()
    k = 1
    while k <= n // 2:
        out.add(k)
        if 3 * k // 2 <= n // 2 and k >= 2:
            out.add(3 * k // 2)
        k *= 2
    return sorted(out)


def structure_functions(u: np.ndarray, rs=None, pmax: int = 6) -> dict:
    """S_p(r) for p = 1..pmax pooled over the three axes, and F4(r).

    For axis a the increment is u_a(x + r e_a) - u_a(x) (periodic)."""
    _, nz, ny, nx = u.shape
    if rs is None:
        rs = separations(min(nx, ny, nz))
    S = np.zeros((len(rs), pmax + 1))
    for i, r in enumerate(rs):
        acc = np.zeros(pmax + 1)
        count = 0
        for a, axis in ((0, 2), (1, 1), (2, 0)):
            d = np.roll(u[a], -r, axis=axis) - u[a]
            for p in range(1, pmax + 1):
                acc[p] += np.sum(d ** p)
            count += d.size
        S[i] = acc / count
    F4 = S[:, 4] / (S[:, 2] ** 2)
    return {"r": list(rs), "S": S, "F4": F4}


def domain_stats(fields: dict, F: np.ndarray, nu0: float, C: float,
                 hist_bins: int = 4096, hist_max: float = 0.05) -> dict:
    """Domain statistics of a state given its per-cell fields (oracle.fields())."""
    drho, u, sn, th = fields["drho"], fields["u"], fields["snorm"], fields["theta"]
    rho = 1.0 + drho
    n = drho.size
    uu = np.sum(u * u, axis=0)
    out = {
        "cells": n,
        "mass": float(np.sum(drho)),
        "momentum": [float(np.sum(rho * u[d])) for d in range(3)],
        "E_k": 0.5 * float(np.mean(uu)),
        "inj": float(np.mean(np.sum(F * u, axis=0))),
        # S_ij S_ij = |S|^2 / 2 with |S| of Eq. (strain_norm).
        "eps0": 2.0 * nu0 * float(np.mean(0.5 * sn * sn)),
        "eps_sgs": 2.0 * float(np.mean(C * sn * 0.5 * sn * sn)),
        "uu": [float(np.mean(u[0] * u[0])), float(np.mean(u[1] * u[1])),
               float(np.mean(u[2] * u[2])), float(np.mean(u[0] * u[1])),
               float(np.mean(u[0] * u[2])), float(np.mean(u[1] * u[2]))],
        "theta_mean": float(np.mean(th)),
        "theta_var": float(np.var(th)),
        "theta_min": float(np.min(th)),
        "theta_max": float(np.max(th)),
        # nearest-rank percentile: the ceil(p n)-th smallest value (inverted CDF)
        "theta_p": {p: float(np.percentile(th, p, method="inverted_cdf")) for p in (5, 50, 95, 99)},
    }
    # K_t = lambda_e / l with lambda_e = (tau_e - 1/2) sqrt(3) dx, l = dx (Eq. Kt_definition).
    kt = math.sqrt(3.0) * th
    out["Kt_mean"] = float(np.mean(kt))
    out["Kt_var"] = float(np.var(kt))
    edges = np.linspace(0.0, hist_max, hist_bins + 1)
    idx = np.floor(th / hist_max * hist_bins).astype(np.int64)
    idx = np.clip(idx, 0, hist_bins - 1)
    out["hist"] = np.bincount(idx.ravel(), minlength=hist_bins)
    out["hist_edges"] = edges
    return out


def derived_scales(E: np.ndarray, n: int, nu0: float, E_k: float) -> dict:
    """L, eps, eta, lambda, u_rms and Re_lambda from the shell spectrum E(s).

    The integrals of Eqs. (integral_length_scale) and (dissipation_rate) become
    sums over shells s >= 1 with k_s = 2 pi s / n (lattice units)."""
    s = np.arange(len(E))
    k = 2.0 * math.pi * s[1:] / n
    Es = E[1:]
    L = 0.75 * math.pi * float(np.sum(Es / k)) / float(np.sum(Es))
    eps = 2.0 * nu0 * float(np.sum(k * k * Es))
    u_rms = math.sqrt(2.0 * E_k / 3.0)
    eta = (nu0 ** 3 / eps) ** 0.25
    lam = math.sqrt(15.0 * nu0 * u_rms * u_rms / eps)
    return {"L": L, "eps": eps, "u_rms": u_rms, "eta": eta, "lambda": lam,
            "Re_lambda": u_rms * lam / nu0}


def isotropy(u: np.ndarray) -> dict:
    """Isotropy diagnostics of a velocity field (3, nz, ny, nx) (Sec. 3.2)."""
    R = np.array([[np.mean(u[i] * u[j]) for j in range(3)] for i in range(3)])
    tr = np.trace(R)
    b = R / tr - np.eye(3) / 3.0
    II = -0.5 * float(np.sum(b * b.T))
    III = float(np.einsum("ij,jk,ki->", b, b, b)) / 3.0
    return {"E_frac": [float(R[i, i] / tr) for i in range(3)],
            "b": [float(b[0, 0]), float(b[1, 1]), float(b[2, 2]), float(b[0, 1]), float(b[0, 2]),
                  float(b[1, 2])],
            "II_b": II, "III_b": III,
            "xi": float(np.cbrt(III / 2.0)), "eta": float(np.sqrt(max(0.0, -II / 3.0)))}


def energy_balance(times, E_k, inj, eps):
    """Relative residual of Eq. (energy_balance) at the interior samples:
    (eps - (-dE_k/dt + <F.u>)) / eps with a central difference of E_k."""
    t = np.asarray(times, dtype=np.float64)
    E = np.asarray(E_k, dtype=np.float64)
    dEdt = (E[2:] - E[:-2]) / (t[2:] - t[:-2])
    rhs = -dEdt + np.asarray(inj, dtype=np.float64)[1:-1]
    e = np.asarray(eps, dtype=np.float64)[1:-1]
    return t[1:-1], (e - rhs) / e
