"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the lattice Boltzmann method: it only draws
the random solenoidal initial velocity fields that stand in for the paper's
forced-turbulence states (the paper's own fields are not available).

Recipe (random spectrum, per seed):

1. Modes: every integer wavevector k with 0 < |k| <= kc, kc = min(n_min/2 - 1,
   6 k0), in the half space (kz > 0, or kz = 0 and ky > 0, or kz = ky = 0 and
   kx > 0); the partner -k carries the complex conjugate.  Beyond 6 k0 the
   target spectrum is below 1e-27 of its peak, so those modes are left empty.
2. Draws: for mode k and component d, two standard normals (real and imaginary
   part) by Box-Muller from two uniforms, each uniform from SplitMix64
   (Steele, Lea & Flood 2014) of a counter that encodes (seed, k, d, part).
3. Solenoidal projection: a <- a - k (k.a) / |k|^2.
4. Shell shape: the modes of integer shell s = round(|k|) are scaled so that the
   shell's energy 1/2 sum |u_hat|^2 equals s^4 exp(-2 (s/k0)^2).
5. Global scale: u_rms = sqrt(<u.u>/3) = urms exactly (evaluated from the
   coefficients via Parseval).
6. Synthesis: u(x) = sum_k u_hat(k) exp(2 pi i k.x / n), as three separable
   contractions (numpy on the host, or torch on a device for large lattices).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to counters x (uint64, wrapping)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + _GOLDEN).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _uniform(counter: np.ndarray) -> np.ndarray:
    r = splitmix64(counter)
    return ((r >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def _counters(seed: int, k: np.ndarray, d: int, part: int) -> np.ndarray:
    with np.errstate(over="ignore"):
        c = np.uint64(seed & 0xFFFFFFFF) * np.uint64(0x100000001B3)
        c = c + ((k[:, 0] + 512).astype(np.uint64) << np.uint64(40))
        c = c + ((k[:, 1] + 512).astype(np.uint64) << np.uint64(28))
        c = c + ((k[:, 2] + 512).astype(np.uint64) << np.uint64(16))
        c = c + np.uint64(d * 4 + part)
        return splitmix64(c)


def _normal(seed: int, k: np.ndarray, d: int, part: int) -> np.ndarray:
    u1 = _uniform(_counters(seed, k, d, 2 * part))
    u2 = _uniform(_counters(seed, k, d, 2 * part + 1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def half_space_modes(kc: int) -> np.ndarray:
    r = np.arange(-kc, kc + 1)
    kz, ky, kx = np.meshgrid(r, r, r, indexing="ij")
    k = np.stack([kx.ravel(), ky.ravel(), kz.ravel()], axis=1)
    k2 = np.sum(k * k, axis=1)
    half = (k[:, 2] > 0) | ((k[:, 2] == 0) & (k[:, 1] > 0)) | ((k[:, 2] == 0) & (k[:, 1] == 0) & (k[:, 0] > 0))
    keep = half & (k2 > 0) & (k2 <= kc * kc)
    return k[keep]


def mode_cutoff(nx: int, ny: int, nz: int, k0: float) -> int:
    return int(max(1, min(min(nx, ny, nz) // 2 - 1, int(6 * k0))))


def spectrum_coefficients(nx: int, ny: int, nz: int, seed: int, k0: float = 4.0,
                          urms: float = 0.05):
    """Half-space wavevectors (M, 3) int (kx, ky, kz) and coefficients (M, 3) complex."""
    kc = mode_cutoff(nx, ny, nz, k0)
    k = half_space_modes(kc)
    a = np.zeros((len(k), 3), dtype=np.complex128)
    for d in range(3):
        a[:, d] = _normal(seed, k, d, 0) + 1j * _normal(seed, k, d, 1)
    kf = k.astype(np.float64)
    k2 = np.sum(kf * kf, axis=1)
    ka = np.sum(kf * a, axis=1)
    a = a - kf * (ka / k2)[:, None]
    s = np.floor(np.sqrt(k2) + 0.5).astype(np.int64)
    e_half = np.sum(np.abs(a) ** 2, axis=1)  # the pair (k, -k) holds 2 * 1/2 |a|^2
    shell_e = np.bincount(s, weights=e_half)
    target = s.astype(np.float64) ** 4 * np.exp(-2.0 * (s / k0) ** 2)
    scale = np.sqrt(target / np.maximum(shell_e[s], 1e-300))
    a = a * scale[:, None]
    total = 2.0 * float(np.sum(np.abs(a) ** 2))  # <u.u> by Parseval
    a = a * (urms / math.sqrt(total / 3.0))
    return k, a


def _dense_cube(k: np.ndarray, a: np.ndarray, kc: int) -> np.ndarray:
    K = 2 * kc + 1
    cube = np.zeros((3, K, K, K), dtype=np.complex128)  # [d, kz, ky, kx]
    cube[:, k[:, 2] + kc, k[:, 1] + kc, k[:, 0] + kc] = a.T
    # conjugate partners
    cube[:, -k[:, 2] + kc, -k[:, 1] + kc, -k[:, 0] + kc] = np.conj(a.T)
    return cube


def _phases(n: int, kc: int) -> np.ndarray:
    kk = np.arange(-kc, kc + 1)[:, None]
    x = np.arange(n)[None, :]
    return np.exp(2j * math.pi * ((kk * x) % n) / n)  # [k, x]


def synthesize(k: np.ndarray, a: np.ndarray, nx: int, ny: int, nz: int) -> np.ndarray:
    """u (3, nz, ny, nx) float64 from the coefficients, on the host."""
    kc = int(np.max(np.abs(k))) if len(k) else 0
    cube = _dense_cube(k, a, kc)
    Ex, Ey, Ez = _phases(nx, kc), _phases(ny, kc), _phases(nz, kc)
    u = np.empty((3, nz, ny, nx))
    for d in range(3):
        t1 = cube[d] @ Ex                                   # [kz, ky, x]
        t2 = np.einsum("zyx,yY->zYx", t1, Ey, optimize=True)  # [kz, y, x]
        u[d] = np.tensordot(Ez, t2, axes=([0], [0])).real   # [z, y, x]
    return u


def synthesize_torch(k: np.ndarray, a: np.ndarray, nx: int, ny: int, nz: int, device,
                     dtype=None, zchunk: int = 64):
    """Same field as synthesize(), built on a torch device; returns (3, nz, ny, nx)."""
    import torch

    dtype = dtype or torch.float64
    kc = int(np.max(np.abs(k))) if len(k) else 0
    cube = torch.from_numpy(_dense_cube(k, a, kc)).to(device)
    Ex = torch.from_numpy(_phases(nx, kc)).to(device)
    Ey = torch.from_numpy(_phases(ny, kc)).to(device)
    Ez = torch.from_numpy(_phases(nz, kc)).to(device)
    out = torch.empty((3, nz, ny, nx), dtype=dtype, device=device)
    K = 2 * kc + 1
    for d in range(3):
        t1 = cube[d].reshape(K * K, K) @ Ex                        # [(kz ky), x]
        t1 = t1.reshape(K, K, nx).permute(0, 2, 1).reshape(K * nx, K)
        t2 = (t1 @ Ey).reshape(K, nx, ny).permute(0, 2, 1).reshape(K, ny * nx)  # [kz, (y x)]
        for z0 in range(0, nz, zchunk):
            z1 = min(nz, z0 + zchunk)
            blk = Ez[:, z0:z1].transpose(0, 1) @ t2                 # [z, (y x)]
            out[d, z0:z1] = blk.real.reshape(z1 - z0, ny, nx).to(dtype)
        del t1, t2
    return out


def random_solenoidal(nx: int, ny: int | None = None, nz: int | None = None, seed: int = 1,
                      k0: float = 4.0, urms: float = 0.05) -> np.ndarray:
    """Random solenoidal velocity (3, nz, ny, nx) float64 on the host."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    k, a = spectrum_coefficients(nx, ny, nz, seed, k0, urms)
    return synthesize(k, a, nx, ny, nz)
