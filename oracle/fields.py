"""Initial fields of the method, computed by the oracle (TEST INFRASTRUCTURE ONLY).

Sec. 3.1 initialises with Taylor-Green vortices (Brachet 1983) without
printing the formula; the standard form is used here, with X = 2 pi x / nx:

* 3-D:  u = u0 sin X cos Y cos Z,  v = -u0 cos X sin Y cos Z,  w = 0
* 2-D:  u = u0 sin X cos Y,        v = -u0 cos X sin Y,        w = 0, with the
        pressure drho = 3 (u0^2 / 4) (cos 2X + cos 2Y) when requested.
"""
from __future__ import annotations

import numpy as np


def _grids(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return 2 * np.pi * x / nx, 2 * np.pi * y / ny, 2 * np.pi * z / nz


def tgv3d(nx: int, ny: int, nz: int, u0: float) -> np.ndarray:
    X, Y, Z = _grids(nx, ny, nz)
    u = np.zeros((3, nz, ny, nx))
    u[0] = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    return u


def tgv2d(nx: int, ny: int, nz: int, u0: float, with_pressure: bool = False):
    X, Y, _ = _grids(nx, ny, nz)
    u = np.zeros((3, nz, ny, nx))
    u[0] = u0 * np.sin(X) * np.cos(Y)
    u[1] = -u0 * np.cos(X) * np.sin(Y)
    drho = 3.0 * (u0 * u0 / 4.0) * (np.cos(2 * X) + np.cos(2 * Y)) if with_pressure else None
    return u, drho
