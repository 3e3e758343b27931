"""Parameter chain of the paper (TEST INFRASTRUCTURE ONLY, part of the oracle).

Sec. 3.1 defines Re = U0 Nx / nu0; Eq. (forcing_amplitude) gives
F0 = Cf rho U0^2 / Nx (rho = rho0 = 1); Eq. (bare_viscosity) ties the bare
viscosity to the shear rate, nu0 = cs^2 (1/s_nu - 1/2) dt with cs^2 = 1/3.
Pinned against the numbers printed in Sec. 4 (tests/golden/parameter_chain.txt).
"""
from __future__ import annotations


def derive_nu0(u0: float, n: int, re: float) -> float:
    """nu0 = U0 N / Re (Sec. 3.1)."""
    return u0 * n / re


def forcing_amplitude(cf: float, u0: float, n: int, rho: float = 1.0) -> float:
    """F0 = Cf rho U0^2 / N (Eq. forcing_amplitude)."""
    return cf * rho * u0 * u0 / n


def bare_shear_rate(nu0: float) -> float:
    """s_nu0 = 1 / (1/2 + 3 nu0) (Eq. bare_viscosity, dt = 1)."""
    return 1.0 / (0.5 + 3.0 * nu0)


def tau_offset(nu: float) -> float:
    """tau - 1/2 = nu / cs^2 (Eq. tau_offset_scaling)."""
    return 3.0 * nu
