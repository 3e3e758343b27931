"""The blow-up of an over-energetic field is the scheme's, not the kernel's.

A 24^3 box, no forcing, C = 0, nu0 = 1e-4, seeded random field with u_rms =
0.1 per component (peaks of |u| near 0.45, Mach ~0.8 in lattice units).  The
GPU's initial populations are handed to the FP64 oracle, then both advance
one step at a time.  The largest |f'| of the two sides follow each other
through the onset: the populations agree to 1e-3 of the largest |f'| while
every |f'| stays below 0.25 (before the runaway growth), the first step at which some |f'| exceeds 1 (a population f = f' + w
outside [0, 1]) is the same on both sides, and both exceed 100 within two
steps of each other.  (The same comparison at 400^3, where the DNS-shape
workload of the benchmark turns unstable, is described with its numbers in
the design notes.)"""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


def test_onset_of_instability_matches_the_oracle(gpu_lib):
    lbm = gpu_lib
    n, nu0 = 24, 1e-4
    u = synthetic.random_solenoidal(n, seed=1, k0=2.0, urms=0.1)
    p = lbm.make_params(n, nu0=nu0, cs=0.0)
    ref = oracle.OracleLBM(n, n, n, nu0, 0.0, oracle.FORCE_NONE)
    first = {}
    over100 = {}
    with lbm.Lattice(p) as L:
        L.init(lbm.LBM_INIT_VELOCITY, u=u)
        ref.set_populations(L.populations())
        for t in range(1, 260):
            L.step(1)
            ref.step(1)
            fg, fo = L.populations(), ref.populations()
            mg, mo = float(np.abs(fg).max()), float(np.abs(fo).max())
            for side, m in (("gpu", mg), ("oracle", mo)):
                if side not in first and not m <= 1.0:
                    first[side] = t
                if side not in over100 and not m <= 100.0:
                    over100[side] = t
            if max(mg, mo) <= 0.25:  # before the runaway growth
                # (at this Mach number some full populations f = f' + w come
                # close to zero, so the difference is measured against the
                # largest |f'| rather than per population)
                dev = float(np.max(np.abs(fg - fo))) / mo
                assert dev <= 1e-3, (t, dev)
            if len(over100) == 2:
                break
    assert "gpu" in first and "oracle" in first, first
    assert first["gpu"] == first["oracle"], first
    assert abs(over100["gpu"] - over100["oracle"]) <= 2, over100
