"""The Smagorinsky-constant study of Sec. 3.3 / 3.4 as a tested result.

The extended-self-similarity exponents zeta_p / zeta_3 (slopes of log S_p
against log |S_3| over the separations 2 <= r <= 16, p = 2, 4, 6) are computed
by the benchmark's own routine (bench.ess_exponents).

* Developed state: a 64^3 run at Re = 5000 with the paper's forcing from the
  seeded random field, 1500 steps on the GPU (about five large-eddy turnover
  times, so that S_3 has the sign and size of an energy cascade), C = 0 and
  C = 0.16.  The exponents from the GPU's structure functions (lbm_stats)
  equal those from the FP64 oracle's structure functions of the same velocity
  field (read back with lbm_get_velocity) to 1e-6, and are ordered
  zeta_2/zeta_3 < 1 < zeta_4/zeta_3 < zeta_6/zeta_3.
* Same run on both sides: 32^3, 100 steps, the GPU's S_p against the oracle's
  run within 1e-4 for p = 2, 4, 6 (S_3 of this barely evolved field is close
  to zero and crosses it between separations, so its exponents are not
  compared there)."""
import numpy as np
import pytest

import oracle
import synthetic
from oracle import diagnostics as dg

from bench import ess_exponents

pytestmark = pytest.mark.gpu

RE = 5000.0


@pytest.mark.parametrize("C", [0.0, 0.16])
def test_ess_exponents_of_a_developed_field(gpu_lib, C):
    lbm = gpu_lib
    n, steps = 64, 1500
    nu0 = 0.043 * n / RE
    F0 = oracle.forcing_amplitude(0.2, 0.043, n)
    p = lbm.make_params(n, nu0=nu0, cs=C, f0=F0, force_mode=lbm.LBM_FORCE_PAPER_SIN)
    with lbm.Lattice(p) as L:
        L.init_random(seed=3, urms=0.05, k0=4.0)
        L.step(steps)
        st = L.stats(what=lbm.LBM_STATS_STRUCTURE)
        u = lbm.lbm_get_velocity(L.h, 0, (n, n, n))
    sf = dg.structure_functions(u)
    assert st["r"] == sf["r"]
    got = ess_exponents(st)
    want = ess_exponents({"r": sf["r"], "Sp": sf["S"][:, 1:]})
    for q in (2, 4, 6):
        assert abs(got[q] - want[q]) <= 1e-6, (C, q, got[q], want[q])
    r = np.array(st["r"])
    sel = (r >= 2) & (r <= 16)
    assert np.all(st["Sp"][sel, 2] < 0.0)  # S_3 < 0: energy flows to small scales
    assert got[2] < 1.0 < got[4] < got[6]


@pytest.mark.parametrize("C", [0.0, 0.16])
def test_structure_functions_of_the_same_run(gpu_lib, C):
    lbm = gpu_lib
    n, steps = 32, 100
    nu0 = 0.043 * n / RE
    F0 = oracle.forcing_amplitude(0.2, 0.043, n)
    u = synthetic.random_solenoidal(n, seed=3, urms=0.05)
    ref = oracle.OracleLBM(n, n, n, nu0, C, oracle.FORCE_PAPER_SIN, F0=F0)
    ref.init_equilibrium(u)
    ref.step(steps)
    sf = dg.structure_functions(ref.fields()["u"])
    p = lbm.make_params(n, nu0=nu0, cs=C, f0=F0, force_mode=lbm.LBM_FORCE_PAPER_SIN)
    with lbm.Lattice(p) as L:
        L.init(lbm.LBM_INIT_VELOCITY, u=u)
        L.step(steps)
        st = L.stats(what=lbm.LBM_STATS_STRUCTURE)
    assert st["r"] == sf["r"]
    for q in (2, 4, 6):
        assert np.allclose(st["Sp"][:, q - 1], sf["S"][:, q], rtol=1e-4, atol=0.0), (C, q)
