"""The paper's 100^3 LES (Sec. 3.1, Sec. 4.1: Re = 2e4, C = 0.13, the paper's
forcing with U0 = 0.043 and Cf = 0.2, from the Taylor-Green field, t0 = 1000
steps) run into its statistically stationary interval, t/t0 in [200, 300],
on the GPU alone (no oracle can run 300,000 steps of it), against the
statements Sec. 3.2 and Sec. 4.1 make about that state:

* no negative offset: tau_e - 1/2 >= 3 nu0 in every cell (Eq. les_viscosity
  with nu_t >= 0), i.e. the smallest theta of every snapshot is the molecular
  one up to FP32 rounding;
* the 5th percentile of theta stays above 1.0e-3;
* the hydrodynamic regime, theta << 1 (here: every cell below 0.1);
* statistical isotropy in the mean: the time-averaged directional energy
  fractions E_i / E within 0.05 of 1/3 (the paper: within 1 % of 1/3 over
  t/t0 in [200, 1000], snapshot deviations ~0.05).

And, in that turbulent state, the strain rate the closure uses (from the
non-equilibrium moments, Eq. yu_strain -> Eq. strain_norm) against the
strain rate of the velocity field itself (spectral gradients, |S| =
sqrt(2 S_ij S_ij)): cell by cell correlated above 0.98, means within 10 %.

The level of theta (the paper prints a mean ~1.34e-3) is reported by the
benchmark, not asserted here."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, T0 = 100, 1000
U0, CF, RE, C = 0.043, 0.2, 2.0e4, 0.13


@pytest.fixture(scope="module")
def stationary_records(gpu_lib):
    lbm = gpu_lib
    nu0 = U0 * N / RE
    p = lbm.make_params(N, nu0=nu0, cs=C, f0=CF * U0 * U0 / N, force_mode=lbm.LBM_FORCE_PAPER_SIN)
    recs = []
    with lbm.Lattice(p) as L:
        L.init(lbm.LBM_INIT_TGV3D, amplitude=U0)
        L.step(200 * T0)
        for _ in range(10):
            L.step(10 * T0)
            recs.append(L.stats())
        fields = L.fields()
    return nu0, recs, fields


def test_no_negative_offset_and_hydrodynamic_regime(stationary_records):
    nu0, recs, _ = stationary_records
    th0 = np.float32(3 * nu0)
    for st in recs:
        assert st["theta_min"] >= th0 * (1 - 1e-6), (st["step"], st["theta_min"], 3 * nu0)
        assert st["theta_max"] < 0.1, st["step"]


def test_fifth_percentile_above_1e_3(stationary_records):
    _, recs, _ = stationary_records
    for st in recs:
        assert st["theta_p05"] > 1.0e-3, (st["step"], st["theta_p05"])


def test_isotropic_in_the_mean(stationary_records):
    _, recs, _ = stationary_records
    frac = np.mean([st["E_frac"] for st in recs], axis=0)
    assert np.all(np.abs(frac - 1.0 / 3.0) <= 0.05), frac


def test_closure_strain_matches_velocity_gradients(stationary_records):
    _, _, fl = stationary_records
    u = fl["u"]  # [3][z][y][x]
    k = np.fft.fftfreq(N) * 2 * np.pi
    kk = (k[None, None, :], k[None, :, None], k[:, None, None])  # along x, y, z
    uh = [np.fft.fftn(u[a]) for a in range(3)]
    G = [[np.real(np.fft.ifftn(1j * kk[b] * uh[a])) for b in range(3)] for a in range(3)]
    S = np.sqrt(2 * sum(0.25 * (G[a][b] + G[b][a]) ** 2 for a in range(3) for b in range(3)))
    sn = fl["snorm"]
    assert np.corrcoef(S.ravel(), sn.ravel())[0, 1] >= 0.98
    assert abs(sn.mean() / S.mean() - 1.0) <= 0.10, (sn.mean(), S.mean())
