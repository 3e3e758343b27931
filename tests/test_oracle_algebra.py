"""Pins of the oracle's algebra (App. A, App. B) against facts that do not come
from the oracle itself: the velocity-set isotropy, the published polynomial
definitions of the d'Humieres moment basis, orthogonality, the Guo source
moments, the paper's worked numbers (tests/golden/)."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v, tol = line.split()
            out[k] = (float(v), float(tol))
    return out


def test_velocity_set_isotropy():
    c, w = oracle.lattice()
    assert len({tuple(v) for v in c}) == 19
    assert tuple(c[18]) == (0, 0, 0)
    # opposite pairs (1,2), (3,4), ... in the paper's order
    for p in range(9):
        assert np.array_equal(c[2 * p], -c[2 * p + 1])
    assert math.isclose(w.sum(), 1.0, abs_tol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    # second and fourth order isotropy of D3Q19: sum w c_a c_b = cs^2 delta,
    # sum w c_a c_b c_c c_d = cs^4 (delta delta + delta delta + delta delta)
    cs2 = 1.0 / 3.0
    T2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(T2, cs2 * np.eye(3), atol=1e-15)
    T4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    ref = cs2 * cs2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(T4, ref, atol=1e-15)


def test_moment_rows_are_the_published_polynomials():
    """Each typed row of M equals the d'Humieres et al. (2002) polynomial of c."""
    c, _ = oracle.lattice()
    M = oracle.moment_matrix()
    cx, cy, cz = c[:, 0].astype(float), c[:, 1].astype(float), c[:, 2].astype(float)
    c2 = cx * cx + cy * cy + cz * cz
    rows = [
        np.ones(19),
        19 * c2 - 30,
        (21 * c2 * c2 - 53 * c2 + 24) / 2,
        cx, (5 * c2 - 9) * cx,
        cy, (5 * c2 - 9) * cy,
        cz, (5 * c2 - 9) * cz,
        3 * cx * cx - c2, (3 * c2 - 5) * (3 * cx * cx - c2),
        cy * cy - cz * cz, (3 * c2 - 5) * (cy * cy - cz * cz),
        cx * cy, cy * cz, cx * cz,
        (cy * cy - cz * cz) * cx, (cz * cz - cx * cx) * cy, (cx * cx - cy * cy) * cz,
    ]
    for k, r in enumerate(rows):
        assert np.array_equal(M[k], r), f"row {k}"


def test_moment_matrix_orthogonal_and_inverse():
    M = oracle.moment_matrix()
    G = M @ M.T
    assert np.array_equal(G, np.diag(np.diag(G)))
    norms = [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    assert np.array_equal(np.diag(G), norms)
    Minv = oracle.invert(M)
    assert np.allclose(Minv @ M, np.eye(19), atol=1e-13)
    # orthogonality gives M^-1 = M^T diag(1/|row|^2): the Gauss-Jordan inverse agrees
    assert np.allclose(Minv, M.T / np.array(norms, dtype=float), atol=1e-14)


def test_shift_by_weights():
    """M w = (1, -11, 3, 0, ...): the weights carry rho0 = 1 (reading: f' = f - w)."""
    _, w = oracle.lattice()
    m = oracle.moment_matrix() @ w
    ref = np.zeros(19)
    ref[:3] = [1.0, -11.0, 3.0]
    assert np.allclose(m, ref, atol=1e-14)


def test_invert_generic():
    rng = np.random.default_rng(3)
    A = rng.normal(size=(7, 7)) + 7 * np.eye(7)
    assert np.allclose(oracle.invert(A) @ A, np.eye(7), atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.invert(np.zeros((3, 3)))


def test_relaxation_rates():
    lam = oracle.relaxation_rates(1.7)
    ref = [1.0, 1.19, 1.4, 1.0, 1.2, 1.0, 1.2, 1.0, 1.2, 1.7, 1.4, 1.7, 1.4, 1.7, 1.7, 1.7,
           1.98, 1.98, 1.98]
    assert np.array_equal(lam, ref)


@pytest.mark.parametrize("seed", range(5))
def test_guo_source_moments(seed):
    """M Phi (Eq. guo_force) equals the printed force moments F_m (Eq. meq_fm);
    Phi has zero mass, momentum F and second moment uF + Fu (Guo 2002)."""
    rng = np.random.default_rng(seed)
    u = rng.normal(scale=0.05, size=3)
    F = rng.normal(scale=1e-3, size=3)
    c, _ = oracle.lattice()
    Phi = oracle.guo_source(u, F)
    assert np.allclose(oracle.moment_matrix() @ Phi, oracle.force_moments_printed(u, F),
                       rtol=1e-13, atol=1e-18)
    assert abs(Phi.sum()) < 1e-18
    assert np.allclose(Phi @ c, F, rtol=1e-13, atol=1e-19)
    second = np.einsum("i,ia,ib->ab", Phi, c, c)
    assert np.allclose(second, np.outer(u, F) + np.outer(F, u), rtol=1e-12, atol=1e-19)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments_vs_polynomial_feq(seed):
    """The printed m^eq agrees with M (f^eq - w) of the polynomial f^eq (Eq. feq) in
    every conserved and hydrodynamic-stress row; it differs only in rows 2, 10, 12,
    where f^eq corresponds to the free parameters (3 drho - 11/2 rho u^2, -1/2 rho
    (3ux^2 - u^2), -1/2 rho (uy^2 - uz^2)) and the paper prints
    (-475/63 rho u^2, 0, 0)."""
    rng = np.random.default_rng(seed)
    u = rng.normal(scale=0.05, size=3)
    drho = rng.normal(scale=1e-2)
    rho = 1.0 + drho
    _, w = oracle.lattice()
    M = oracle.moment_matrix()
    mpoly = M @ (oracle.feq_poly(rho, u) - w)
    meq = oracle.meq(drho, u)
    same = [0, 1, 3, 4, 5, 6, 7, 8, 9, 11, 13, 14, 15, 16, 17, 18]
    assert np.allclose(mpoly[same], meq[same], rtol=1e-12, atol=1e-15)
    uu = float(u @ u)
    assert math.isclose(mpoly[2], 3 * drho - 5.5 * rho * uu, rel_tol=1e-12, abs_tol=1e-15)
    assert math.isclose(mpoly[10], -0.5 * rho * (3 * u[0] ** 2 - uu), rel_tol=1e-12, abs_tol=1e-15)
    assert math.isclose(mpoly[12], -0.5 * rho * (u[1] ** 2 - u[2] ** 2), rel_tol=1e-12, abs_tol=1e-15)
    assert math.isclose(meq[2], -475.0 / 63.0 * rho * uu, rel_tol=1e-14)
    assert meq[10] == 0.0 and meq[12] == 0.0


def test_strain_special_cases():
    s1, s9 = 1.19, 1.6
    m = np.zeros(19)
    m[13] = 2e-4
    S = oracle.strain(m, s1, s9)
    assert np.allclose(S, [0, 0, 0, -1.5 * s9 * 2e-4, 0, 0], atol=1e-18)
    assert math.isclose(oracle.strain_norm(S), 2 * abs(S[3]), rel_tol=1e-14)
    m = np.zeros(19)
    m[14], m[15] = 1e-4, -3e-4
    S = oracle.strain(m, s1, s9)
    assert math.isclose(S[5], -1.5 * s9 * 1e-4) and math.isclose(S[4], 1.5 * s9 * 3e-4)
    # trace: Sxx + Syy + Szz = -(s1 m1)(1/38 + 2/76 + 2/76) = -3 s1 m1 / 38, the
    # Chapman-Enskog divergence of the energy mode (m9, m11 cancel)
    m = np.zeros(19)
    m[1], m[9], m[11] = 3e-4, 1e-4, -2e-4
    S = oracle.strain(m, s1, s9)
    assert math.isclose(S[0] + S[1] + S[2], -3.0 * s1 * 3e-4 / 38.0, rel_tol=1e-12)
    # traceless part: m1 = 0 -> Syy - Szz = -(3/2) s9 m11 ... from the printed formula
    m = np.zeros(19)
    m[11] = 1e-4
    S = oracle.strain(m, s1, s9)
    assert math.isclose(S[0] + S[1] + S[2], 0.0, abs_tol=1e-20)
    # diag(a, -a, 0): |S| = 2|a|
    assert math.isclose(oracle.strain_norm([0.3, -0.3, 0, 0, 0, 0]), 0.6, rel_tol=1e-14)


def test_k41_worked_example():
    """Sec. 4: |S| = 0.00926 -> tau_t = 0.0036114, tau_e = 0.5042564,
    nu_e = 0.0014188, Re_e ~ 3030 (tests/golden/k41_chain.txt)."""
    g = _golden("k41_chain.txt")
    nu0 = oracle.derive_nu0(0.043, 100, 2e4)
    # |S| ~ U0 / (L^(1/3) l^(2/3)), L = 100, l = 1
    S = 0.043 / (100.0 ** (1.0 / 3.0))
    assert abs(S - g["S_norm"][0]) <= g["S_norm"][1]
    Sp = g["S_norm"][0]  # the paper carries the rounded value forward
    te = oracle.tau_e(nu0, 0.13, Sp)
    tau_t = te - oracle.tau_e(nu0, 0.0, Sp)
    assert abs(tau_t - g["tau_t"][0]) <= g["tau_t"][1]
    assert abs(te - g["tau_e"][0]) <= g["tau_e"][1]
    nu_e = (te - 0.5) / 3.0
    assert abs(nu_e - g["nu_e"][0]) <= g["nu_e"][1]
    assert abs(0.043 * 100 / nu_e - g["Re_e"][0]) <= g["Re_e"][1]
    assert abs(tau_t / (3 * nu0) - g["ratio"][0]) <= g["ratio"][1]
    assert abs((te - 0.5) - g["offset_bound"][0]) <= g["offset_bound"][1]


def test_parameter_chain():
    g = _golden("parameter_chain.txt")

    def ok(name, val):
        ref, tol = g[name]
        assert math.isclose(val, ref, rel_tol=tol), (name, val, ref)

    ok("nu0_les", oracle.derive_nu0(0.043, 100, 2e4))
    ok("nu0_dns", oracle.derive_nu0(0.043, 800, 2e4))
    ok("tau_offset_les", oracle.params.tau_offset(oracle.derive_nu0(0.043, 100, 2e4)))
    ok("tau_offset_dns", oracle.params.tau_offset(oracle.derive_nu0(0.043, 800, 2e4)))
    ok("F0_100", oracle.forcing_amplitude(0.2, 0.043, 100))
    ok("F0_800", oracle.forcing_amplitude(0.2, 0.043, 800))
    # Eq. bare_viscosity round trip
    s = oracle.bare_shear_rate(0.01)
    assert math.isclose((1.0 / s - 0.5) / 3.0, 0.01, rel_tol=1e-14)


def test_selfconsistent_strain_closed_form_pure_shear():
    """Pure shear (only m13 non-equilibrium): |S| = s_nu |P| with |P| the norm at
    s9 = 1 and s_nu = 1/(1/2 + 3 nu0 + 3 C |S|), so 3C|S|^2 + (1/2 + 3 nu0)|S| - |P| = 0
    (the closed form of the BGK-Smagorinsky relaxation time)."""
    nu0, C = 2.15e-4, 0.13
    m = np.zeros(19)
    m[13] = -4e-3
    P = oracle.strain_norm(oracle.strain(m, 1.19, 1.0))
    a, b = 3 * C, 0.5 + 3 * nu0
    exact = (-b + math.sqrt(b * b + 4 * a * P)) / (2 * a)
    assert math.isclose(oracle.strain_norm_selfconsistent(m, 1.19, nu0, C), exact, rel_tol=1e-13)
    # C = 0 reduces to the explicit formula with the bare rate
    S0 = oracle.strain_norm(oracle.strain(m, 1.19, 1.0 / (0.5 + 3 * nu0)))
    assert math.isclose(oracle.strain_norm_selfconsistent(m, 1.19, nu0, 0.0), S0, rel_tol=1e-15)
    # with the closure active the local rate is slower, so |S| is smaller
    assert oracle.strain_norm_selfconsistent(m, 1.19, nu0, C) < S0


def test_selfconsistent_strain_is_a_fixed_point():
    rng = np.random.default_rng(11)
    for _ in range(5):
        m = np.zeros(19)
        m[[1, 9, 11, 13, 14, 15]] = rng.normal(scale=2e-3, size=6)
        nu0, C = 1e-3, 0.2
        s = oracle.strain_norm_selfconsistent(m, 1.19, nu0, C)
        again = oracle.strain_norm(oracle.strain(m, 1.19, 1.0 / (0.5 + 3 * (nu0 + C * s))))
        assert math.isclose(again, s, rel_tol=1e-13)


# The relaxation rates printed in Eq. (relaxation-matrix), by moment row: the
# conserved rows 0, 3, 5, 7 (any rate: m = m^eq there), the energy mode 1, the
# energy square 2, the heat fluxes 4, 6, 8, the stress rows 9, 11, 13, 14, 15
# (the shear rate s_nu), their fourth-order partners 10, 12 and the
# third-order rows 16-18.
PRINTED_RATES = {1: 1.19, 2: 1.4, 4: 1.2, 6: 1.2, 8: 1.2, 10: 1.4, 12: 1.4, 16: 1.98, 17: 1.98, 18: 1.98}
SHEAR_ROWS = (9, 11, 13, 14, 15)


@pytest.mark.parametrize("k", [1, 2, 4, 6, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18])
@pytest.mark.parametrize("flow", [False, True])
def test_one_collision_relaxes_each_moment_at_its_rate(k, flow):
    """Observed, not read from the oracle's rate table: a uniform cell at its
    equilibrium (at rest, or in a uniform flow) with one moment k moved off
    equilibrium by delta, no force, C = 0; after one collision of Eq.
    (mrt_les_guo) the moment's departure is (1 - s_k) delta and every other
    moment is still at equilibrium.  This observes every rate of Eq.
    (relaxation-matrix), including the ones without a hydrodynamic effect (s2,
    s4, s10 = s12, s16-18), and, in a flow, the equilibrium each row relaxes to
    (e.g. m2 -> -475/63 rho u^2 of Eq. meq_fm)."""
    nu0 = 0.01
    s_nu = 1.0 / (0.5 + 3.0 * nu0)  # Eq. (bare_viscosity)
    s_k = s_nu if k in SHEAR_ROWS else PRINTED_RATES[k]
    u = np.array([0.03, -0.02, 0.01]) if flow else np.zeros(3)
    drho = 0.004 if flow else 0.0
    M = oracle.moment_matrix()
    m_eq = oracle.meq(drho, u)
    delta = 1e-3
    m = m_eq.copy()
    m[k] += delta
    fp = np.linalg.solve(M, m)  # library solve: the oracle's own inverse is not used here
    fstar, _ = oracle.collide_one(fp, np.zeros(3), nu0, 0.0)
    mstar = M @ fstar
    want = m_eq.copy()
    want[k] += (1.0 - s_k) * delta
    assert np.allclose(mstar, want, rtol=0.0, atol=1e-13), (k, mstar - want)


def test_energy_square_relaxes_to_the_printed_equilibrium():
    """Row 2 in a uniform flow, started at m2 = 0: one collision moves it to
    s2 m2^eq with m2^eq = -475/63 rho |u|^2 (Eq. meq_fm) and s2 = 1.4 (Eq.
    relaxation-matrix), values typed from the paper; repeated collisions
    converge to m2^eq."""
    u = np.array([0.04, 0.01, -0.03])
    drho = 0.002
    rho = 1.0 + drho
    M = oracle.moment_matrix()
    m = oracle.meq(drho, u)
    m[2] = 0.0
    fp = np.linalg.solve(M, m)
    f1, _ = oracle.collide_one(fp, np.zeros(3), 0.01, 0.0)
    eq2 = -475.0 / 63.0 * rho * float(u @ u)
    assert math.isclose((M @ f1)[2], 1.4 * eq2, rel_tol=1e-12)
    f = fp
    for _ in range(40):
        f, _ = oracle.collide_one(f, np.zeros(3), 0.01, 0.0)
    assert math.isclose((M @ f)[2], eq2, rel_tol=1e-12)
