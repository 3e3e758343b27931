"""Physics pins of the oracle's time step: what the method fixes independently of
any implementation (equilibrium fixed point, conservation laws, the C -> 0
limit of Sec. 2.3, viscous decay of a Taylor-Green vortex, the closed-form
Kolmogorov-flow amplitude F/(nu k^2), the strain of Eq. (yu_strain) against the
analytic velocity gradient, and the cubic symmetry of the collision)."""
import math

import numpy as np
import pytest

import oracle
from oracle import fields


def _random_state(shape, seed, scale=1e-3):
    """A smooth-ish random near-equilibrium field: equilibrium of a random velocity
    plus a small random non-equilibrium part."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    u = rng.normal(scale=0.03, size=(3, nz, ny, nx))
    L = oracle.OracleLBM(nx, ny, nz, 0.02, 0.1)
    L.init_equilibrium(u)
    f = L.populations() + rng.normal(scale=scale, size=(19, nz, ny, nx))
    return f


def _mom(p, c):
    return c.T.astype(float) @ p.reshape(19, -1).sum(axis=1)


def test_equilibrium_is_fixed_point():
    """Uniform (drho, u), F = 0: f' = M^-1 m^eq(drho, u) is unchanged by collide and
    stream, for any C (m_neq = 0 gives |S| = 0 and s_nu = s_nu0)."""
    for C in (0.0, 0.13):
        L = oracle.OracleLBM(5, 4, 3, 0.01, C)
        u = np.zeros((3, 3, 4, 5))
        u[0], u[1], u[2] = 0.04, -0.02, 0.01
        drho = np.full((3, 4, 5), 3e-3)
        L.init_equilibrium(u, drho)
        f0 = L.populations()
        L.step(7)
        assert np.abs(L.populations() - f0).max() < 1e-15
        fl = L.fields()
        assert np.abs(fl["snorm"]).max() < 1e-14
        assert np.allclose(fl["theta"], 3 * 0.01, atol=1e-14)


@pytest.mark.parametrize("force_mode", [oracle.FORCE_NONE, oracle.FORCE_PAPER_SIN])
def test_mass_and_momentum_conserved(force_mode):
    shape = (6, 5, 7)
    f = _random_state(shape, 1)
    L = oracle.OracleLBM(7, 5, 6, 0.005, 0.13, force_mode, F0=1e-4)
    L.set_populations(f)
    c, _ = oracle.lattice()
    m0 = L.populations().sum()
    j0 = _mom(L.populations(), c)
    for _ in range(3):
        L.step(4)
        p = L.populations()
        assert abs(p.sum() - m0) < 1e-14
        # the paper's forcing sums to zero over the periodic box: momentum conserved
        assert np.allclose(_mom(p, c), j0, atol=1e-14)


def test_constant_force_momentum_increment():
    """Guo forcing: every step adds exactly F to j = sum f c in every cell, so the
    box momentum grows by ncell * F per step."""
    shape = (4, 6, 5)
    f = _random_state(shape, 2)
    F = np.array([1e-6, -2e-6, 5e-7])
    L = oracle.OracleLBM(5, 6, 4, 0.01, 0.1, oracle.FORCE_CONST, body=F)
    L.set_populations(f)
    c, _ = oracle.lattice()
    j0 = _mom(L.populations(), c)
    L.step(10)
    j1 = _mom(L.populations(), c)
    assert np.allclose(j1 - j0, 10 * 120 * F, rtol=1e-9, atol=1e-15)


def test_C_zero_is_constant_viscosity_mrt_bitwise():
    """Sec. 2.3: the LES model reduces to DNS-MRT as C -> 0, bit for bit."""
    shape = (4, 5, 6)
    f = _random_state(shape, 3)
    A = oracle.OracleLBM(6, 5, 4, 0.01, 0.0, oracle.FORCE_PAPER_SIN, F0=1e-4)
    B = oracle.OracleLBM(6, 5, 4, 0.01, 0.0, oracle.FORCE_PAPER_SIN, F0=1e-4)
    B.set_fixed_rate(True)
    A.set_populations(f)
    B.set_populations(f)
    A.step(5)
    B.step(5)
    assert np.array_equal(A.populations(), B.populations())
    # and C > 0 changes the result (the closure is active)
    Cq = oracle.OracleLBM(6, 5, 4, 0.01, 0.2, oracle.FORCE_PAPER_SIN, F0=1e-4)
    Cq.set_populations(f)
    Cq.step(5)
    assert np.abs(Cq.populations() - A.populations()).max() > 1e-9


def test_theta_bounded_below():
    """theta = tau_e - 1/2 = 3 (nu0 + nu_t) >= 3 nu0 everywhere (Sec. 4.1)."""
    shape = (6, 6, 6)
    f = _random_state(shape, 4, scale=3e-3)
    L = oracle.OracleLBM(6, 6, 6, 2.15e-4, 0.13)
    L.set_populations(f)
    L.step(3)
    th = L.fields()["theta"]
    assert th.min() >= 3 * 2.15e-4 - 1e-18
    assert th.max() > 3 * 2.15e-4  # the closure is active somewhere


def test_taylor_green_2d_viscous_decay():
    """2-D Taylor-Green vortex: the amplitude decays as exp(-2 nu0 k^2 t),
    k = 2 pi / N (gate: rate within 1 %)."""
    n, u0, nu0 = 32, 0.01, 0.02
    u, drho = fields.tgv2d(n, n, 1, u0, with_pressure=True)
    L = oracle.OracleLBM(n, n, 1, nu0, 0.0)
    L.init_equilibrium(u, drho)
    X = 2 * np.pi * np.arange(n) / n
    mode = np.sin(X)[None, None, :] * np.cos(X)[None, :, None]

    def amp():
        return float(np.mean(L.fields()["u"][0] * mode) / np.mean(mode * mode))

    L.step(100)
    a1 = amp()
    L.step(400)
    a2 = amp()
    rate = math.log(a1 / a2) / 400.0
    k = 2 * np.pi / n
    assert abs(rate / (2 * nu0 * k * k) - 1.0) < 0.01


def test_kolmogorov_flow_amplitude_and_strain():
    """Kolmogorov flow F = F0 sin(k y) x: steady u_x = F0/(nu k^2) sin(k y) (the
    nonlinear term vanishes); the strain of Eq. (yu_strain) gives
    |S| = 2 |S_xy| = U k |cos(k y)|.  Gates: 1 %."""
    ny, nu0, F0 = 32, 0.1, 1e-6
    L = oracle.OracleLBM(2, ny, 2, nu0, 0.0, oracle.FORCE_KOLMOGOROV, F0=F0)
    L.init_equilibrium(np.zeros((3, 2, ny, 2)))
    k = 2 * np.pi / ny
    L.step(int(12 / (nu0 * k * k)))
    fl = L.fields()
    y = np.arange(ny)
    prof = fl["u"][0][0, :, 0]
    U = float(np.sum(prof * np.sin(k * y)) / np.sum(np.sin(k * y) ** 2))
    assert abs(U / (F0 / (nu0 * k * k)) - 1.0) < 0.01
    assert np.abs(fl["u"][1]).max() < 1e-3 * U and np.abs(fl["u"][2]).max() < 1e-3 * U
    sn = fl["snorm"][0, :, 0]
    ref = U * k * np.abs(np.cos(k * y))
    assert np.abs(sn - ref).max() < 0.01 * U * k


def test_strain_matches_velocity_gradient_taylor_green():
    """Decaying 2-D Taylor-Green flow: the moment-based strain norm equals
    |S| = sqrt(2 S_ij S_ij) of the analytic gradient of the current field,
    S_xx = -S_yy = u0' k cos X cos Y, S_xy = 0 (gate: 2 % of the maximum)."""
    n, u0, nu0 = 32, 0.01, 0.05
    u, drho = fields.tgv2d(n, n, 1, u0, with_pressure=True)
    L = oracle.OracleLBM(n, n, 1, nu0, 0.0)
    L.init_equilibrium(u, drho)
    L.step(60)
    fl = L.fields()
    X = 2 * np.pi * np.arange(n) / n
    mode = np.sin(X)[None, None, :] * np.cos(X)[None, :, None]
    a = float(np.mean(fl["u"][0] * mode) / np.mean(mode * mode))
    k = 2 * np.pi / n
    Sxx = a * k * np.cos(X)[None, None, :] * np.cos(X)[None, :, None]
    ref = np.sqrt(2 * (2 * Sxx * Sxx))
    assert np.abs(fl["snorm"] - ref).max() < 0.02 * np.abs(ref).max()


def _rotate_z(fp, c):
    """Rotate a population field by +90 degrees about z on an n x n periodic
    plane: cell (x, y) moves to (-y mod n, x) and population c_a becomes the
    population with velocity R c_a."""
    nz, ny, nx = fp.shape[1:]
    assert nx == ny
    out = np.empty_like(fp)
    R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]])
    perm = np.empty(19, dtype=int)
    for a in range(19):
        rc = R @ c[a]
        perm[a] = [b for b in range(19) if np.array_equal(c[b], rc)][0]
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    xn = (-yy) % nx
    yn = xx
    for a in range(19):
        out[perm[a]][:, yn, xn] = fp[a][:, yy, xx]
    return out


def test_cubic_symmetry_of_the_collision():
    """Rotating the lattice by 90 degrees commutes with the time step (the MRT
    rates of Eq. relaxation-matrix and |S| are invariant under the cubic group)."""
    c, _ = oracle.lattice()
    n = 6
    f = _random_state((4, n, n), 5, scale=2e-3)
    A = oracle.OracleLBM(n, n, 4, 0.003, 0.13)
    B = oracle.OracleLBM(n, n, 4, 0.003, 0.13)
    A.set_populations(f)
    B.set_populations(_rotate_z(f, c))
    A.step(3)
    B.step(3)
    assert np.abs(_rotate_z(A.populations(), c) - B.populations()).max() < 1e-15


def test_mirror_symmetry():
    """x -> -x mirror commutes with the time step."""
    c, _ = oracle.lattice()
    f = _random_state((3, 4, 5), 6, scale=2e-3)
    perm = [[b for b in range(19) if np.array_equal(c[b], c[a] * np.array([-1, 1, 1]))][0]
            for a in range(19)]

    def mirror(fp):
        out = np.empty_like(fp)
        nx = fp.shape[-1]
        idx = (-np.arange(nx)) % nx
        for a in range(19):
            out[perm[a]] = fp[a][..., idx]
        return out

    A = oracle.OracleLBM(5, 4, 3, 0.004, 0.1)
    B = oracle.OracleLBM(5, 4, 3, 0.004, 0.1)
    A.set_populations(f)
    B.set_populations(mirror(f))
    A.step(4)
    B.step(4)
    assert np.abs(mirror(A.populations()) - B.populations()).max() < 1e-15


def test_streaming_direction():
    """Streaming moves population a by +c_a per step with periodic wrap: perturb
    every population of one cell of a rest state and find, after one step, the
    largest deviation of population a one link away along c_a."""
    c, _ = oracle.lattice()
    n = 8
    L = oracle.OracleLBM(n, n, n, 0.1, 0.0)
    L.init_equilibrium(np.zeros((3, n, n, n)))
    f = L.populations()
    f[:, 2, 3, 4] += 1e-3  # perturb one cell in every population
    L.set_populations(f)
    L.step(1)
    g = L.populations()
    for a in range(19):
        # the largest deviation of population a after one step sits at x + c_a
        z, y, x = np.unravel_index(np.argmax(np.abs(g[a])), g[a].shape)
        assert (x, y, z) == ((4 + c[a][0]) % n, (3 + c[a][1]) % n, (2 + c[a][2]) % n)


def test_single_cell_collision_matches_the_lattice_step():
    """orc_collide_one reproduces, cell by cell, the collision inside the lattice
    step: after one push step, f_a(x + c_a) = f*_a(x)."""
    c, _ = oracle.lattice()
    shape = (3, 4, 5)
    f = _random_state(shape, 8, scale=2e-3)
    L = oracle.OracleLBM(5, 4, 3, 0.004, 0.13, oracle.FORCE_PAPER_SIN, F0=1e-3)
    L.set_populations(f)
    F = L.force_field()
    L.step(1)
    g = L.populations()
    for (z, y, x) in [(0, 0, 0), (1, 2, 3), (2, 3, 4)]:
        fs, th = oracle.collide_one(f[:, z, y, x], F[:, z, y, x], 0.004, 0.13)
        for a in range(19):
            xd, yd, zd = (x + c[a][0]) % 5, (y + c[a][1]) % 4, (z + c[a][2]) % 3
            assert g[a, zd, yd, xd] == fs[a]
        assert th >= 3 * 0.004


def test_paper_forcing_is_a_solenoidal_large_scale_field():
    """Eq. (forcing_pattern) with the amplitude of Eq. (forcing_amplitude): each
    component is a single Fourier mode of the box (|k| = 2 pi / N) along a
    coordinate other than its own, so the force is divergence-free, sums to
    zero over the box, and has mean square F0^2 / 2 per component and peak
    value F0 (N divisible by 4).  A component tied to its own coordinate, a
    wrong wave number or a lost component fails here."""
    n, F0 = 8, 1e-3
    L = oracle.OracleLBM(n, n, n, 0.01, 0.0, oracle.FORCE_PAPER_SIN, F0=F0)
    F = L.force_field()  # [3][z][y][x], components (x, y, z)
    Fh = np.fft.fftn(F, axes=(1, 2, 3))
    k = np.rint(np.fft.fftfreq(n) * n).astype(int)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    div = kx * Fh[0] + ky * Fh[1] + kz * Fh[2]
    assert np.abs(div).max() <= 1e-12 * np.abs(Fh).max()
    own_axis = {0: 2, 1: 1, 2: 0}  # array axis (of z, y, x) of component i's own coordinate
    for i in range(3):
        assert abs(F[i].sum()) <= 1e-15
        assert np.isclose((F[i] ** 2).mean(), F0 ** 2 / 2, rtol=1e-12)
        assert np.isclose(np.abs(F[i]).max(), F0, rtol=1e-12)
        P = np.abs(Fh[i]) ** 2
        modes = np.argwhere(P > 1e-20 * P.max())
        assert len(modes) == 2  # +k and -k of one wave vector
        kvec = [tuple(int(k[j]) for j in m) for m in modes]  # (kz, ky, kx)
        nonzero_axes = {a for kv in kvec for a in range(3) if kv[a] != 0}
        assert len(nonzero_axes) == 1
        (ax,) = nonzero_axes
        assert {abs(kv[ax]) for kv in kvec} == {1}
        assert ax != own_axis[i]


def test_sound_wave_speed_and_bulk_viscosity():
    """A standing sound wave (drho = A cos kx at rest) oscillates at c_s k,
    c_s^2 = 1/3 (set by the energy-moment equilibrium -11 drho + 19 rho u^2 of
    Eq. meq_fm), and decays at Gamma = (k^2 / 2)(4 nu / 3 + zeta), the
    attenuation of the linearised Navier-Stokes equations with the bulk
    viscosity zeta = (2/9)(1/s1 - 1/2) that the energy mode's rate s1 = 1.19 of
    Eq. relaxation-matrix gives a D3Q19 MRT model.  The shear tests do not see
    s1; this one does (s1 = 1.9 would give a third of the decay).  Frequency and
    rate from Prony's fit of the mode amplitude, 64 x 1 x 1 box, 2000 steps."""
    n, nu0, A = 64, 0.01, 1e-5
    k = 2 * np.pi / n
    x = np.arange(n)
    L = oracle.OracleLBM(n, 1, 1, nu0, 0.0)
    L.init_equilibrium(np.zeros((3, 1, 1, n)), (A * np.cos(k * x)).reshape(1, 1, n))
    T = 2000
    a = np.zeros(T + 1)
    for t in range(T + 1):
        if t:
            L.step(1)
        a[t] = 2.0 / n * np.dot(L.fields()["drho"].reshape(n), np.cos(k * x))
    # damped oscillation: a(t + 1) = 2 r cos(w) a(t) - r^2 a(t - 1), r = exp(-Gamma)
    c1, c2 = np.linalg.lstsq(np.stack([a[1:-1], a[:-2]], 1), a[2:], rcond=None)[0]
    r = np.sqrt(-c2)
    gamma, omega = -np.log(r), np.arccos(c1 / (2 * r))
    zeta = 2.0 / 9.0 * (1.0 / 1.19 - 0.5)
    assert np.isclose(omega, k / np.sqrt(3.0), rtol=5e-3)
    assert np.isclose(gamma, 0.5 * k * k * (4.0 * nu0 / 3.0 + zeta), rtol=1e-2)


def test_shear_wave_advected_by_a_uniform_flow():
    """Galilean invariance: a shear wave u_y = A sin kx carried by a uniform
    flow U along x travels at U (phase -k U t) and decays at nu k^2, as in the
    frame moving with the flow.  The advection comes from the nonlinear
    momentum-flux equilibrium rho u_x u_y (Eq. meq_fm row 13): without it the
    wave would stand still.  64 x 1 x 1 box, U = 0.05, 1000 steps (4.9 rad of
    phase, 9 % decay)."""
    n, nu0, A, U, T = 64, 0.01, 1e-4, 0.05, 1000
    k = 2 * np.pi / n
    x = np.arange(n)
    L = oracle.OracleLBM(n, 1, 1, nu0, 0.0)
    u = np.zeros((3, 1, 1, n))
    u[0] = U
    u[1, 0, 0, :] = A * np.sin(k * x)
    L.init_equilibrium(u)

    def mode():
        return 2.0 / n * np.sum(L.fields()["u"][1].reshape(n) * np.exp(-1j * k * x))

    c0 = mode()
    L.step(T)
    c1 = mode()
    assert np.isclose(np.log(abs(c1) / abs(c0)), -nu0 * k * k * T, rtol=1e-2)
    dphi = np.angle(c1 / c0) + k * U * T
    assert abs((dphi + np.pi) % (2 * np.pi) - np.pi) <= 1e-3


def test_smagorinsky_kolmogorov_flow_closed_form():
    """Kolmogorov flow with the Smagorinsky closure (C = 0.1): in the steady
    state the momentum balance of Eqs. (eddy_visc), (les_viscosity) integrates
    once to (nu0 + C |u'|) u' = (F0 / k) cos(k y), whose root gives the strain
    |S| = |u'| cell by cell and theta = 3 (nu0 + C |S|).  Forcing chosen so that
    the eddy viscosity equals nu0 at the peak: the peak strain is half the
    C = 0 value, so a squared C, a missing eddy viscosity or a wrong |S|
    convention fails by tens of per cent.  Gates: 2 % (|S|), 1 % (theta)."""
    ny, nu0, C, smax = 16, 0.001, 0.1, 0.01
    k = 2 * np.pi / ny
    F0 = (nu0 + C * smax) * smax * k
    L = oracle.OracleLBM(1, ny, 1, nu0, C, oracle.FORCE_KOLMOGOROV, F0=F0)
    L.init_equilibrium(np.zeros((3, 1, ny, 1)))
    L.step(int(12 / ((nu0 + 0.5 * C * smax) * k * k)))
    fl = L.fields()
    c = (F0 / k) * np.cos(k * np.arange(ny))
    du = np.sign(c) * (np.sqrt(nu0 ** 2 + 4 * C * np.abs(c)) - nu0) / (2 * C)
    sn, th = fl["snorm"][0, :, 0], fl["theta"][0, :, 0]
    assert np.abs(sn - np.abs(du)).max() <= 0.02 * smax
    assert np.abs(th - 3 * (nu0 + C * np.abs(du))).max() <= 0.01 * th.max()
    assert np.isclose(np.abs(du).max(), 0.5 * F0 / (nu0 * k))


def test_taylor_green_3d_viscous_decay_converges():
    """The 3-D Taylor-Green field (u = u0 sin X cos Y cos Z, v = -u0 cos X sin Y
    cos Z, w = 0; all three wave-vector components nonzero, so every
    off-diagonal stress row of the moment basis takes part) at small amplitude
    decays at 3 nu k^2, the linear viscous rate.  The lattice rate converges to
    it at second order in k: the normalised error falls by ~4 from N = 16 to
    N = 32, and the Richardson extrapolation of the two is within 0.5 %.  A
    wrong rate on any stress row leaves an O(1) error instead."""
    nu0, u0 = 0.05, 1e-4
    err = {}
    for n in (16, 32):
        k = 2 * np.pi / n
        u = fields.tgv3d(n, n, n, u0)
        L = oracle.OracleLBM(n, n, n, nu0, 0.0)
        L.init_equilibrium(u)
        T = int(2.0 / (3 * nu0 * k * k))

        def amp():
            return float(np.sum(L.fields()["u"] * u) / np.sum(u * u))

        a0 = amp()
        L.step(T)
        err[n] = -np.log(amp() / a0) / T / (3 * nu0 * k * k) - 1.0
    assert abs(err[32]) < 0.02
    assert 3.0 < err[16] / err[32] < 5.0
    assert abs((4 * err[32] - err[16]) / 3) < 5e-3
