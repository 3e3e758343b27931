"""GPU parity of the fused diagnostics against the oracle: domain statistics,
theta histogram and percentiles, energy spectrum, structure functions and
flatness, derived scales, the in-step record series, theta slices, and the
non-finite detection (C ABI)."""
import math

import numpy as np
import pytest

import oracle
import synthetic
from oracle import diagnostics as dg

from gpu_helpers import KINDS, fp32_mass_tolerance, make_pair

pytestmark = pytest.mark.gpu


def _les_case(lbm, n=24, steps=30, kind=0, stats_every=0, hist_bins=4096, hist_max=0.02):
    u = synthetic.random_solenoidal(n, seed=1, urms=0.05)
    nu0 = oracle.derive_nu0(0.043, n, 2e3)
    F0 = oracle.forcing_amplitude(0.2, 0.043, n)
    gpu, ref = make_pair(lbm, (n, n, n), nu0=nu0, C=0.13, force_mode=lbm.LBM_FORCE_PAPER_SIN, F0=F0,
                         kind=kind, stats_every=stats_every, hist_bins=hist_bins, hist_max=hist_max)
    gpu.init(lbm.LBM_INIT_VELOCITY, u=u)
    ref.init_equilibrium(u)
    return gpu, ref, nu0


def test_domain_stats_match_oracle(gpu_lib):
    lbm = gpu_lib
    # this small, strongly sheared case reaches theta ~ 0.05: the histogram covers [0, 0.2)
    gpu, ref, nu0 = _les_case(lbm, hist_bins=16384, hist_max=0.2)
    with gpu:
        gpu.step(30)
        st = gpu.stats(what=lbm.LBM_STATS_SPECTRUM | lbm.LBM_STATS_STRUCTURE)
        E_gpu = gpu.spectrum(dg.max_shell(24, 24, 24))
    ref.step(30)
    fl = ref.fields()
    F = ref.force_field()
    want = dg.domain_stats(fl, F, nu0, 0.13, hist_bins=16384, hist_max=0.2)
    assert st["step"] == 30 and st["cells"] == 24 ** 3
    fmax = np.abs(ref.populations()).max()
    assert abs(st["mass"] - want["mass"]) <= fp32_mass_tolerance(24 ** 3, 30, fmax)
    for k in ("E_k", "eps0", "eps_sgs", "theta_mean", "theta_max", "theta_min", "Kt_mean"):
        assert math.isclose(st[k], want[k], rel_tol=2e-5), (k, st[k], want[k])
    assert math.isclose(st["inj"], want["inj"], rel_tol=1e-4, abs_tol=1e-12)
    for k in ("theta_var", "Kt_var"):
        assert math.isclose(st[k], want[k], rel_tol=1e-3), (k, st[k], want[k])
    assert np.allclose(st["uu"], want["uu"], rtol=2e-5, atol=1e-12)
    # total momentum is zero (sum F = 0); FP32 storage drifts by round-off at the
    # scale of FP32 precision times the summed magnitude sum |rho u|
    scale = float(np.sum(np.abs((1.0 + fl["drho"]) * fl["u"])))
    assert np.abs(np.array(st["momentum"]) - np.array(want["momentum"])).max() <= 2 ** -23 * scale
    # percentiles: centre of the bin holding the exact percentile (width 0.2/16384)
    width = 0.2 / 16384
    for p, key in ((5, "theta_p05"), (50, "theta_p50"), (95, "theta_p95"), (99, "theta_p99")):
        assert abs(st[key] - want["theta_p"][p]) <= width, (key, st[key], want["theta_p"][p])
    # spectrum and derived scales
    E_ref = dg.spectrum(fl["u"])
    big = E_ref > 1e-10 * E_ref.max()
    assert np.allclose(E_gpu[big], E_ref[big], rtol=1e-4)
    assert np.all(np.abs(E_gpu[~big] - E_ref[~big]) <= 1e-9 * E_ref.max())
    d = dg.derived_scales(E_ref, 24, nu0, want["E_k"])
    for k, kk in (("L", "L"), ("eps_spec", "eps"), ("eta", "eta"), ("lambda", "lambda"),
                  ("u_rms", "u_rms"), ("Re_lambda", "Re_lambda")):
        assert math.isclose(st[k], d[kk], rel_tol=1e-4), (k, st[k], d[kk])
    # structure functions and flatness
    sf = dg.structure_functions(fl["u"])
    assert st["r"] == sf["r"]
    for p in (2, 4, 6):
        assert np.allclose(st["Sp"][:, p - 1], sf["S"][:, p], rtol=1e-4)
    assert np.allclose(st["F4"], sf["F4"], rtol=1e-4)
    assert np.all(np.abs(st["Sp"][:, 0]) < 1e-9)  # S1 = 0 on a periodic box
    # isotropy (Sec. 3.2) from the fused <u_i u_j>
    iso = dg.isotropy(fl["u"])
    assert np.allclose(st["E_frac"], iso["E_frac"], rtol=2e-5)
    assert np.allclose(st["b"], iso["b"], atol=2e-6)
    for k, kk in (("II_b", "II_b"), ("III_b", "III_b"), ("lumley_xi", "xi"), ("lumley_eta", "eta")):
        assert math.isclose(st[k], iso[kk], rel_tol=1e-3, abs_tol=1e-7), (k, st[k], iso[kk])


# (kernel configuration, bins): the statistics pass of the direct kernel keeps
# up to 12000 bins in shared memory, global counts above; the TMA kernel's
# keeps a window of bins from that of theta = 3 nu0 up in shared memory behind
# its stages, as many as fit (runtime-stride tiles of two 16-cell x-lines,
# 2.4 KB stages: all of 4096, ~55,000 of 60,000; 5760 B slots, 214 KB of
# stages: ~2000) and counts the rest in global memory, summed over the warp's
# lanes that flush the same bin
HIST_PATHS = [
    (dict(kernel=1, tile_rows=2, threads=256), 4096),
    (dict(kernel=1, tile_rows=2, threads=256), 20000),
    (dict(kernel=2, tile_rows=2, stages=2, threads=256, tma_slots=1), 4096),
    (dict(kernel=2, tile_rows=2, stages=2, threads=256), 4096),
    (dict(kernel=2, tile_rows=2, stages=2, threads=256, tma_slots=1), 60000),
]


@pytest.mark.parametrize("steps", [10, 11])
@pytest.mark.parametrize("cfg,bins", HIST_PATHS)
def test_histogram_counts(gpu_lib, cfg, bins, steps):
    """Every histogram path of the statistics pass, at both AA parities: the
    counts are exactly those of the pass's own per-cell theta (a per-thread
    run of cells in one bin is added when the bin changes, so no cell may be
    lost or counted twice)."""
    lbm = gpu_lib
    n = 16
    u = synthetic.random_solenoidal(n, seed=1, urms=0.05)
    nu0 = oracle.derive_nu0(0.043, n, 2e3)
    F0 = oracle.forcing_amplitude(0.2, 0.043, n)
    p = lbm.make_params(n, nu0=nu0, cs=0.13, f0=F0, force_mode=lbm.LBM_FORCE_PAPER_SIN, hist_bins=bins,
                        hist_max=0.02, **cfg)
    with lbm.Lattice(p) as L:
        assert L.config()["kind"] == cfg["kernel"]
        L.init(lbm.LBM_INIT_VELOCITY, u=u)
        L.step(steps)
        L.stats()
        h = lbm.lbm_histogram(L.h, 0, bins)
        th = L.fields()["theta"]
    assert int(h.sum()) == n ** 3
    # bin = floor(theta * bins / hist_max) in FP32; theta >= hist_max -> overflow bin
    q = th.astype(np.float32) * np.float32(bins / 0.02)
    idx = np.where(q < bins, np.floor(q), bins).astype(np.int64)
    want = np.bincount(idx.ravel(), minlength=bins + 1)
    assert np.array_equal(h, want)
    assert np.count_nonzero(h[:bins]) > 10  # theta spread over many bins


@pytest.mark.parametrize("bins,hist_max", [(4096, 0.01), (4096, 0.02), (16384, 0.04)])
def test_histogram_split_between_shared_and_global_counts(gpu_lib, bins, hist_max):
    """TMA statistics pass with 5760 B slots: the shared memory left behind
    the 214 KB of stages holds a window of about 2000 bins from the bin of
    theta = 3 nu0 up; the cells of this strongly sheared 16^3 LES (theta from
    3 nu0 = 1.03e-3 to a few 1e-2) spread over more bins than that, so they
    are counted on both sides of the window's end (and in the overflow bin),
    and the counts are still exactly those of the pass's own per-cell theta."""
    lbm = gpu_lib
    n = 16
    u = synthetic.random_solenoidal(n, seed=1, urms=0.05)
    nu0 = oracle.derive_nu0(0.043, n, 2e3)
    F0 = oracle.forcing_amplitude(0.2, 0.043, n)
    p = lbm.make_params(n, nu0=nu0, cs=0.13, f0=F0, force_mode=lbm.LBM_FORCE_PAPER_SIN, hist_bins=bins,
                        hist_max=hist_max, kernel=2, tile_rows=2, stages=2, threads=256)
    with lbm.Lattice(p) as L:
        assert L.config()["slot_bytes"] == 5760
        L.init(lbm.LBM_INIT_VELOCITY, u=u)
        L.step(10)
        L.stats()
        h = lbm.lbm_histogram(L.h, 0, bins)
        th = L.fields()["theta"]
    q = th.astype(np.float32) * np.float32(bins / hist_max)
    idx = np.where(q < bins, np.floor(q), bins).astype(np.int64)
    want = np.bincount(idx.ravel(), minlength=bins + 1)
    used = np.nonzero(want)[0]
    # no window of the shared memory left behind these stages (8 KB) spans it
    assert used[-1] - used[0] > 8256 // 4, (used[0], used[-1])
    assert int(h.sum()) == n ** 3
    assert np.array_equal(h, want)


def test_spectrum_single_mode(gpu_lib):
    """u_x = A cos(2 pi (x + 2y + 2z)/N): the whole energy A^2/4 in shell 3."""
    lbm = gpu_lib
    n, A = 12, 0.04
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = A * np.cos(2 * np.pi * (x + 2 * y + 2 * z) / n)
    gpu, _ = make_pair(lbm, (n, n, n), nu0=0.01, C=0.0)
    with gpu:
        gpu.init(lbm.LBM_INIT_VELOCITY, u=u)
        E = gpu.spectrum(dg.max_shell(n, n, n))
    assert math.isclose(E[3], A * A / 4, rel_tol=1e-6)
    assert np.abs(np.delete(E, 3)).max() < 1e-12 * A * A


def test_odd_sizes_spectrum_parseval(gpu_lib):
    lbm = gpu_lib
    shape = (9, 10, 11)
    u = synthetic.random_solenoidal(11, 10, 9, seed=2)
    gpu, _ = make_pair(lbm, shape, nu0=0.01, C=0.0)
    with gpu:
        gpu.init(lbm.LBM_INIT_VELOCITY, u=u)
        kmax = dg.max_shell(11, 10, 9)
        E = gpu.spectrum(kmax)
        st = gpu.stats()
    assert np.allclose(E, dg.spectrum(u, kmax), rtol=1e-4, atol=1e-12)
    assert math.isclose(E.sum(), st["E_k"], rel_tol=1e-5)


@pytest.mark.parametrize("kind", KINDS)
def test_series_records(gpu_lib, kind):
    """Statistics fused into the step (every 5 steps) match the oracle's fields
    for every step kernel."""
    lbm = gpu_lib
    gpu, ref, nu0 = _les_case(lbm, n=16, stats_every=5, kind=kind)
    with gpu:
        gpu.step(20)
        recs = gpu.series()
        again = gpu.series()
    assert [r["step"] for r in recs] == [0, 5, 10, 15]
    assert again == []
    F = ref.force_field()
    for r in recs:
        while ref.time < r["step"]:
            ref.step(1)
        want = dg.domain_stats(ref.fields(), F, nu0, 0.13)
        for k in ("E_k", "theta_mean", "theta_max", "theta_min"):
            assert math.isclose(r[k], want[k], rel_tol=2e-5), (r["step"], k)
        # eps at t = 0 is the strain of the half-force shift alone (~1e-14): FP32
        # cancellation in m - m^eq bounds |S| to ~1e-9 absolute
        for k in ("eps0", "eps_sgs"):
            assert math.isclose(r[k], want[k], rel_tol=2e-4, abs_tol=1e-12), (r["step"], k)
        fmax = np.abs(ref.populations()).max()
        assert abs(r["mass"] - want["mass"]) <= fp32_mass_tolerance(16 ** 3, r["step"], fmax)


def test_series_batched_instances(gpu_lib):
    """In-step records of a two-instance handle are kept per instance."""
    lbm = gpu_lib
    p1 = lbm.make_params(12, nu0=0.01, cs=0.13, stats_every=4)
    p2 = lbm.make_params(8, 6, 10, nu0=0.02, cs=0.0, stats_every=4)
    with lbm.Lattice([p1, p2]) as g:
        g.init(lbm.LBM_INIT_TGV3D, amplitude=0.05, inst=0)
        g.init(lbm.LBM_INIT_TGV3D, amplitude=0.02, inst=1)
        g.step(9)
        r0 = g.series(inst=0)
        r1 = g.series(inst=1)
    assert [r["step"] for r in r0] == [0, 4, 8] == [r["step"] for r in r1]
    assert math.isclose(r0[0]["E_k"], 0.05 ** 2 / 8, rel_tol=1e-5)
    assert math.isclose(r1[0]["E_k"], 0.02 ** 2 / 8, rel_tol=1e-5)
    assert math.isclose(r1[0]["theta_mean"], 3 * 0.02, rel_tol=1e-6)


@pytest.mark.parametrize("kind", KINDS)
def test_theta_slice(gpu_lib, kind):
    """Slices on every axis equal the read-only pass's theta field, bit for
    bit; a z-plane is computed from that plane's tiles alone."""
    lbm = gpu_lib
    gpu, _, _ = _les_case(lbm, n=16, kind=kind)
    with gpu:
        gpu.step(6)
        th = gpu.fields()["theta"]
        for axis, idx in ((0, 3), (1, 0), (2, 15), (2, 0), (2, 7)):
            s = gpu.theta_slice(axis, idx)
            want = {0: th[:, :, idx], 1: th[:, idx, :], 2: th[idx]}[axis]
            assert np.array_equal(s, want), (axis, idx)


def test_theta_slice_of_a_later_instance(gpu_lib):
    """z-plane slices of the second and third instances of a batched handle
    (whose tiles start after the first instance's) and an x-plane, against
    each instance's theta field; tiles of 3 x-lines, so a plane's last tile
    is ragged."""
    lbm = gpu_lib
    shapes = [(6, 10, 12), (9, 7, 20), (5, 11, 16)]  # (nz, ny, nx)
    params = [lbm.make_params(nx, ny, nz, nu0=0.01, cs=0.13, kernel=2, tile_rows=3, stages=2, threads=256)
              for (nz, ny, nx) in shapes]
    with lbm.Lattice(params) as g:
        for i in range(3):
            g.init(lbm.LBM_INIT_TGV3D, amplitude=0.04 + 0.01 * i, inst=i)
        g.step(5)
        for i in (1, 2):
            th = g.fields(inst=i)["theta"]
            nz = shapes[i][0]
            for idx in (0, nz // 2, nz - 1):
                assert np.array_equal(g.theta_slice(2, idx, inst=i), th[idx]), (i, idx)
            assert np.array_equal(g.theta_slice(0, 5, inst=i), th[:, :, 5]), i


def test_nonfinite_state_is_reported_and_recoverable(gpu_lib):
    """Host-side fault injection: a NaN in the initial velocity surfaces as
    LBM_ERR_UNSTABLE at the next statistics call; the handle stays usable."""
    lbm = gpu_lib
    n = 8
    u = np.zeros((3, n, n, n))
    u[0, 2, 3, 4] = np.nan
    gpu, _ = make_pair(lbm, (n, n, n), nu0=0.01, C=0.1)
    with gpu:
        gpu.init(lbm.LBM_INIT_VELOCITY, u=u)
        gpu.step(2)
        with pytest.raises(lbm.LbmError) as ei:
            gpu.stats()
        assert ei.value.code == lbm.LBM_ERR_UNSTABLE
        gpu.init(lbm.LBM_INIT_TGV3D, amplitude=0.01)
        gpu.step(2)
        st = gpu.stats()
        assert st["cells"] == n ** 3 and math.isfinite(st["E_k"])


def test_invalid_calls_on_a_live_handle(gpu_lib):
    lbm = gpu_lib
    gpu, _ = make_pair(lbm, (4, 4, 4), nu0=0.01, C=0.0)
    with gpu:
        for fn in (lambda: lbm.lbm_step(gpu.h, -1),
                   lambda: lbm.lbm_init_field(gpu.h, 5, lbm.LBM_INIT_REST),
                   lambda: lbm.lbm_init_field(gpu.h, 0, 42),
                   lambda: lbm.lbm_get_theta_slice(gpu.h, 0, 3, 0, (4, 4, 4)),
                   lambda: lbm.lbm_spectrum(gpu.h, 0, -1)):
            with pytest.raises(lbm.LbmError) as ei:
                fn()
            assert ei.value.code == lbm.LBM_ERR_INVALID_ARG
        gpu.step(1)
        gpu.sync()
    # the two-block slot layout needs two stages whose tile rows fit its slots
    p = lbm.make_params(64, nu0=0.01, kernel=2, tile_rows=2, stages=3, threads=256, tma_slots=2)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(p)
    assert ei.value.code == lbm.LBM_ERR_UNSUPPORTED and "tma_slots" in str(ei.value)


def test_energy_balance_series_matches_oracle(gpu_lib):
    """Residual of Eq. (energy_balance) along the fused in-step records of a
    forced LES run (stats every 20 steps), against the same residual from the
    oracle's states."""
    lbm = gpu_lib
    n = 24
    gpu, ref, nu0 = _les_case(lbm, n=n, stats_every=20)
    with gpu:
        gpu.step(200)
        recs = gpu.series()
    assert [r["step"] for r in recs] == list(range(0, 200, 20))
    at, res = lbm.lbm_energy_balance(recs)
    F = ref.force_field()
    E, inj, eps, times = [], [], [], []
    for t in range(0, 200, 20):
        while ref.time < t:
            ref.step(1)
        d = dg.domain_stats(ref.fields(), F, nu0, 0.13)
        times.append(t)
        E.append(d["E_k"])
        inj.append(d["inj"])
        eps.append(d["eps0"] + d["eps_sgs"])
    t_ref, r_ref = dg.energy_balance(times, E, inj, eps)
    assert list(at) == list(t_ref)
    assert np.allclose(res, r_ref, atol=1e-4), (res, r_ref)


def test_batch_entry_points_and_velocity(gpu_lib):
    """The ensemble entry points equal the functions they stand for:
    lbm_batch_stats gives each instance's lbm_stats, lbm_get_velocity the u of
    lbm_get_fields (same read-only pass, bit for bit)."""
    lbm = gpu_lib
    shapes = [(8, 8, 8), (6, 10, 12)]
    h = lbm.lbm_batch_create([lbm.make_params(nx, ny, nz, nu0=0.01, cs=0.1) for (nz, ny, nx) in shapes])
    try:
        for i in range(len(shapes)):
            lbm.lbm_init_field(h, i, lbm.LBM_INIT_TGV3D, 0.05)
        lbm.lbm_batch_step(h, 5)
        st = lbm.lbm_batch_stats(h, len(shapes))
        for i, shape in enumerate(shapes):
            one = lbm.lbm_stats(h, i)
            assert st[i]["step"] == 5 and st[i]["cells"] == int(np.prod(shape))
            for k in ("E_k", "eps0", "eps_sgs", "theta_mean", "mass"):
                assert st[i][k] == one[k], k
            u = lbm.lbm_get_velocity(h, i, shape)
            assert np.array_equal(u, lbm.lbm_get_fields(h, i, shape)["u"])
            assert np.abs(u).max() > 0.01
    finally:
        lbm.lbm_destroy(h)


def test_series_many_instances_match_single_handles(gpu_lib):
    """In-step records of a 16-instance handle (320 reduced values, so the
    reduction spans many blocks, replayed from captured graphs): one record per
    statistics step for every instance, each equal to the record of the same
    instance advanced in a handle of its own."""
    lbm = gpu_lib
    shapes = [(8 + (i % 4) * 2, 6 + (i % 3) * 4, 10 + (i % 5)) for i in range(16)]
    params = [lbm.make_params(nx, ny, nz, nu0=0.01 + 0.001 * i, cs=0.13 if i % 2 else 0.0, stats_every=3)
              for i, (nz, ny, nx) in enumerate(shapes)]
    amps = [0.01 + 0.002 * i for i in range(16)]
    steps = 70
    with lbm.Lattice(params) as g:
        for i, a in enumerate(amps):
            g.init(lbm.LBM_INIT_TGV3D, amplitude=a, inst=i)
        g.step(steps)
        batch = [g.series(inst=i) for i in range(16)]
    want_steps = list(range(0, steps, 3))
    for i in (0, 5, 10, 15):
        with lbm.Lattice(params[i]) as one:
            one.init(lbm.LBM_INIT_TGV3D, amplitude=amps[i])
            one.step(steps)
            single = one.series()
        assert [r["step"] for r in single] == want_steps
        for rb, rs in zip(batch[i], single):
            for k in ("E_k", "eps0", "theta_mean", "theta_max", "theta_min"):
                assert math.isclose(rb[k], rs[k], rel_tol=1e-6, abs_tol=1e-30), (i, rb["step"], k)
    for i in range(16):
        assert [r["step"] for r in batch[i]] == want_steps, i
        assert math.isclose(batch[i][0]["E_k"], amps[i] ** 2 / 8, rel_tol=1e-5), i
