"""GPU parity of the stream + collide step against the FP64 oracle (C ABI).

FP32 storage: relative error of every full population f = f' + w at most
1e-5 (the per-population tolerance of the 32^3 Taylor-Green case).  FP16 and
BF16 storage: absolute error of f' at most n_steps x ulp(max |f'|) of the
storage format (one rounding of the stored value per step: the arithmetic is
FP32 and each step stores its result once in the storage type)."""
import numpy as np
import pytest

import oracle
import synthetic
from oracle import fields

from gpu_helpers import KINDS, LAYOUTS, fp32_mass_tolerance, full_f_rel_error, make_pair, random_populations, ulp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("steps", [100, 37])
def test_tgv3d_32_cubed_constant_force(gpu_lib, kind, steps, layout):
    """32^3 Taylor-Green, u0 = 0.05, rho = 1, nu0 = 0.01, C = 0.1, F = 1e-6 x."""
    lbm = gpu_lib
    n, F = 32, (1e-6, 0.0, 0.0)
    gpu, ref = make_pair(lbm, (n, n, n), nu0=0.01, C=0.1, force_mode=lbm.LBM_FORCE_CONST, body=F,
                         kind=kind, layout=layout)
    with gpu:
        assert gpu.config()["kind"] == kind
        assert gpu.config()["layout"] == layout
        gpu.init(lbm.LBM_INIT_TGV3D, amplitude=0.05)
        f0 = gpu.populations()
        gpu.step(steps)
        g = gpu.populations()
    ref.init_equilibrium(fields.tgv3d(n, n, n, 0.05))
    assert np.abs(f0 - ref.populations()).max() < 1e-8  # the GPU init kernel
    ref.step(steps)
    r = ref.populations()
    assert full_f_rel_error(g, r) <= 1e-5
    # mass conserved to FP32 round-off; momentum grows by ncell * F per step (Guo forcing)
    c, _ = oracle.lattice()
    assert abs(g.sum() - f0.sum()) <= fp32_mass_tolerance(n ** 3, steps, np.abs(f0).max())
    # FP32 storage rounds the injected 1e-6 per cell and step: the box momentum
    # follows n^3 F t to 1e-3 of the injection (the FP64 oracle to 1e-9)
    dj = c.T.astype(float) @ (g - f0).reshape(19, -1).sum(axis=1)
    want = np.array(F) * n ** 3 * steps
    assert np.abs(dj - want).max() <= 1e-3 * np.abs(want).max()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("shape", [(10, 12, 20), (7, 9, 33), (16, 16, 16)])
def test_random_les_field_paper_forcing(gpu_lib, kind, shape, layout):
    """Random solenoidal field (seeded generator), the paper's sinusoidal forcing,
    C = 0.13, LES viscosity; ragged sizes exercise padding and wrap."""
    lbm = gpu_lib
    nz, ny, nx = shape
    u = synthetic.random_solenoidal(nx, ny, nz, seed=7, urms=0.05)
    F0 = oracle.forcing_amplitude(0.2, 0.043, nx) * 50  # larger than the paper's, to be visible
    gpu, ref = make_pair(lbm, shape, nu0=2.15e-4 * 10, C=0.13, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                         F0=F0, kind=kind, layout=layout)
    with gpu:
        gpu.init(lbm.LBM_INIT_VELOCITY, u=u)
        gpu.step(51)
        g = gpu.populations()
        fl = gpu.fields()
    ref.init_equilibrium(u)
    ref.step(51)
    assert full_f_rel_error(g, ref.populations()) <= 1e-5
    fr = ref.fields()
    umax = np.abs(fr["u"]).max()
    assert np.abs(fl["u"] - fr["u"]).max() <= 1e-5 * umax
    assert np.abs(fl["theta"] - fr["theta"]).max() <= 1e-5 * fr["theta"].max()
    assert np.abs(fl["snorm"] - fr["snorm"]).max() <= 1e-4 * fr["snorm"].max() + 1e-9
    assert np.abs(fl["drho"] - fr["drho"]).max() <= 1e-6


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 3), (1, 4, 5), (3, 7, 1), (2, 3, 33)])
def test_degenerate_and_tiny_lattices(gpu_lib, kind, shape):
    """Extents of 1 (a link wraps onto its own cell), 2 (x - 1 = x + 1) and a
    ragged x; random near-equilibrium populations set through the ABI."""
    lbm = gpu_lib
    f = random_populations(shape, seed=11)
    gpu, ref = make_pair(lbm, shape, nu0=0.05, C=0.2, force_mode=lbm.LBM_FORCE_CONST,
                         body=(1e-5, -2e-5, 3e-5), kind=kind)
    with gpu:
        gpu.set_populations(f)
        assert np.array_equal(gpu.populations(), f.astype(np.float32).astype(np.float64))
        gpu.step(9)
        g = gpu.populations()
    ref.set_populations(f.astype(np.float32).astype(np.float64))
    ref.step(9)
    assert full_f_rel_error(g, ref.populations()) <= 1e-5


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("precision,mant", [(1, 10), (2, 7)])
def test_shifted_low_precision_storage(gpu_lib, kind, precision, mant):
    lbm = gpu_lib
    n, steps = 20, 12
    u = synthetic.random_solenoidal(n, seed=3, urms=0.05)
    gpu, ref = make_pair(lbm, (n, n, n), nu0=0.005, C=0.13, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                         F0=1e-4, kind=kind, precision=precision)
    ref.init_equilibrium(u)
    fmax = np.abs(ref.populations()).max()
    with gpu:
        gpu.init(lbm.LBM_INIT_VELOCITY, u=u)
        gpu.step(steps)
        g = gpu.populations()
    ref.step(steps)
    err = np.abs(g - ref.populations()).max()
    assert err <= (steps + 1) * ulp(fmax, mant), (err, ulp(fmax, mant))


@pytest.mark.parametrize("kind", KINDS)
def test_C_zero_is_constant_viscosity(gpu_lib, kind):
    """Sec. 2.3: C = 0 gives theta = 3 nu0 in every cell, bit for bit in FP32, and
    matches the oracle's fixed-rate MRT path."""
    lbm = gpu_lib
    n, nu0 = 12, 0.0123
    u = synthetic.random_solenoidal(n, seed=5)
    gpu, ref = make_pair(lbm, (n, n, n), nu0=nu0, C=0.0, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                         F0=1e-4, kind=kind)
    ref.set_fixed_rate(True)
    with gpu:
        gpu.init(lbm.LBM_INIT_VELOCITY, u=u)
        gpu.step(10)
        th = gpu.fields()["theta"]
        g = gpu.populations()
    assert np.all(th == float(np.float32(3.0) * np.float32(nu0)))
    ref.init_equilibrium(u)
    ref.step(10)
    assert full_f_rel_error(g, ref.populations()) <= 1e-5


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
def test_checkpoint_resume_bitwise(gpu_lib, kind, layout):
    """get_populations + set_time + set_populations resumes bit for bit, from an
    odd time (twisted AA layout) into a fresh handle."""
    lbm = gpu_lib
    shape = (8, 10, 12)
    u = synthetic.random_solenoidal(12, 10, 8, seed=9)
    gpu_a, _ = make_pair(lbm, shape, nu0=0.003, C=0.13, force_mode=lbm.LBM_FORCE_PAPER_SIN, F0=1e-4, kind=kind,
                         layout=layout)
    gpu_b, _ = make_pair(lbm, shape, nu0=0.003, C=0.13, force_mode=lbm.LBM_FORCE_PAPER_SIN, F0=1e-4, kind=kind,
                         layout=layout)
    with gpu_a, gpu_b:
        gpu_a.init(lbm.LBM_INIT_VELOCITY, u=u)
        gpu_a.step(13)
        snap = gpu_a.populations()
        gpu_b.init(lbm.LBM_INIT_REST)
        lbm.lbm_set_time(gpu_b.h, 13)
        gpu_b.set_populations(snap)
        assert np.array_equal(gpu_b.populations(), snap)
        gpu_a.step(10)
        gpu_b.step(10)
        assert gpu_a.time == gpu_b.time == 23
        assert np.array_equal(gpu_a.populations(), gpu_b.populations())
        # changing the parity of a live state keeps the canonical populations
        before = gpu_b.populations()
        lbm.lbm_set_time(gpu_b.h, 24)
        assert np.array_equal(gpu_b.populations(), before)


@pytest.mark.parametrize("kind", KINDS)
def test_graph_replay_equals_single_steps(gpu_lib, kind):
    lbm = gpu_lib
    shape = (12, 12, 12)
    u = synthetic.random_solenoidal(12, seed=2)
    a, _ = make_pair(lbm, shape, nu0=0.002, C=0.13, force_mode=lbm.LBM_FORCE_PAPER_SIN, F0=1e-4, kind=kind)
    b, _ = make_pair(lbm, shape, nu0=0.002, C=0.13, force_mode=lbm.LBM_FORCE_PAPER_SIN, F0=1e-4, kind=kind)
    with a, b:
        a.init(lbm.LBM_INIT_VELOCITY, u=u)
        b.init(lbm.LBM_INIT_VELOCITY, u=u)
        a.step(70)          # two captured 32-step graphs + 6 direct launches
        for _ in range(70):
            b.step(1)
        assert np.array_equal(a.populations(), b.populations())


def test_all_kernels_agree(gpu_lib):
    lbm = gpu_lib
    shape = (16, 24, 40)
    u = synthetic.random_solenoidal(40, 24, 16, seed=4)
    out = []
    for kind in KINDS:
        g, _ = make_pair(lbm, shape, nu0=0.001, C=0.13, force_mode=lbm.LBM_FORCE_PAPER_SIN, F0=1e-4, kind=kind)
        with g:
            g.init(lbm.LBM_INIT_VELOCITY, u=u)
            g.step(33)
            out.append(g.populations())
    for o in out[1:]:
        assert np.abs(out[0] - o).max() <= 1e-7


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("kind", KINDS)
def test_batch_of_uneven_instances(gpu_lib, kind, layout):
    """Three instances of different sizes and physics in one handle (one launch
    per step) match three separate oracle runs."""
    lbm = gpu_lib
    specs = [
        dict(shape=(16, 16, 16), nu0=0.002, C=0.13, fm=lbm.LBM_FORCE_PAPER_SIN, F0=1e-4, body=(0, 0, 0)),
        dict(shape=(8, 12, 20), nu0=0.01, C=0.0, fm=lbm.LBM_FORCE_CONST, F0=0.0, body=(1e-6, 0, 2e-6)),
        dict(shape=(5, 6, 7), nu0=0.03, C=0.2, fm=lbm.LBM_FORCE_NONE, F0=0.0, body=(0, 0, 0)),
    ]
    params, refs, inits = [], [], []
    for i, s in enumerate(specs):
        nz, ny, nx = s["shape"]
        params.append(lbm.make_params(nx, ny, nz, nu0=s["nu0"], cs=s["C"], f0=s["F0"], body_force=s["body"],
                                      force_mode=s["fm"], kernel=kind, layout=layout))
        refs.append(oracle.OracleLBM(nx, ny, nz, s["nu0"], s["C"],
                                     {0: 0, 1: 1, 2: 2, 3: 3}[s["fm"]], F0=s["F0"], body=s["body"]))
        inits.append(synthetic.random_solenoidal(nx, ny, nz, seed=20 + i))
    with lbm.Lattice(params) as g:
        for i in range(3):
            g.init(lbm.LBM_INIT_VELOCITY, u=inits[i], inst=i)
        g.step(21)
        for i in range(3):
            refs[i].init_equilibrium(inits[i])
            refs[i].step(21)
            assert full_f_rel_error(g.populations(inst=i), refs[i].populations()) <= 1e-5, i


@pytest.mark.parametrize("kind", KINDS)
def test_subnormal_strain_stays_finite(gpu_lib, kind):
    """A cell whose non-equilibrium stress is ~1e-20 (its strain norm squared is
    subnormal in FP32) must collide to finite values that match the oracle (a
    reciprocal square root of a subnormal once turned such cells into NaN)."""
    lbm = gpu_lib
    shape = (4, 4, 4)
    f = np.zeros((19, *shape))
    f[6, 1, 2, 3] = f[7, 1, 2, 3] = 5e-21
    f[8, 1, 2, 3] = f[9, 1, 2, 3] = -5e-21
    gpu, ref = make_pair(lbm, shape, nu0=0.002, C=0.13, kind=kind)
    with gpu:
        gpu.set_populations(f)
        gpu.step(3)
        g = gpu.populations()
        st = gpu.stats()
    assert np.all(np.isfinite(g)) and np.isfinite(st["theta_max"])
    ref.set_populations(f.astype(np.float32).astype(np.float64))
    ref.step(3)
    assert np.abs(g - ref.populations()).max() <= 1e-24


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("row_align", [256, 4096])
def test_padded_x_lines(gpu_lib, kind, row_align):
    """x-lines padded to a larger alignment (the TMA kernel then copies each
    line's live cells on their own) give the same populations as the oracle."""
    lbm = gpu_lib
    nz, ny, nx = 6, 9, 20
    u = synthetic.random_solenoidal(nx, ny, nz, seed=13)
    p = lbm.make_params(nx, ny, nz, nu0=0.003, cs=0.13, f0=1e-4, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                        kernel=kind, row_align=row_align)
    ref = oracle.OracleLBM(nx, ny, nz, 0.003, 0.13, oracle.FORCE_PAPER_SIN, F0=1e-4)
    with lbm.Lattice(p) as g:
        _, nbytes, nxp = lbm.lbm_device_ptr(g.h)
        assert nxp * 4 % row_align == 0 and nxp >= nx
        g.init(lbm.LBM_INIT_VELOCITY, u=u)
        g.step(15)
        got = g.populations()
    ref.init_equilibrium(u)
    ref.step(15)
    assert full_f_rel_error(got, ref.populations()) <= 1e-5


@pytest.mark.parametrize("kind", KINDS)
def test_selfconsistent_strain_mode(gpu_lib, kind):
    """strain_mode = 1 (local shear rate in Eq. yu_strain, solved per cell)
    matches the oracle's bisection solution; it differs from the explicit mode."""
    lbm = gpu_lib
    n = 16
    u = synthetic.random_solenoidal(n, seed=21, urms=0.05)
    F0 = 2e-5
    p1 = lbm.make_params(n, nu0=2.15e-4 * 4, cs=0.13, f0=F0, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                         kernel=kind, strain_mode=1)
    ref = oracle.OracleLBM(n, n, n, 2.15e-4 * 4, 0.13, oracle.FORCE_PAPER_SIN, F0=F0)
    ref.set_strain_mode(1)
    with lbm.Lattice(p1) as g:
        g.init(lbm.LBM_INIT_VELOCITY, u=u)
        g.step(25)
        got = g.populations()
        th = g.fields()["theta"]
    ref.init_equilibrium(u)
    ref.step(25)
    assert full_f_rel_error(got, ref.populations()) <= 1e-5
    fr = ref.fields()
    assert np.abs(th - fr["theta"]).max() <= 1e-5 * fr["theta"].max()
    expl = oracle.OracleLBM(n, n, n, 2.15e-4 * 4, 0.13, oracle.FORCE_PAPER_SIN, F0=F0)
    expl.init_equilibrium(u)
    expl.step(25)
    assert np.abs(expl.fields()["theta"] - fr["theta"]).max() > 1e-6


def test_initial_field_sources_agree(gpu_lib):
    """lbm_init_field from staged host memory (u_on_device = 0), device memory
    (1) and page-locked host memory read in place (2), and
    lbm_init_velocity_f32 from the FP32 rounding of the same field in each of
    the three places, give identical populations; mode 2 rejects memory that is
    not page-locked."""
    import ctypes

    import torch

    lbm = gpu_lib
    n = 24
    u = synthetic.random_solenoidal(n, seed=7, urms=0.05)
    u32 = u.astype(np.float32)
    sources = [u, torch.from_numpy(u).cuda(), torch.from_numpy(u).pin_memory(),
               u32, torch.from_numpy(u32).cuda(), torch.from_numpy(u32).pin_memory()]
    pops = []
    for src in sources:
        # one fixed kernel configuration: the comparison is bitwise, and two
        # kernels agree only to rounding
        p = lbm.make_params(n, nu0=0.002, cs=0.13, kernel=2, tile_rows=4, stages=2, threads=256)
        with lbm.Lattice(p) as L:
            L.init(lbm.LBM_INIT_VELOCITY, u=src)
            L.step(3)
            pops.append(L.populations())
    # the FP32 sources (lbm_init_velocity_f32) give exactly the FP64 ones' populations
    for p in pops[1:]:
        assert np.array_equal(pops[0], p)
    with lbm.Lattice(lbm.make_params(n, nu0=0.002, cs=0.13)) as L:
        pageable = np.ascontiguousarray(u)
        rc = lbm.load().lbm_init_field(L.h, 0, lbm.LBM_INIT_VELOCITY, 0.0,
                                       pageable.ctypes.data_as(ctypes.c_void_p), 2)
        assert rc == lbm.LBM_ERR_INVALID_ARG
        rc = lbm.load().lbm_init_field(L.h, 0, lbm.LBM_INIT_VELOCITY, 0.0,
                                       pageable.ctypes.data_as(ctypes.c_void_p), 3)
        assert rc == lbm.LBM_ERR_INVALID_ARG
        L.sync()


@pytest.mark.parametrize("precision", [0, 1])
def test_tma_shared_memory_layouts_agree(gpu_lib, precision):
    """The TMA kernel's shared-memory layouts (3840 B slots with 3 stages,
    5760 B slots with 2, the runtime stride rows x nxp with 4 stages, and the
    2880 B slots with 2 stages sized for two co-resident blocks per SM)
    compute every cell identically: bitwise-equal populations after 33 steps,
    including a ragged last tile (ny = 23 with 2 x-lines per tile)."""
    lbm = gpu_lib
    nx, ny, nz = 40, 23, 12
    u = synthetic.random_solenoidal(nx, ny, nz, seed=5)
    out = []
    for stages, slots, slot_bytes, bps in ((3, 0, 3840, 1), (2, 0, 5760, 1), (4, 0, 0, None), (2, 2, 2880, 2)):
        p = lbm.make_params(nx, ny, nz, precision=precision, nu0=0.002, cs=0.13, f0=1e-4,
                            force_mode=lbm.LBM_FORCE_PAPER_SIN, kernel=2, tile_rows=2, stages=stages,
                            threads=256, tma_slots=slots)
        with lbm.Lattice(p) as L:
            cfg = L.config()
            assert (cfg["kind"], cfg["tile_rows"], cfg["stages"], cfg["slot_bytes"]) == (2, 2, stages, slot_bytes)
            if bps is not None:
                assert cfg["blocks_per_sm"] == bps
            L.init(lbm.LBM_INIT_VELOCITY, u=u)
            L.step(33)
            out.append(L.populations())
    for o in out[1:]:
        assert np.array_equal(out[0], o)


@pytest.mark.parametrize("kind", KINDS)
def test_population_layouts_agree(gpu_lib, kind):
    """The population-major and row-interleaved arrays give bitwise-equal
    canonical populations and statistics (same kernel), through even and odd
    steps, statistics steps and a parity change.  For the TMA kernel the
    configurations cover compile-time slots (2 stages) and the runtime stride
    with one-x-line tiles (4 stages), where odd steps of the row-interleaved
    array copy each slot group of a cell row in one piece."""
    lbm = gpu_lib
    nx, ny, nz = 24, 10, 7
    u = synthetic.random_solenoidal(nx, ny, nz, seed=11)
    if kind == 2:
        cfgs = [dict(kernel=2, tile_rows=2, stages=2, threads=256), dict(kernel=2, tile_rows=1, stages=4, threads=256),
                dict(kernel=2, tile_rows=1, stages=3, threads=384),
                dict(kernel=2, tile_rows=1, stages=2, threads=256, tma_slots=1)]
    else:
        cfgs = [dict(kernel=1, tile_rows=1, threads=256)]
    out, st = [], []
    for cfg in cfgs:
        for layout in (1, 2):
            p = lbm.make_params(nx, ny, nz, nu0=0.002, cs=0.13, f0=1e-4, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                                stats_every=4, layout=layout, **cfg)
            with lbm.Lattice(p) as L:
                c = L.config()
                assert c["layout"] == layout and c["tile_rows"] == cfg["tile_rows"]
                if kind == 2:  # compile-time slots exactly where they apply
                    assert (c["slot_bytes"] == 0) == (cfg["stages"] == 4 or cfg.get("tma_slots", 0) == 1)
                L.init(lbm.LBM_INIT_VELOCITY, u=u)
                L.step(9)
                lbm.lbm_set_time(L.h, 10)
                L.step(3)
                out.append(L.populations())
                st.append(L.stats())
    for o in out[1:]:
        assert np.array_equal(out[0], o)
    for x in st[1:]:
        for k in ("E_k", "eps0", "eps_sgs", "theta_mean", "mass"):
            assert x[k] == st[0][k], k


def test_grouped_copies_across_uneven_instances(gpu_lib):
    """A batch of instances of different x-line lengths in the row-interleaved
    array with one-x-line tiles in the runtime stride (grouped odd-step copies):
    the producer's shared-memory regions change at every instance boundary.
    Each instance matches its own oracle run."""
    lbm = gpu_lib
    shapes = [(6, 8, 40), (9, 5, 12), (4, 7, 64)]
    params, refs, inits = [], [], []
    for i, (nz, ny, nx) in enumerate(shapes):
        params.append(lbm.make_params(nx, ny, nz, nu0=0.004, cs=0.13, f0=1e-4, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                                      kernel=2, tile_rows=1, stages=4, threads=256, layout=2))
        refs.append(oracle.OracleLBM(nx, ny, nz, 0.004, 0.13, oracle.FORCE_PAPER_SIN, F0=1e-4))
        inits.append(synthetic.random_solenoidal(nx, ny, nz, seed=30 + i))
    with lbm.Lattice(params) as g:
        assert g.config()["layout"] == 2
        for i in range(len(shapes)):
            g.init(lbm.LBM_INIT_VELOCITY, u=inits[i], inst=i)
        g.step(17)
        for i in range(len(shapes)):
            refs[i].init_equilibrium(inits[i])
            refs[i].step(17)
            assert full_f_rel_error(g.populations(inst=i), refs[i].populations()) <= 1e-5, i


@pytest.mark.parametrize("kind", KINDS)
def test_smagorinsky_kolmogorov_flow_closed_form(gpu_lib, kind):
    """The CUDA path against physics rather than the oracle: Kolmogorov flow
    with the Smagorinsky closure (C = 0.1) reaches the steady state of
    (nu0 + C |u'|) u' = (F0 / k) cos(k y), |S| = |u'| and theta =
    3 (nu0 + C |S|) cell by cell (the eddy viscosity halves the peak strain
    here).  Gates: 2 % (|S|), 1 % (theta), as for the oracle."""
    lbm = gpu_lib
    ny, nu0, C, smax = 16, 0.001, 0.1, 0.01
    k = 2 * np.pi / ny
    F0 = (nu0 + C * smax) * smax * k
    gpu, _ = make_pair(lbm, (1, ny, 1), nu0=nu0, C=C, force_mode=lbm.LBM_FORCE_KOLMOGOROV, F0=F0, kind=kind)
    with gpu:
        gpu.init(lbm.LBM_INIT_REST)
        gpu.step(int(12 / ((nu0 + 0.5 * C * smax) * k * k)))
        fl = gpu.fields()
    c = (F0 / k) * np.cos(k * np.arange(ny))
    du = np.sign(c) * (np.sqrt(nu0 ** 2 + 4 * C * np.abs(c)) - nu0) / (2 * C)
    sn, th = fl["snorm"][0, :, 0], fl["theta"][0, :, 0]
    assert np.abs(sn - np.abs(du)).max() <= 0.02 * smax
    assert np.abs(th - 3 * (nu0 + C * np.abs(du))).max() <= 0.01 * th.max()


@pytest.mark.parametrize("kind", KINDS)
def test_sound_wave_speed_and_bulk_viscosity(gpu_lib, kind):
    """The CUDA path against physics: a standing sound wave oscillates at
    c_s k (c_s^2 = 1/3) and decays at (k^2 / 2)(4 nu / 3 + zeta), zeta =
    (2/9)(1/s1 - 1/2), s1 = 1.19 (64 x 1 x 1 box, 2000 steps, Prony fit)."""
    lbm = gpu_lib
    n, nu0, A = 64, 0.01, 1e-5
    k = 2 * np.pi / n
    x = np.arange(n)
    gpu, ref = make_pair(lbm, (1, 1, n), nu0=nu0, C=0.0, kind=kind)
    ref.init_equilibrium(np.zeros((3, 1, 1, n)), (A * np.cos(k * x)).reshape(1, 1, n))
    T = 2000
    a = np.zeros(T + 1)
    with gpu:
        gpu.set_populations(ref.populations())
        for t in range(T + 1):
            if t:
                gpu.step(1)
            a[t] = 2.0 / n * np.dot(gpu.fields()["drho"].reshape(n), np.cos(k * x))
    c1, c2 = np.linalg.lstsq(np.stack([a[1:-1], a[:-2]], 1), a[2:], rcond=None)[0]
    r = np.sqrt(-c2)
    gamma, omega = -np.log(r), np.arccos(c1 / (2 * r))
    zeta = 2.0 / 9.0 * (1.0 / 1.19 - 0.5)
    assert np.isclose(omega, k / np.sqrt(3.0), rtol=5e-3)
    assert np.isclose(gamma, 0.5 * k * k * (4.0 * nu0 / 3.0 + zeta), rtol=1e-2)


@pytest.mark.parametrize("kind", KINDS)
def test_shear_wave_advected_by_a_uniform_flow(gpu_lib, kind):
    """The CUDA path against physics: a shear wave carried by a uniform flow
    U = 0.05 travels at U and decays at nu k^2 (64 x 1 x 1 box, 1000 steps)."""
    lbm = gpu_lib
    n, nu0, A, U, T = 64, 0.01, 1e-4, 0.05, 1000
    k = 2 * np.pi / n
    x = np.arange(n)
    u = np.zeros((3, 1, 1, n))
    u[0] = U
    u[1, 0, 0, :] = A * np.sin(k * x)
    gpu, _ = make_pair(lbm, (1, 1, n), nu0=nu0, C=0.0, kind=kind)
    with gpu:
        gpu.init(lbm.LBM_INIT_VELOCITY, u=u)
        c0 = 2.0 / n * np.sum(gpu.fields()["u"][1].reshape(n) * np.exp(-1j * k * x))
        gpu.step(T)
        c1 = 2.0 / n * np.sum(gpu.fields()["u"][1].reshape(n) * np.exp(-1j * k * x))
    assert np.isclose(np.log(abs(c1) / abs(c0)), -nu0 * k * k * T, rtol=1e-2)
    dphi = np.angle(c1 / c0) + k * U * T
    assert abs((dphi + np.pi) % (2 * np.pi) - np.pi) <= 1e-3
