"""The library's on-device seeded random field (lbm_init_random_spectrum)
against the host-side input generator of the test suite (synthetic/, numpy
FP64, separable DFT synthesis), which follows the same recipe: the FP32
velocity the library builds the equilibrium from equals the FP64 host field
to within 1e-6 of u_rms (FP32 rounding is 2e-7 of it), for a cube and a
non-cubic box with another k0, seed and u_rms; the populations equal those of
initialising from the host field; the same seed gives the same field bit for
bit; invalid arguments are rejected."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,seed,urms,k0", [((64, 64, 64), 1, 0.05, 4.0), ((40, 36, 32), 7, 0.02, 3.0)])
def test_device_random_field_matches_host_generator(gpu_lib, shape, seed, urms, k0):
    lbm = gpu_lib
    nx, ny, nz = shape
    want = synthetic.random_solenoidal(nx, ny, nz, seed=seed, k0=k0, urms=urms)
    p = lbm.make_params(nx, ny, nz, nu0=0.01, cs=0.1)
    u32 = np.zeros((3, nz, ny, nx), dtype=np.float32)
    with lbm.Lattice(p) as L:
        L.init_random(seed=seed, urms=urms, k0=k0, u_out=u32)
        f_dev = L.populations()
        L.init(lbm.LBM_INIT_VELOCITY, u=want)
        f_host = L.populations()
        again = np.zeros_like(u32)
        L.init_random(seed=seed, urms=urms, k0=k0, u_out=again)
    err = np.abs(u32.astype(np.float64) - want).max()
    assert err <= 1e-6 * urms, err
    assert np.array_equal(u32, again)
    # the equilibrium is built from the FP32 velocity either way: equal up to
    # the rare cell whose FP32 rounding differs
    assert np.abs(f_dev - f_host).max() <= 1e-7


def test_device_random_field_rejects_bad_arguments(gpu_lib):
    lbm = gpu_lib
    with lbm.Lattice(lbm.make_params(8, nu0=0.01)) as L:
        for kw in (dict(urms=0.0), dict(urms=float("nan")), dict(k0=-1.0)):
            with pytest.raises(lbm.LbmError) as ei:
                L.init_random(**kw)
            assert ei.value.code == lbm.LBM_ERR_INVALID_ARG
    with lbm.Lattice(lbm.make_params(8, 8, 2, nu0=0.01)) as L:
        with pytest.raises(lbm.LbmError) as ei:
            L.init_random()
        assert ei.value.code == lbm.LBM_ERR_INVALID_ARG
