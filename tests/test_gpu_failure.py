"""Failure detection on the GPU without a fault: a device-side wait that runs out.

The test hook makes block 0 of the next TMA step launch skip the loads of its
first tile, so nothing ever completes the barrier its consumers wait on (a flag
that nothing sets).  The bounded wait (0.2 s here) must run out, the kernel
must record LBM_ERR_TIMEOUT, drain and return, and the handle must stay
usable: after re-initialisation the next steps match the oracle again."""
import time

import numpy as np
import pytest

import oracle
from oracle import fields

from gpu_helpers import full_f_rel_error

pytestmark = pytest.mark.gpu


def test_device_wait_timeout_is_reported_and_recoverable(gpu_lib):
    lbm = gpu_lib
    n = 48
    p = lbm.make_params(n, nu0=0.01, cs=0.1, kernel=2, tile_rows=1, stages=2, threads=256)
    with lbm.Lattice(p) as L:
        assert L.config()["kind"] == 2
        L.init(lbm.LBM_INIT_TGV3D, amplitude=0.05)
        lbm.lbm_debug_withhold_load(L.h, 0.2)
        t0 = time.time()
        L.step(1)
        with pytest.raises(lbm.LbmError) as ei:
            L.sync()
        elapsed = time.time() - t0
        assert ei.value.code == lbm.LBM_ERR_TIMEOUT
        assert elapsed < 5.0
        L.sync()  # the error word was cleared
        L.init(lbm.LBM_INIT_TGV3D, amplitude=0.05)
        L.step(6)
        g = L.populations()
    ref = oracle.OracleLBM(n, n, n, 0.01, 0.1)
    ref.init_equilibrium(fields.tgv3d(n, n, n, 0.05))
    ref.step(6)
    assert full_f_rel_error(g, ref.populations()) <= 1e-5


def test_debug_hook_arguments(gpu_lib):
    lbm = gpu_lib
    with lbm.Lattice(lbm.make_params(8, nu0=0.01, kernel=1, tile_rows=1, threads=256)) as L:
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_debug_withhold_load(L.h, 0.2)
        assert ei.value.code == lbm.LBM_ERR_UNSUPPORTED
    with lbm.Lattice(lbm.make_params(8, nu0=0.01, kernel=2, tile_rows=1, stages=2, threads=256)) as L:
        for bad in (0.0, -1.0, 11.0):
            with pytest.raises(lbm.LbmError) as ei:
                lbm.lbm_debug_withhold_load(L.h, bad)
            assert ei.value.code == lbm.LBM_ERR_INVALID_ARG


def test_allocation_failure_is_reported_not_raised(gpu_lib):
    """A lattice larger than the device (8192 x 8192 x 128 cells need 653 GB of
    FP32 populations) fails to allocate: lbm_create returns LBM_ERR_OOM with
    the size in the text, releases what it had allocated, and the next handle
    works (a real allocation failure, no test hook needed)."""
    lbm = gpu_lib
    p = lbm.make_params(8192, 8192, 128, nu0=0.01)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(p)
    assert ei.value.code == lbm.LBM_ERR_OOM
    assert "population array" in str(ei.value)
    with lbm.Lattice(lbm.make_params(16, nu0=0.01)) as L:
        L.init(lbm.LBM_INIT_TGV3D, amplitude=0.05)
        L.step(4)
        L.sync()
        assert np.isfinite(L.populations()).all()
