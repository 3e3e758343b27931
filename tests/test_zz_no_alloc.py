"""The allocation-free structure-function entry point.

Some callers cannot call cudaMalloc: code that shares the GPU with a framework
whose pool allocator owns the device memory, or pipelines that must not pay
the implicit device synchronisation of cudaMalloc / cudaFree.  For them
lbm_structure_functions_noalloc works on a velocity field and an output buffer
the caller already owns and keeps its partial sums in a fixed device array.
This test checks it, through the C ABI, against the structure functions of
lbm_stats on the same field, on two calls in a row, and that the calls after
the first do not change the free device memory.  The file is named to be
collected last."""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


def test_noalloc_structure_functions_match_lbm_stats(gpu_lib):
    import torch

    lbm = gpu_lib
    n = 20
    u0 = synthetic.random_solenoidal(n, seed=12, urms=0.05)
    p = lbm.make_params(n, nu0=0.002, cs=0.13, f0=1e-4, force_mode=lbm.LBM_FORCE_PAPER_SIN)
    with lbm.Lattice(p) as L:
        L.init(lbm.LBM_INIT_VELOCITY, u=u0)
        L.step(11)
        st = L.stats(what=lbm.LBM_STATS_STRUCTURE)
        u = L.fields()["u"]  # the library's FP32 velocity, exactly, as float64
    r = st["r"]
    ref = st["Sp"]
    dev = torch.device("cuda", 0)
    ut = torch.from_numpy(u.astype(np.float32)).to(dev)
    stream = torch.cuda.Stream(device=dev)
    for call in range(2):
        sp = torch.full((len(r) * 6,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        lbm.lbm_structure_functions_noalloc(ut, r, sp, stream=stream)
        stream.synchronize()
        free_after = torch.cuda.mem_get_info(dev)[0]
        got = sp.cpu().numpy().reshape(len(r), 6)
        # the same tolerance as the structure-function parity tests
        assert np.allclose(got[:, 1:], ref[:, 1:], rtol=1e-4), call
        assert np.all(np.abs(got[:, 0]) < 1e-9), call  # S1 = 0 on a periodic box
        if call == 1:
            assert free_after == free_before  # no device allocation once set up


def test_noalloc_rejects_sizes_beyond_the_limit(gpu_lib):
    import torch

    lbm = gpu_lib
    dev = torch.device("cuda", 0)
    u = torch.zeros((3, 4, 4, 4), dtype=torch.float32, device=dev)
    sp = torch.zeros(25 * 6, dtype=torch.float64, device=dev)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_structure_functions_noalloc(u, list(range(1, 26)), sp)
    assert ei.value.code == lbm.LBM_ERR_INVALID_ARG and "24" in str(ei.value)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_structure_functions_noalloc(u, [1, 0], sp)
    assert ei.value.code == lbm.LBM_ERR_INVALID_ARG


def _structure_functions_numpy(u, r):
    """S_p(r), p = 1..6: the mean over cells and the three axes of the
    longitudinal increment u_a(x + r e_a) - u_a(x) to the power p, periodic
    wrap, in FP64 (the definition written out with np.roll)."""
    out = np.zeros((len(r), 6))
    for k, rk in enumerate(r):
        # component a of u is (nz, ny, nx): its axis a (x, y, z) is array axis 2 - a
        d = [np.roll(u[a], -rk, axis=2 - a) - u[a] for a in range(3)]
        for p in range(1, 7):
            out[k, p - 1] = np.mean([np.mean(da ** p) for da in d])
    return out


def test_noalloc_non_cubic_field_and_long_separations(gpu_lib):
    """A 24 x 20 x 16 field with separations beyond one or more extents (the
    periodic wrap r mod n per axis) against the definition in numpy."""
    import torch

    lbm = gpu_lib
    rng = np.random.default_rng(5)
    nx, ny, nz = 24, 20, 16
    u = rng.normal(scale=0.05, size=(3, nz, ny, nx)).astype(np.float32)
    r = [1, 3, 17, 21, 30]
    want = _structure_functions_numpy(u.astype(np.float64), r)
    dev = torch.device("cuda", 0)
    ut = torch.from_numpy(u).to(dev)
    for call in range(2):
        sp = torch.full((len(r) * 6,), float("nan"), dtype=torch.float64, device=dev)
        lbm.lbm_structure_functions_noalloc(ut, r, sp)
        torch.cuda.synchronize()
        got = sp.cpu().numpy().reshape(len(r), 6)
        assert np.allclose(got[:, 1:], want[:, 1:], rtol=1e-9, atol=0.0), call
        assert np.allclose(got[:, 0], want[:, 0], rtol=0.0, atol=1e-12), call


def test_noalloc_rejects_host_buffers_before_any_launch(gpu_lib):
    """The C entry point given host memory for the velocity or for the output
    returns INVALID_ARG (a kernel given a host pointer would fault)."""
    import ctypes

    import torch

    lbm = gpu_lib
    lib = lbm.load()
    n = 4
    r = (ctypes.c_int32 * 1)(1)
    u_host = np.zeros((3, n, n, n), dtype=np.float32)
    sp_host = np.zeros(6, dtype=np.float64)
    dev = torch.device("cuda", 0)
    u_dev = torch.zeros((3, n, n, n), dtype=torch.float32, device=dev)
    sp_dev = torch.zeros(6, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    vp = ctypes.c_void_p
    cases = [(u_host.ctypes.data, sp_dev.data_ptr()), (u_dev.data_ptr(), sp_host.ctypes.data)]
    for up, spp in cases:
        rc = lib.lbm_structure_functions_noalloc(vp(up), n, n, n, r, 1, vp(spp), None)
        assert rc == lbm.LBM_ERR_INVALID_ARG
        assert "device memory" in lbm.lbm_last_error(None)
