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
