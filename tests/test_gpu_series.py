"""The JSON-lines statistics time series (paper_2512_23116_gb300.series): one
record per interval with the library's statistics, spectrum and theta slice,
equal to what the entry points return for the same state."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_series_records_match_the_entry_points(gpu_lib, tmp_path):
    lbm = gpu_lib
    from paper_2512_23116_gb300 import series

    n = 24
    p = lbm.make_params(n, nu0=0.002, cs=0.13, f0=1e-5, force_mode=lbm.LBM_FORCE_PAPER_SIN)
    path = str(tmp_path / "run.jsonl")
    with lbm.Lattice(p) as L:
        L.init_random(seed=2, urms=0.04, k0=3.0)
        recs = series.run_with_statistics(L, 100, 40, path, theta_slice=(1, 5))
        st = L.stats(what=lbm.LBM_STATS_SPECTRUM | lbm.LBM_STATS_STRUCTURE)
        E = L.spectrum(len(recs[-1]["E"]) - 1)
        sl = L.theta_slice(1, 5)
    back = series.read_series(path)
    assert [r["step"] for r in back] == [40, 80, 100] == [r["step"] for r in recs]
    last = back[-1]
    for k in ("E_k", "inj", "eps0", "eps_sgs", "theta_mean", "theta_var", "theta_p95", "Kt_mean", "L", "eta"):
        assert last[k] == st[k], k
    assert np.array_equal(np.array(last["Sp"]), st["Sp"])
    assert np.array_equal(np.array(last["E"]), E)
    saved = np.load(os.path.join(tmp_path, last["theta_slice"]["file"]))
    assert np.array_equal(saved, sl)
