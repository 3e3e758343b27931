"""The C-ABI library without a GPU: it loads, exports every entry point that
include/lbm.h declares, the ctypes structures match the C layout, and the
host-side argument validation answers before any device call."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    import paper_2512_23116_gb300 as lbm
    from paper_2512_23116_gb300 import _build
    _build.build()
    return lbm


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for core in ("lbm_create", "lbm_init_field", "lbm_step", "lbm_stats", "lbm_spectrum",
                 "lbm_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    so = ctypes.CDLL(lib.library_path())
    for name in _declared():
        assert hasattr(so, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(_declared())
    assert set(lib.EXPORTED) == set(_declared())


def test_struct_layout_matches_c(lib):
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "lbm.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(lbm_params), sizeof(lbm_stats_t), sizeof(lbm_record_t));
  printf("%zu %zu %zu %zu\n", offsetof(lbm_params, stream), offsetof(lbm_params, tile_rows),
         offsetof(lbm_params, hist_max), offsetof(lbm_params, body_force));
  printf("%zu %zu %zu %zu\n", offsetof(lbm_stats_t, nr), offsetof(lbm_stats_t, Sp), offsetof(lbm_stats_t, F4),
         offsetof(lbm_stats_t, lumley_eta));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    assert sizes == [ctypes.sizeof(lib.LbmParams), ctypes.sizeof(lib.LbmStats), ctypes.sizeof(lib.LbmRecord)]
    offs = [int(v) for v in lines[1].split()]
    P = lib.LbmParams
    assert offs == [P.stream.offset, P.tile_rows.offset, P.hist_max.offset, P.body_force.offset]
    offs = [int(v) for v in lines[2].split()]
    S = lib.LbmStats
    assert offs == [S.nr.offset, S.Sp.offset, S.F4.offset, S.lumley_eta.offset]


@pytest.mark.parametrize("kw,frag", [
    (dict(nx=0, nu0=0.01), "lattice size"),
    (dict(nx=8, nu0=0.0, re=0.0), "nu0"),
    (dict(nx=8, nu0=0.01, cs=-0.1), "Smagorinsky"),
    (dict(nx=8, nu0=0.01, precision=7), "precision"),
    (dict(nx=8, nu0=0.01, force_mode=9), "force_mode"),
    (dict(nx=8, nu0=0.01, hist_bins=-1), "hist_bins"),
    (dict(nx=8, nu0=0.01, kernel=5), "kernel"),
    (dict(nx=8, nu0=0.01, tma_slots=3), "tma_slots"),
    (dict(nx=8, nu0=0.01, layout=3), "layout"),
    (dict(nx=8, nu0=0.01, strain_mode=2), "strain_mode"),
])
def test_invalid_parameters_rejected_before_any_device_call(lib, kw, frag):
    nx = kw.pop("nx")
    p = lib.make_params(nx, **kw)
    with pytest.raises(lib.LbmError) as ei:
        lib.lbm_create(p)
    assert ei.value.code == lib.LBM_ERR_INVALID_ARG
    assert frag in str(ei.value)


def test_mixed_precision_batch_rejected(lib):
    a = lib.make_params(8, nu0=0.01)
    b = lib.make_params(8, nu0=0.01, precision=lib.LBM_FP16_SHIFTED)
    with pytest.raises(lib.LbmError) as ei:
        lib.lbm_create_batch([a, b])
    assert ei.value.code == lib.LBM_ERR_UNSUPPORTED


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.LbmError) as ei:
        lib.lbm_create(lib.make_params(8, nu0=0.01))
    assert ei.value.code == lib.LBM_ERR_CUDA


def test_energy_balance_host_function(lib):
    """lbm_energy_balance is host arithmetic: runs without a GPU.  An exactly
    balanced synthetic series (E = E0 exp(-2at), eps = 2aE + I) gives residuals
    within the O(dt^2) central-difference error; bad input is rejected."""
    import numpy as np

    a, E0, I = 1e-3, 2e-3, 3e-7
    recs = []
    for t in range(0, 2000, 50):
        E = E0 * np.exp(-2 * a * t)
        recs.append({"step": t, "E_k": E, "inj": I, "eps0": 2 * a * E + I, "eps_sgs": 0.0})
    at, r = lib.lbm_energy_balance(recs)
    assert list(at) == list(range(50, 1950, 50))
    assert np.abs(r).max() < 2 * (2 * a * 50) ** 2 / 6
    with pytest.raises(lib.LbmError):
        lib.lbm_energy_balance(recs[:2])
    with pytest.raises(lib.LbmError):
        lib.lbm_energy_balance([recs[1], recs[0], recs[2]])


def test_batch_and_velocity_entry_points_validate_arguments(lib):
    """lbm_batch_create / lbm_batch_step / lbm_batch_stats / lbm_get_velocity
    reject bad arguments before any device call, like the functions they
    stand for."""
    calls = (lambda: lib.lbm_batch_step(None, 1), lambda: lib.lbm_batch_stats(None, 1),
             lambda: lib.lbm_get_velocity(None, 0, (2, 2, 2)), lambda: lib.lbm_batch_create([]))
    for call in calls:
        with pytest.raises(lib.LbmError) as ei:
            call()
        assert ei.value.code == lib.LBM_ERR_INVALID_ARG
    a = lib.make_params(8, nu0=0.01)
    b = lib.make_params(8, nu0=0.01, precision=lib.LBM_FP16_SHIFTED)
    with pytest.raises(lib.LbmError) as ei:
        lib.lbm_batch_create([a, b])
    assert ei.value.code == lib.LBM_ERR_UNSUPPORTED


def test_series_shell_count_matches_the_oracle_rule():
    """The series writer bins the spectrum into the same shells as the oracle."""
    from oracle import diagnostics as dg
    from paper_2512_23116_gb300 import series

    for shape in ((24, 24, 24), (100, 100, 100), (40, 36, 32), (7, 5, 3), (800, 800, 800)):
        assert series._max_shell(*shape) == dg.max_shell(*shape)
