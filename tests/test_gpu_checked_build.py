"""The bounds-checked build (liblbm_gb300_checked.so, -DLBM_BOUNDS_CHECK), the
stand-in for a device memory checker: every device index of the step kernels,
the statistics pass, the initialisation, population access, structure
functions and random-field kernels is checked before the access; a failed
check skips the access and is reported as LBM_ERR_CUDA at the next
synchronising call.  The small-lattice parity, diagnostics, random-field,
relaxation-rate and failure-path tests run against that build in a child
process (LBM_LIBRARY=checked) and must pass unchanged: no access out of
bounds in any kernel variant they exercise (both kernels, both population
layouts, every shared-memory slot layout, FP32 / FP16 / BF16, batches, ragged
and degenerate extents)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_small_lattice_suite_under_the_checked_build(gpu_lib):
    from paper_2512_23116_gb300 import _build

    assert os.path.exists(_build.LIB_CHECKED), "build() makes the checked library"
    env = dict(os.environ, LBM_LIBRARY="checked")
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_diagnostics.py", "tests/test_gpu_random_field.py",
             "tests/test_gpu_rates.py", "tests/test_gpu_failure.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", *files],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout


def test_checked_build_is_the_library_loaded_under_the_switch(gpu_lib):
    env = dict(os.environ, LBM_LIBRARY="checked")
    code = ("import paper_2512_23116_gb300 as lbm; lbm.load(); "
            "print(lbm.library_path())")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().endswith("liblbm_gb300_checked.so")
