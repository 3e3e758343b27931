"""The seeded input generator (synthetic/): solenoidal, exact u_rms, the
k^4 exp(-2 (k/k0)^2) shell shape, deterministic per seed, and the same field
from the host and the torch synthesis."""
import math

import numpy as np

import synthetic
from oracle import diagnostics as dg


def test_splitmix64_reference_values():
    """SplitMix64 from state 0 (Vigna's reference generator, state += golden ratio
    before mixing): the first outputs are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4."""
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        out = synthetic.splitmix64(np.array([0, g], dtype=np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_random_field_properties():
    n = 32
    u = synthetic.random_solenoidal(n, seed=1, k0=4.0, urms=0.05)
    assert math.isclose(math.sqrt(np.mean(np.sum(u * u, axis=0)) / 3), 0.05, rel_tol=1e-12)
    k = np.fft.fftfreq(n, 1 / n)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    uh = [np.fft.fftn(u[d]) for d in range(3)]
    div = KX * uh[0] + KY * uh[1] + KZ * uh[2]
    assert np.abs(div).max() < 1e-12 * np.abs(uh[0]).max()
    E = dg.spectrum(u)
    s = np.arange(1, 15)
    shape = s ** 4.0 * np.exp(-2 * (s / 4.0) ** 2)
    ratio = E[1:15] / shape
    assert np.allclose(ratio, ratio[0], rtol=1e-9)


def test_seed_determinism_and_variation():
    a = synthetic.random_solenoidal(16, seed=3)
    b = synthetic.random_solenoidal(16, seed=3)
    c = synthetic.random_solenoidal(16, seed=4)
    assert np.array_equal(a, b)
    assert np.abs(a - c).max() > 1e-3


def test_torch_synthesis_matches_host():
    import torch

    k, a = synthetic.spectrum_coefficients(12, 10, 8, seed=5)
    host = synthetic.synthesize(k, a, 12, 10, 8)
    dev = synthetic.synthesize_torch(k, a, 12, 10, 8, "cpu", zchunk=3).numpy()
    assert np.abs(host - dev).max() < 1e-15
