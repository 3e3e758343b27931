"""Parity at the benchmark's full size, in the launch configuration bench.py times.

The 800^3 forced-HIT DNS-shape workload (FP32, FP16- and BF16-shifted storage) is
far beyond what the oracle can run, so sampled cells are checked one by one:
the population array is read in place through lbm_device_ptr (zero-copy, in
the layout lbm_kernel_config reports), the
19 pre-collision populations of each sampled cell are taken from the AA layout,
one step is run, and the post-collision values the kernel stored for that cell
are compared with the oracle's single-cell collision (Eq. mrt_les_guo).

Where they live (AA pattern): at even time t, cell x's f_a is slot a of x and
the even step stores f*_a in slot opp(a) of x; at odd time, f_a is slot opp(a)
of x - c_a and the odd step stores f*_a in slot a of x + c_a.
"""
import numpy as np
import pytest

import oracle

from gpu_helpers import fp32_mass_tolerance

pytestmark = pytest.mark.gpu

N = 800
U0, CF, RE = 0.043, 0.2, 2.0e4


def _populations_view(torch, lbm, L, dev, typestr):
    """Zero-copy [19][nz][ny][nxp] view of the population array in either
    layout (row-interleaved [nz][ny][19][nxp] arrays are viewed permuted)."""
    ptr, nbytes, nxp = lbm.lbm_device_ptr(L.h)
    shape = (19, N, N, nxp) if L.config()["layout"] == 1 else (N, N, 19, nxp)
    word = "<i2" if typestr == "bf16" else typestr
    A = torch.as_tensor(_CudaArray(ptr, shape, word), device=dev)
    if typestr == "bf16":  # no array-interface type string: view the raw 16-bit words
        A = A.view(torch.bfloat16)
    assert A.numel() * A.element_size() == nbytes
    return A if L.config()["layout"] == 1 else A.permute(2, 0, 1, 3)


# Position of population slot a inside a cell row of the row-interleaved array
# (the order include/lbm.h documents for lbm_device_ptr)
GPOS = [0, 1, 15, 4, 11, 8, 16, 5, 6, 17, 18, 3, 14, 7, 12, 9, 10, 13, 2]


def _slot_map(lbm, L):
    return GPOS if L.config()["layout"] == 2 else list(range(19))


class _CudaArray:
    """Minimal __cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _sample_cells(rng, n, k):
    return rng.integers(0, n, size=(k, 3))  # (x, y, z)


@pytest.mark.parametrize("precision,C", [(0, 0.0), (1, 0.0), (2, 0.0), (0, 0.13), (1, 0.13)])
def test_800_cubed_sampled_cells_match_oracle(gpu_lib, precision, C):
    """C = 0: the DNS shape the bench times.  C = 0.13: the Smagorinsky branch
    (strain, eddy viscosity, local shear rate) at the same size, the cells
    sampled in four z planes whose theta = tau_e - 1/2 is read before each step
    with lbm_get_theta_slice and compared with the theta of the oracle's
    collision of the same cell."""
    import torch

    lbm = gpu_lib
    dev = torch.device("cuda", 0)
    nu0 = U0 * N / RE
    F0 = CF * U0 * U0 / N
    p = lbm.make_params(N, precision=precision, nu0=nu0, cs=C, f0=F0,
                        force_mode=lbm.LBM_FORCE_PAPER_SIN)
    c, w = oracle.lattice()
    opp = [1, 0, 3, 2, 5, 4, 7, 6, 9, 8, 11, 10, 13, 12, 15, 14, 17, 16, 18]
    rng = np.random.default_rng(2024)
    cells = _sample_cells(rng, N, 2048)
    planes = [0, 317, 511, N - 1]
    if C > 0:
        cells[:, 2] = np.array(planes)[np.arange(len(cells)) % len(planes)]
    xs = np.arange(N)
    Fx = F0 * np.sin(2 * np.pi * xs / N)  # Fx(y), Fy(z), Fz(x) share this table
    try:
        with lbm.Lattice(p) as L:
            L.init_random(seed=1, urms=0.05, k0=4.0)  # the bench's workload field
            L.step(2)
            L.sync()
            A = _populations_view(torch, lbm, L, dev, ["<f4", "<f2", "bf16"][precision])
            sm = _slot_map(lbm, L)  # slot -> index along A's first axis
            X = torch.as_tensor(cells[:, 0], device=dev)
            Y = torch.as_tensor(cells[:, 1], device=dev)
            Z = torch.as_tensor(cells[:, 2], device=dev)
            for parity in ("even", "odd"):
                assert (L.time % 2 == 0) == (parity == "even")
                pre = torch.empty((19, len(cells)), dtype=torch.float64, device=dev)
                for q in range(19):
                    if parity == "even":
                        pre[q] = A[sm[q], Z, Y, X].double()
                    else:
                        xs_ = (X - int(c[q][0])) % N
                        ys_ = (Y - int(c[q][1])) % N
                        zs_ = (Z - int(c[q][2])) % N
                        pre[q] = A[sm[opp[q]], zs_, ys_, xs_].double()
                # theta of the state the step collides (read-only statistics pass)
                theta_pre = {z: lbm.lbm_get_theta_slice(L.h, 0, 2, z, (N, N, N)) for z in planes} if C > 0 else {}
                L.step(1)
                L.sync()
                post = torch.empty_like(pre)
                for q in range(19):
                    if parity == "even":
                        post[q] = A[sm[opp[q]], Z, Y, X].double()
                    else:
                        xd = (X + int(c[q][0])) % N
                        yd = (Y + int(c[q][1])) % N
                        zd = (Z + int(c[q][2])) % N
                        post[q] = A[sm[q], zd, yd, xd].double()
                pre_h = pre.cpu().numpy()
                post_h = post.cpu().numpy()
                want = np.empty_like(post_h)
                theta_want = np.empty(len(cells))
                for i, (x, y, z) in enumerate(cells):
                    F = (Fx[y], Fx[z], Fx[x])
                    want[:, i], theta_want[i] = oracle.collide_one(pre_h[:, i], F, nu0, C)
                if C > 0:
                    theta_got = np.array([theta_pre[z][y, x] for (x, y, z) in cells])
                    assert np.all(np.abs(theta_got - theta_want) <= 1e-5 * theta_want), parity
                    # the eddy viscosity is active (the 800^3 field is smooth: a few percent)
                    assert theta_want.max() > 1.02 * 3 * nu0
                if precision == 0:
                    rel = np.abs(post_h - want) / (want + w[:, None])
                    assert rel.max() <= 1e-5, (parity, rel.max())
                else:
                    # one FP16 / BF16 rounding of the stored result (10 / 7 mantissa bits),
                    # on top of FP32 arithmetic
                    mant = 10 if precision == 1 else 7
                    spacing = 2.0 ** (np.floor(np.log2(np.abs(want) + 1e-30)) - mant)
                    assert np.all(np.abs(post_h - want) <= spacing + 1e-7), parity
            del A
    finally:
        torch.cuda.empty_cache()


def test_800_cubed_mass_conservation(gpu_lib):
    """Sum of f' over the 9.7e9 stored values (FP64 sum on the device) after the
    bench's warm-up and a few steps equals the initial sum to FP32 round-off."""
    import torch

    lbm = gpu_lib
    dev = torch.device("cuda", 0)
    nu0 = U0 * N / RE
    p = lbm.make_params(N, nu0=nu0, cs=0.0, f0=CF * U0 * U0 / N, force_mode=lbm.LBM_FORCE_PAPER_SIN)
    try:
        with lbm.Lattice(p) as L:
            L.init_random(seed=1, urms=0.05, k0=4.0)
            A = _populations_view(torch, lbm, L, dev, "<f4")

            def mass():
                s = torch.zeros((), dtype=torch.float64, device=dev)
                for q in range(19):
                    s += A[q, :, :, :N].double().sum()
                return float(s)

            m0 = mass()
            fmax = float(A[:, :, :, :N].abs().max())
            L.step(6)
            L.sync()
            m1 = mass()
            st = L.stats()
            del A
        tol = fp32_mass_tolerance(N ** 3, 6, fmax)
        assert abs(m1 - m0) <= tol, (m1 - m0, tol)
        # lbm_stats sums per-cell drho (FP32 sums of 19 values) in FP64
        assert abs(st["mass"] - m1) <= 0.01 * tol
    finally:
        torch.cuda.empty_cache()
