"""Onset of the instability of the DNS-shape setting, on the GPU and in the
FP64 oracle from the same state (a measurement script, not collected by
pytest: it runs for several minutes, most of them in the oracle).

    python tests/stability_handover.py [n] [nu0] [t_handover] [t_max]

A lattice of n^3 cells (default 400), C = 0, nu0 (default 1e-4), the paper's
forcing with U0 = 0.043, Cf = 0.2, the seeded random field with u_rms = 0.05
per component (k0 = 4), advanced on the GPU to t_handover (default 760); its
populations are handed to the oracle (canonical FP64), then both advance one
step at a time and each step prints the largest |f'| of either side and where
the oracle's sits, until both have passed |f'| = 1 (a population f = f' + w
outside [0, 1]) by three steps or t_max (default 830) is reached.  The last
line gives the first step at which each side passed 1."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _View:
    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": "<f4", "data": (ptr, False), "version": 3}


def main(argv):
    import torch

    import oracle
    import paper_2512_23116_gb300 as lbm

    n = int(argv[1]) if len(argv) > 1 else 400
    nu0 = float(argv[2]) if len(argv) > 2 else 1e-4
    t_handover = int(argv[3]) if len(argv) > 3 else 760
    t_max = int(argv[4]) if len(argv) > 4 else 830
    U0, CF = 0.043, 0.2
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    p = lbm.make_params(n, nu0=nu0, cs=0.0, f0=CF * U0 ** 2 / n, force_mode=lbm.LBM_FORCE_PAPER_SIN,
                        stream=stream.cuda_stream, layout=1)
    t0 = time.time()
    first = {}
    with lbm.Lattice(p) as L:
        L.init_random(seed=1, urms=0.05, k0=4.0)
        L.step(t_handover)
        ptr, nbytes, nxp = lbm.lbm_device_ptr(L.h)
        A = torch.as_tensor(_View(ptr, (19, n, n, nxp)), device=dev)
        ref = oracle.OracleLBM(n, n, n, nu0, 0.0, oracle.FORCE_PAPER_SIN, F0=CF * U0 ** 2 / n)
        ref.set_populations(L.populations())
        print(json.dumps({"config": L.config(), "handover_at": t_handover}), flush=True)
        t = t_handover
        while t < t_max:
            L.step(1)
            ref.step(1)
            t += 1
            torch.cuda.synchronize()
            gmax = float(A[:, :, :, :n].abs().max())  # the AA slots hold the same values
            fo = np.abs(ref.populations())
            omax = float(np.nanmax(fo)) if np.isfinite(fo).all() else float("inf")
            where = [int(v) for v in np.unravel_index(int(np.nanargmax(fo)), fo.shape)] if np.isfinite(omax) else None
            del fo
            for side, m in (("gpu", gmax), ("oracle", omax)):
                if side not in first and not m <= 1.0:
                    first[side] = t
            print(json.dumps({"t": t, "gpu_max_abs_fprime": gmax, "oracle_max_abs_fprime": omax,
                              "oracle_argmax_a_z_y_x": where, "s": round(time.time() - t0, 1)}), flush=True)
            if len(first) == 2 and t >= max(first.values()) + 3:
                break
    print(json.dumps({"first_step_max_abs_fprime_above_1": first}), flush=True)


if __name__ == "__main__":
    main(sys.argv)
