"""Statistics time series of a run, written as JSON lines.

The paper computes its statistics "on the fly" at set intervals of a run
(Sec. 3.1) and reads the operating regime off their time series (Sec. 4.1,
Fig. tau_timeseries).  ``run_with_statistics`` advances a handle and, every
``every`` steps, appends one JSON object per line to a file: the domain
statistics of ``lbm_stats`` (energy, injection, both dissipation terms, theta =
tau_e - 1/2 mean / variance / extremes / percentiles, K_t, isotropy, and with
the flags the derived scales and S_p(r), F4(r)), the shell spectrum E(k) of
``lbm_spectrum`` and, optionally, a theta slice (the K_t map) saved beside the
file as a ``.npy`` array.  Every quantity comes from the library's kernels;
this module only sequences the calls and writes the file.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import (LBM_STATS_SPECTRUM, LBM_STATS_STRUCTURE, lbm_get_theta_slice, lbm_spectrum, lbm_stats,
               lbm_step)


def _plain(v):
    if isinstance(v, np.ndarray):
        return [_plain(x) for x in v.tolist()]
    if isinstance(v, (list, tuple)):
        return [_plain(x) for x in v]
    if isinstance(v, float) and not math.isfinite(v):
        return None
    if isinstance(v, (np.floating, np.integer)):
        return _plain(v.item())
    return v


def run_with_statistics(lattice, steps: int, every: int, path: str, inst: int = 0,
                        what: int = LBM_STATS_SPECTRUM | LBM_STATS_STRUCTURE, spectrum: bool = True,
                        theta_slice=None) -> list:
    """Advance ``lattice`` (a ``Lattice``) by ``steps`` steps and record the
    statistics of instance ``inst`` after every ``every`` steps (and after the
    last one) as JSON lines appended to ``path``.

    ``what``: the ``lbm_stats`` flags; ``spectrum``: add E(k) for shells
    0..kmax; ``theta_slice``: None or (axis, index) of a theta plane, saved as
    ``<path without extension>_theta_t<step>.npy``.  Returns the records."""
    if steps < 0 or every < 1:
        raise ValueError("steps must be >= 0 and every >= 1")
    nz, ny, nx = lattice.shapes[inst]
    kmax = _max_shell(nx, ny, nz)
    stem = os.path.splitext(path)[0]
    records = []
    done = 0
    if steps > 0:
        n = min(every, steps)
        lbm_step(lattice.h, n)
        done = n
    with open(path, "a") as fh:
        while records or done > 0:
            # statistics of the state after `done` steps (these calls wait for
            # the steps enqueued before them)
            st = lbm_stats(lattice.h, inst, what)
            E = lbm_spectrum(lattice.h, inst, kmax) if spectrum else None
            sl = None
            if theta_slice is not None:
                sl = lbm_get_theta_slice(lattice.h, inst, theta_slice[0], theta_slice[1], lattice.shapes[inst])
            # enqueue the next interval, so that the device steps while the
            # host writes this record
            more = done < steps
            if more:
                n = min(every, steps - done)
                lbm_step(lattice.h, n)
                done += n
            rec = {k: _plain(v) for k, v in st.items()}
            if E is not None:
                rec["E"] = _plain(E)
            if sl is not None:
                fname = f"{stem}_theta_t{st['step']}.npy"
                np.save(fname, sl)
                rec["theta_slice"] = {"axis": theta_slice[0], "index": theta_slice[1],
                                      "file": os.path.basename(fname)}
            fh.write(json.dumps(rec) + "\n")
            fh.flush()
            records.append(rec)
            if not more:
                break
    return records


def read_series(path: str) -> list:
    """The records of a JSON-lines statistics file, oldest first."""
    with open(path) as fh:
        return [json.loads(ln) for ln in fh if ln.strip()]


def _max_shell(nx: int, ny: int, nz: int) -> int:
    """Largest integer shell holding a mode of the box (the shells the spectrum bins into)."""
    K = (nx // 2) ** 2 + (ny // 2) ** 2 + (nz // 2) ** 2
    r = math.isqrt(K)
    return r + 1 if K > r * r + r else r
