"""The oracle's exact Hessian over a pool of host processes.

Column blocks of H are independent Hessian-vector products with unit vectors
(Sec. 5.1), so a large H is assembled from oracle.hessian_columns calls on
column ranges in separate processes.  The pool is started with the 'spawn'
method (safe after the parent has used the GPU) and each worker runs its BLAS
single-threaded.  Nothing here computes anything itself.
"""

from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _columns(args):
    from oracle import mlp as O
    om, widths, acts, X, Y, lo, hi = args
    return lo, O.hessian_columns(om, widths, acts, X, Y, range(lo, hi))


def hessian(om, widths, acts, X, Y, procs: int | None = None, block: int = 256) -> np.ndarray:
    from oracle import mlp as O
    P = O.num_params(widths)
    procs = procs or max(1, min(32, os.cpu_count() or 1))
    tasks = [(om, widths, acts, X, Y, lo, min(P, lo + block)) for lo in range(0, P, block)]
    H = np.empty((P, P))
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    try:
        for v in saved:
            os.environ[v] = "1"
        with mp.get_context("spawn").Pool(procs) as pool:
            for lo, cols in pool.imap_unordered(_columns, tasks):
                H[:, lo:lo + cols.shape[1]] = cols
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
    return H
