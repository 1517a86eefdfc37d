"""The FP64 CPU oracle spread over host processes (test infrastructure).

TEST INFRASTRUCTURE, like oracle/swkb_oracle.py: only the tests, the smoke
check and the CPU-baseline leg of the benchmark may use it.

ParallelOracle computes exactly what Oracle computes, in the same
arithmetic: the screen's DFT (step a) runs in the parent; the modes are split
into contiguous slices, and each worker process marches its slice's rays
(step b, elementwise arithmetic, so the result does not depend on how the
modes are sliced) and forms every mode's term of the modal sum (steps c, d)
with Oracle.mode_term; the parent adds the terms in mode order, as
Oracle.modal_sum does.  The fields are therefore bit-identical to the serial
oracle's (a CPU test checks this), only faster on many cores.

Workers are started with the "spawn" method (never forked) and touch no GPU.
One OraclePool can serve many problems in turn: a problem reaches the workers
through a pickle file, which each worker loads once.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
import pickle
import tempfile
import uuid

import numpy as np

from oracle.swkb_oracle import Oracle

_CACHE: dict = {}


def _oracle_for(path, key):
    o = _CACHE.get(key)
    if o is None:
        with open(path, "rb") as f:
            pb = pickle.load(f)
        _CACHE.clear()
        o = _CACHE[key] = Oracle(pb)
    return o


def _terms(task):
    """Rays of modes i0 .. i1-1 across screen q and their terms of the sum."""
    path, key, q, i0, i1, c = task
    o = _oracle_for(path, key)
    g = o.g
    rays = o.march(q, o.kappa[i0:i1, None], o.launch_points()[None, :])
    delta = (rays["z"] - g.z_lo) / g.dz
    out = np.empty((i1 - i0, g.N), dtype=np.complex128)
    for j in range(i1 - i0):
        out[j] = o.mode_term(int(o.n[i0 + j]), c[j], delta[j], rays["r"][j], rays["a"][j])
    return out


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """A pool of spawned worker processes (default: one per usable core)."""

    def __init__(self, workers: int | None = None):
        self.workers = int(workers or host_cores())
        self.pool = mp.get_context("spawn").Pool(self.workers)
        self.dir = tempfile.mkdtemp(prefix="swkb_oracle_")

    def close(self):
        if self.pool is not None:
            self.pool.terminate()
            self.pool.join()
            self.pool = None
            for f in os.listdir(self.dir):
                os.remove(os.path.join(self.dir, f))
            os.rmdir(self.dir)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


class ParallelOracle(Oracle):
    """Oracle whose screens run on the processes of `pool` (or of a pool of
    its own with `workers` processes).  Use as a context manager, or call
    close()."""

    def __init__(self, pb, workers: int | None = None, pool: OraclePool | None = None):
        super().__init__(pb)
        self._own = pool is None
        self._pool = OraclePool(workers) if pool is None else pool
        self.workers = self._pool.workers
        self._key = uuid.uuid4().hex
        self._path = os.path.join(self._pool.dir, self._key + ".pkl")
        with open(self._path, "wb") as f:
            pickle.dump(pb, f)

    def close(self):
        if self._pool is not None:
            try:
                os.remove(self._path)
            except OSError:
                pass
            if self._own:
                self._pool.close()
            self._pool = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def screen(self, u, q, keep_rays=False):
        """Gamma_q -> Gamma_{q+1} on the full period, as Oracle.screen (the
        rays are not kept: they live in the workers)."""
        if keep_rays:
            raise ValueError("ParallelOracle does not return rays")
        g = self.g
        u = self.project(u)
        c = self.modes(u)                                            # (a)
        M = len(self.n)
        size = max(1, math.ceil(M / (4 * self.workers)))
        tasks = [(self._path, self._key, q, i0, min(M, i0 + size), c[i0:min(M, i0 + size)])
                 for i0 in range(0, M, size)]
        out = np.zeros(g.N, dtype=np.complex128)
        for terms in self._pool.pool.imap(_terms, tasks):            # (b), (c), (d)
            for t in terms:
                out += t
        return out * self.W
