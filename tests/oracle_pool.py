"""Oracle corrections of large fields, run in worker processes.

The at-scale parity tests need the CPU oracle's whole correction of fields of
up to 512^3 vertices (tens of seconds each on one core).  The workers are
started with the ``spawn`` method (never forked from a process that has
touched the GPU), each regenerates its field from the seeded recipe, runs the
oracle and writes the result to a scratch ``.npz`` file whose path it returns.
Nothing here imports torch or the CUDA library: the workers use only the
oracle and the input generators.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile
from concurrent.futures import ProcessPoolExecutor

import numpy as np

import oracle
from paper_2601_01787_gb300 import synth


def make_field(spec):
    """A field from its recipe: ("perlin", kwargs), ("peaks", kwargs) or
    ("batch", k) for field k of the 64-field uneven batch."""
    kind, arg = spec
    if kind == "perlin":
        return synth.perlin3d_prequant(**arg)
    if kind == "peaks":
        return synth.peaks3d(**arg)
    if kind == "batch":
        shape, eb, seed = synth.batch_shapes()[arg]
        return synth.perlin3d_prequant(shape, seed=seed, eb_rel=eb)
    raise ValueError(spec)


def _job(spec, kwargs, outdir):
    fl = make_field(spec)
    r = oracle.correct(fl.f, fl.fhat, fl.xi, log_capacity=100000, **kwargs)
    fd, path = tempfile.mkstemp(suffix=".npz", dir=outdir)
    os.close(fd)
    np.savez(path, g=r.g, edit_idx=r.edit_idx, edit_delta=r.edit_delta, sweep_log=r.sweep_log,
             stats=np.array([r.status, r.sweeps, r.edits, r.edited, r.first_distorted, r.left, r.examined,
                             r.edit_count], dtype=np.int64))
    return path


class OracleResult:
    def __init__(self, path):
        with np.load(path) as z:
            self.g = z["g"]
            self.edit_idx = z["edit_idx"]
            self.edit_delta = z["edit_delta"]
            self.sweep_log = z["sweep_log"]
            s = z["stats"]
        os.unlink(path)
        (self.status, self.sweeps, self.edits, self.edited, self.first_distorted, self.left, self.examined,
         self.edit_count) = (int(v) for v in s)


class Pool:
    """A spawn-started pool of oracle workers; submit() returns a future whose
    result() is an OracleResult."""

    def __init__(self, workers: int | None = None):
        n = workers or max(1, min(12, (os.cpu_count() or 2) - 2))
        self.dir = tempfile.mkdtemp(prefix="msz_oracle_")
        self.ex = ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))

    def submit(self, spec, **kwargs):
        fut = self.ex.submit(_job, spec, kwargs, self.dir)
        return _Future(fut)

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)
        try:
            for name in os.listdir(self.dir):
                os.unlink(os.path.join(self.dir, name))
            os.rmdir(self.dir)
        except OSError:
            pass


class _Future:
    def __init__(self, fut):
        self._fut = fut
        self._res = None

    def result(self) -> OracleResult:
        if self._res is None:
            self._res = OracleResult(self._fut.result())
        return self._res
