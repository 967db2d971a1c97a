"""Pins of the relaxed-synchronization oracle (Sec. IV-B emulated on one
device): one tile covering the grid is the synchronous loop itself; any
tiling ends in a field that satisfies every invariant of the method."""
import numpy as np
import pytest

import oracle
from paper_2601_01787_gb300 import synth


def _cases():
    return [
        ("perlin3d", synth.perlin3d_prequant((20, 30, 40), seed=5, eb_rel=1e-3, octaves=4)),
        ("peaks3d", synth.peaks3d((24, 28, 36), seed=6, eb_rel=1e-4)),
        ("perlin2d", synth.perlin2d((60, 70), seed=7)),
    ]


@pytest.mark.parametrize("name,fl", _cases())
def test_one_tile_is_the_synchronous_loop(name, fl):
    ref = oracle.correct(fl.f, fl.fhat, fl.xi)
    st, g, stats = oracle.correct_relaxed(fl.f, fl.fhat, fl.xi, fl.f.shape)
    assert st == ref.status == oracle.OK
    assert np.array_equal(g.view(np.uint32), ref.g.view(np.uint32))
    assert stats[1] == ref.sweeps          # local sweeps of the one run = the loop's sweeps
    assert stats[0] == (1 if ref.sweeps else 0) and stats[5] == (1 if ref.first_distorted else 0)
    assert stats[2] == ref.edited and stats[3] == ref.first_distorted


@pytest.mark.parametrize("name,fl", _cases())
@pytest.mark.parametrize("tile", [(8, 8, 32), (2, 3, 5), (1, 1, 1)])
def test_any_tiling_keeps_the_invariants(name, fl, tile):
    tile = tile if fl.f.ndim == 3 else tile[1:]
    st, g, stats = oracle.correct_relaxed(fl.f, fl.fhat, fl.xi, tile)
    assert st == oracle.OK
    assert np.array_equal(oracle.codes(g), oracle.codes(fl.f))
    assert oracle.validate(fl.f, g, fl.xi) == oracle.OK and np.all(g <= fl.fhat)
    mn_f, mx_f = oracle.labels(oracle.codes(fl.f))
    mn_g, mx_g = oracle.labels(oracle.codes(g))
    assert np.array_equal(mn_f, mn_g) and np.array_equal(mx_f, mx_g)
    assert stats[4] == 0


def test_relaxed_needs_fewer_global_iterations_than_sweeps():
    fl = synth.peaks3d((32, 40, 48), seed=8, eb_rel=1e-4)
    ref = oracle.correct(fl.f, fl.fhat, fl.xi)
    st, g, stats = oracle.correct_relaxed(fl.f, fl.fhat, fl.xi, (8, 8, 32))
    assert st == oracle.OK and ref.sweeps > 5
    assert stats[0] < ref.sweeps


def test_iteration_cap_and_already_correct_input():
    fl = synth.peaks3d((16, 16, 40), seed=9, eb_rel=1e-4)
    st, g, stats = oracle.correct_relaxed(fl.f, fl.fhat, fl.xi, (4, 4, 8), max_iters=0)
    assert st == oracle.ERR_MAX_SWEEPS and stats[4] == stats[3] > 0
    assert np.array_equal(g.view(np.uint32), fl.fhat.view(np.uint32))
    st, g2, stats = oracle.correct_relaxed(fl.f, fl.f, fl.xi, (4, 4, 8))
    assert st == oracle.OK and stats[0] == 0 and stats[3] == 0
