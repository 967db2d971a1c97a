"""Pins of the oracle's correction loop: the paper's worked examples, the
invariants the paper states for the corrected field, worklist == dense sweeps,
and the termination paths."""
import glob
import json
import os

import numpy as np
import pytest

import oracle
from paper_2601_01787_gb300 import synth
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fixture(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        d = json.load(fh)
    shape = (d["ny"], d["nx"])
    f = np.array(d["f"], dtype=np.float32).reshape(shape)
    fhat = np.array(d["fhat"], dtype=np.float32).reshape(shape)
    return d, f, fhat, np.float32(d["xi"])


def test_fixtures_are_valid_inputs():
    for p in glob.glob(os.path.join(GOLDEN, "*.json")):
        d, f, fhat, xi = _fixture(os.path.basename(p))
        assert oracle.validate(f, fhat, xi) == oracle.OK, p


def test_fpmax_example():
    """Sec. III-B / Fig. fpmax: the false maximum is the vertex that gets lowered;
    its two requests in sweep 0 (FPmax at i, FNmax at the 0.35 vertex) are one
    application (Sec. IV-B: conflicting candidates resolve to one value)."""
    d, f, fhat, xi = _fixture("fpmax_fig_fpmax.json")
    pf = d["paper_facts"]
    r = oracle.correct(f, fhat, xi, log_capacity=8)
    assert r.status == oracle.OK
    assert list(r.edit_idx) == [pf["distorted_vertex"]]
    g = r.g.reshape(-1)
    assert g[pf["distorted_vertex"]] < g[pf["higher_neighbour"]]
    assert r.sweep_log[0, 1] == 2 and r.sweep_log[0, 2] == 1
    assert np.array_equal(oracle.codes(r.g), oracle.codes(f))


@pytest.mark.parametrize("rule", [oracle.RULE_SNAP, oracle.RULE_HALVE])
def test_descending_example(rule):
    """Sec. IV-A descending rule: the ORIGINAL minimum (0.1) is lowered, not the
    spurious 0.08; with the edit taken to the floor it reaches 0 as in Fig. nonextrema (c)."""
    d, f, fhat, xi = _fixture("descending_fig_nonextrema_abc.json")
    pf = d["paper_facts"]
    assert oracle.codes(fhat).reshape(-1)[pf["i"]] >> 4 != oracle.codes(f).reshape(-1)[pf["i"]] >> 4
    r = oracle.correct(f, fhat, xi, rule=rule)
    assert r.status == oracle.OK
    assert list(r.edit_idx) == [pf["A"]]
    g = r.g.reshape(-1)
    assert g[pf["B"]] == np.float32(pf["B_value"])
    assert g[pf["A"]] < g[pf["B"]]
    if rule == oracle.RULE_SNAP:
        assert g[pf["A"]] == np.float32(pf["A_after_figure"])
    assert np.array_equal(oracle.codes(r.g), oracle.codes(f))


def test_ascending_example():
    """Sec. IV-A ascending rule: the spurious maximum 0.4 drops to 0.3 or below and
    the ascending path from 0.15 runs 0.15 -> 0.2 -> 0.3 again."""
    d, f, fhat, xi = _fixture("ascending_fig_nonextrema_def.json")
    pf = d["paper_facts"]
    r = oracle.correct(f, fhat, xi)
    assert r.status == oracle.OK
    assert list(r.edit_idx) == [pf["D"]]
    g = r.g.reshape(-1)
    assert g[pf["D"]] <= np.float32(pf["C_value"])
    codes = oracle.codes(r.g).reshape(-1)
    path = [pf["P"]]
    while (codes[path[-1]] & 15) != 15:
        path.append(oracle.neighbour(f.shape, path[-1], int(codes[path[-1]] & 15)))
    assert [np.float32(g[p]) for p in path] == [np.float32(v) for v in pf["path"]]


CASES = [
    ("perlin2d", lambda: synth.perlin2d((70, 93), seed=11)),
    ("perlin3d_prequant", lambda: synth.perlin3d_prequant((21, 34, 47), seed=12, eb_rel=1e-3, octaves=4)),
    ("peaks3d", lambda: synth.peaks3d((19, 23, 29), seed=13, eb_rel=1e-3, npeaks=6)),
    ("perlin3d_fine", lambda: synth.perlin3d_prequant((16, 16, 16), seed=14, eb_rel=1e-4)),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def solved(request):
    fl = request.param[1]()
    r = oracle.correct(fl.f, fl.fhat, fl.xi, log_capacity=10000)
    return fl, r


def test_invariants_after_correction(solved):
    """Sec. IV-A relaxed condition + Sec. III-B bound: after the loop, g has the
    codes (extrema and n_min/n_max) of f, the segmentation labels of f, stays in
    [f - xi, fhat] (edits only lower values), and the edit list is exactly the
    set of changed vertices with delta = g - fhat."""
    fl, r = solved
    assert r.status == oracle.OK
    cf, cg = oracle.codes(fl.f), oracle.codes(r.g)
    assert np.array_equal(cf, cg)
    lf, lg = oracle.labels(cf), oracle.labels(cg)
    assert np.array_equal(lf[0], lg[0]) and np.array_equal(lf[1], lg[1])
    assert oracle.compare(cf, cg, *lf, *lg)["wrong_labels"] == 0
    assert np.all(r.g <= fl.fhat)
    lo = np.array([oracle.floor_bound(a, fl.xi) for a in fl.f.reshape(-1)], dtype=np.float32)
    assert np.all(r.g.reshape(-1) >= lo)
    gb = r.g.reshape(-1).view(np.uint32)
    hb = fl.fhat.reshape(-1).view(np.uint32)
    changed = np.flatnonzero(gb != hb)
    assert np.array_equal(r.edit_idx, changed.astype(np.uint32))
    want = (r.g.reshape(-1)[changed] - fl.fhat.reshape(-1)[changed]).astype(np.float32)
    assert np.array_equal(r.edit_delta.view(np.uint32), want.view(np.uint32))
    assert r.edited == len(changed) and r.edit_count == len(changed)
    assert r.first_distorted > 0 and r.sweeps >= 1


def test_edits_are_monotone_and_logged(solved):
    """Sec. III-B convergence argument: every sweep only lowers values; the log
    shows distortions falling to zero with each sweep changing something."""
    fl, r = solved
    log = r.sweep_log
    assert log.shape[0] == r.sweeps + 1
    assert log[-1, 1] == 0
    assert np.all(log[:-1, 3] > 0)
    assert np.all(log[:-1, 3] <= log[:-1, 2])
    assert int(log[:, 3].sum()) == r.edits


def test_worklist_equals_dense(solved):
    """The worklist reading (closed neighbourhood of changed vertices plus the
    distorted ones) gives the same g^k as dense Jacobi sweeps."""
    fl, r = solved
    d = oracle.correct(fl.f, fl.fhat, fl.xi, worklist=False, log_capacity=10000)
    assert d.status == r.status
    assert np.array_equal(d.g.view(np.uint32), r.g.view(np.uint32))
    assert np.array_equal(d.stats[:5], r.stats[:5])
    assert np.array_equal(d.sweep_log[:, 1:], r.sweep_log[:, 1:])
    assert d.examined == fl.n * (d.sweeps + 1) >= r.examined


def test_random_tiny_grids_converge_with_invariants():
    rng = np.random.default_rng(21)
    for trial in range(60):
        ndim = 2 + trial % 2
        shape = tuple(int(s) for s in rng.integers(1, 6, size=ndim))
        f = rng.integers(0, 6, size=shape).astype(np.float32) / np.float32(8)
        xi = np.float32(rng.choice([0.05, 0.1, 0.3]))
        noise = rng.uniform(-1, 1, size=shape) * float(xi) * 0.999
        fhat = (f.astype(np.float64) + noise).astype(np.float32)
        assert oracle.validate(f, fhat, xi) == oracle.OK
        r = oracle.correct(f, fhat, xi)
        assert r.status == oracle.OK  # floors of values 1/8 apart never collapse
        assert np.array_equal(bf.brute_codes(r.g), bf.brute_codes(f))
        d = oracle.correct(f, fhat, xi, worklist=False)
        assert d.status == r.status and np.array_equal(d.g.view(np.uint32), r.g.view(np.uint32))


def test_stuck_when_floors_collapse():
    """f_0 > f_1 but xi so large that both floors round to the same float: at the
    floor the index tie-break puts vertex 1 above vertex 0, which no lowering can
    undo, so the loop reports STUCK instead of spinning."""
    f = np.array([[1.0000001, 1.0]], dtype=np.float32)
    xi = np.float32(1e8)
    L = np.array([oracle.floor_bound(v, xi) for v in f.reshape(-1)], dtype=np.float32).reshape(f.shape)
    assert L[0, 0] == L[0, 1]
    r = oracle.correct(f, L.copy(), xi)
    assert r.status == oracle.STUCK
    assert r.sweeps == 1 and r.left > 0 and r.edits == 0


def test_max_sweeps_and_capacity():
    fl = synth.perlin2d((40, 50), seed=3)
    full = oracle.correct(fl.f, fl.fhat, fl.xi)
    assert full.status == oracle.OK and full.sweeps >= 2
    capped = oracle.correct(fl.f, fl.fhat, fl.xi, max_sweeps=1)
    assert capped.status == oracle.ERR_MAX_SWEEPS and capped.sweeps == 1 and capped.left > 0
    small = oracle.correct(fl.f, fl.fhat, fl.xi, edit_capacity=3)
    assert small.status == oracle.ERR_CAPACITY and small.edit_count == full.edit_count
    assert np.array_equal(small.g.view(np.uint32), full.g.view(np.uint32))


def test_already_correct_input_needs_no_sweep():
    fl = synth.perlin2d((30, 31), seed=4)
    r = oracle.correct(fl.f, fl.f.copy(), fl.xi)
    assert r.status == oracle.OK and r.sweeps == 0 and r.edit_count == 0 and r.first_distorted == 0


def test_g_init_start_inside_bound():
    """A proposed start (as the learned proposal gives) still ends with the invariants."""
    fl = synth.perlin3d_prequant((12, 13, 14), seed=5, eb_rel=1e-3)
    lo = np.array([oracle.floor_bound(a, fl.xi) for a in fl.f.reshape(-1)], dtype=np.float32).reshape(fl.shape)
    g0 = np.maximum(lo, (fl.fhat.astype(np.float64) - 0.3 * (fl.fhat - lo)).astype(np.float32))
    r = oracle.correct(fl.f, fl.fhat, fl.xi, g_init=g0)
    assert r.status == oracle.OK
    assert np.array_equal(oracle.codes(r.g), oracle.codes(fl.f))
    assert np.all(r.g <= g0)
