"""Pins of the oracle's edit-target rule, one branch at a time.

Sec. III-B names four extremum distortions fixed by the C-loop (FPmax spelled
out; FNmax, FPmin and FNmin left to MSz) and Sec. IV-A adds the two ordering
cases.  Because edits only lower values, each case has one fix:

- FPmax (g makes i a maximum): lower i;
- FNmax and the ascending ordering case (g has a neighbour of i above where f
  has it): lower that neighbour, the spurious maximum;
- FNmin (f makes i a minimum, g does not): lower i;
- FPmin and the descending ordering case: lower f's smallest neighbour of i.

Each golden fixture (tests/golden/) is a tiny grid where exactly one case
fires at exactly one vertex, checked here by brute force before the oracle
runs.  The planted-mistake tests then compile copies of the oracle with one
branch swapped for another plausible choice and show that some fixture fails
with each of them: every branch is pinned by a fixture.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SRC = os.path.join(os.path.dirname(oracle.__file__), "msz_oracle.c")

FIXTURES = ["fpmax_fig_fpmax.json", "fnmax_c_loop.json", "fpmin_c_loop.json", "fnmin_c_loop.json",
            "descending_fig_nonextrema_abc.json", "ascending_fig_nonextrema_def.json"]
NEW = ["fnmax_c_loop.json", "fpmin_c_loop.json", "fnmin_c_loop.json"]


def load(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        d = json.load(fh)
    shape = (d["ny"], d["nx"])
    f = np.array(d["f"], dtype=np.float32).reshape(shape)
    fhat = np.array(d["fhat"], dtype=np.float32).reshape(shape)
    return d, f, fhat, np.float32(d["xi"])


def distorted(f, g):
    """[(vertex, asc differs, desc differs, asc_f, asc_g, desc_f, desc_g)] by brute force."""
    cf, cg = bf.brute_codes(f).reshape(-1), bf.brute_codes(g).reshape(-1)
    out = []
    for i in np.flatnonzero(cf != cg):
        a_f, a_g, d_f, d_g = int(cf[i] & 15), int(cg[i] & 15), int(cf[i] >> 4), int(cg[i] >> 4)
        out.append((int(i), a_f != a_g, d_f != d_g, a_f, a_g, d_f, d_g))
    return out


@pytest.mark.parametrize("name", NEW)
def test_exactly_one_case_fires(name):
    """The fixture's precondition, from the brute-force codes alone."""
    d, f, fhat, xi = load(name)
    pf = d["paper_facts"]
    assert oracle.validate(f, fhat, xi) == oracle.OK
    dist = distorted(f, fhat)
    assert len(dist) == 1 and dist[0][0] == pf["distorted"], dist
    i, asc, desc, a_f, a_g, d_f, d_g = dist[0]
    rule = pf["rule"]
    if rule == "FNmax":
        assert asc and not desc and a_f == oracle.SELF and a_g != oracle.SELF
    elif rule == "FPmin":
        assert desc and not asc and d_f != oracle.SELF and d_g == oracle.SELF
    elif rule == "FNmin":
        assert desc and not asc and d_f == oracle.SELF and d_g != oracle.SELF
    assert pf["lowered"] != pf["not_lowered"]


@pytest.mark.parametrize("rule", [oracle.RULE_HALVE, oracle.RULE_SNAP])
@pytest.mark.parametrize("name", NEW)
def test_the_one_fix_is_applied(name, rule):
    """The oracle lowers exactly the vertex the case's only fix lowers, in one
    sweep, and the loop ends with the codes of f (brute force)."""
    d, f, fhat, xi = load(name)
    pf = d["paper_facts"]
    r = oracle.correct(f, fhat, xi, rule=rule, log_capacity=8)
    assert r.status == oracle.OK
    assert list(r.edit_idx) == [pf["lowered"]]
    assert r.sweep_log[0, 1] == 1 and r.sweep_log[0, 2] == 1
    g = r.g.reshape(-1)
    assert g[pf["lowered"]] < fhat.reshape(-1)[pf["lowered"]]
    assert g[pf["not_lowered"]] == fhat.reshape(-1)[pf["not_lowered"]]
    assert np.array_equal(bf.brute_codes(r.g), bf.brute_codes(f))


# ------------------------------------------------------- planted mistakes
# Each mutant replaces one line of targets_of (the original text must be
# present) with another non-increasing choice a reader could make.
ASC_SELF = "if (asc_g == ORC_SELF) t[k++] = i;"
ASC_NB = "else if (orc_neighbour(ndim, nx, ny, nz, i, asc_g, &j)) t[k++] = j;"
DESC_SELF = "if (desc_f == ORC_SELF) t[k++] = i;"
DESC_NB = "else if (orc_neighbour(ndim, nx, ny, nz, i, desc_f, &j)) t[k++] = j;"

MUTANTS = {
    # FPmax: lower f's largest neighbour instead of the false maximum
    "fpmax_lowers_f_nmax": (ASC_SELF, "if (asc_g == ORC_SELF) { if (orc_neighbour(ndim, nx, ny, nz, i, asc_f, &j)) "
                                      "t[k++] = j; }"),
    # FNmax / ascending ordering: lower the vertex instead of the spurious maximum
    "fnmax_lowers_self": (ASC_NB, "else t[k++] = i;"),
    # FNmin: lower g's smaller neighbour instead of the vertex
    "fnmin_lowers_g_nmin": (DESC_SELF, "if (desc_f == ORC_SELF) { if (orc_neighbour(ndim, nx, ny, nz, i, desc_g, &j)) "
                                       "t[k++] = j; }"),
    # FPmin / descending ordering: lower g's smallest neighbour instead of f's
    "fpmin_lowers_g_nmin": (DESC_NB, "else if (orc_neighbour(ndim, nx, ny, nz, i, desc_g, &j)) t[k++] = j;"),
    # the descending branch written as a mirror of the ascending one
    "desc_mirrors_asc": (DESC_SELF, "if (desc_g == ORC_SELF) t[k++] = i;"),
}


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


def build_mutant(name, outdir):
    old, new = MUTANTS[name]
    with open(SRC) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"targets_of no longer holds the line {old!r}"
    path = os.path.join(str(outdir), f"{name}.c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    so = os.path.join(str(outdir), f"lib{name}.so")
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", path, "-o", so, "-lm"],
                   check=True)
    return oracle._configure(ctypes.CDLL(so))


def passes(name):
    d, f, fhat, xi = load(name)
    pf = d["paper_facts"]
    r = oracle.correct(f, fhat, xi, log_capacity=64)
    if r.status != oracle.OK or not np.array_equal(bf.brute_codes(r.g), bf.brute_codes(f)):
        return False
    if "lowered" in pf:
        return list(r.edit_idx) == [pf["lowered"]]
    for key in ("distorted_vertex", "A", "D"):  # the figures' lowered vertex
        if key in pf:
            return list(r.edit_idx) == [pf[key]]
    return True


def test_every_fixture_passes_with_the_oracle():
    assert all(passes(n) for n in FIXTURES)


@pytest.mark.parametrize("mutant", list(MUTANTS))
def test_planted_mistake_fails_a_fixture(mutant, mutant_dir, monkeypatch):
    lib = build_mutant(mutant, mutant_dir)
    monkeypatch.setattr(oracle, "_lib", lib)
    failing = [n for n in FIXTURES if not passes(n)]
    assert failing, f"no fixture catches the mutant {mutant}"


def floors_reorder(f, xi):
    """Is there a neighbour pair whose order (value, then index) at the floors
    differs from its order in f?  Only then can the loop end STUCK."""
    L = np.array([oracle.floor_bound(v, xi) for v in f.reshape(-1)], dtype=np.float32)
    flat = f.reshape(-1)
    ns = oracle.num_slots(f.ndim)
    for i in range(flat.size):
        for s in range(ns):
            j = oracle.neighbour(f.shape, i, s)
            if j is None:
                continue
            if ((flat[j], j) > (flat[i], i)) != ((L[j], j) > (L[i], i)):
                return True
    return False


def test_random_tiny_grids_never_stuck_without_collapsed_floors():
    """Sec. III-B convergence: with floors in the order of f the loop always ends
    OK; STUCK is reserved for floors that collapse (test_oracle_loop)."""
    rng = np.random.default_rng(21)
    stuck = 0
    for trial in range(80):
        ndim = 2 + trial % 2
        shape = tuple(int(s) for s in rng.integers(1, 6, size=ndim))
        f = rng.integers(0, 6, size=shape).astype(np.float32) / np.float32(8)
        xi = np.float32(rng.choice([0.05, 0.1, 0.3]))
        noise = rng.uniform(-1, 1, size=shape) * float(xi) * 0.999
        fhat = (f.astype(np.float64) + noise).astype(np.float32)
        r = oracle.correct(f, fhat, xi)
        if r.status == oracle.STUCK:
            stuck += 1
            assert floors_reorder(f, xi)
        else:
            assert r.status == oracle.OK
            assert np.array_equal(bf.brute_codes(r.g), bf.brute_codes(f))
    assert stuck == 0


# ------------------------------------------------------- BELOW-REFERENCE
def below(v, t, r):
    """The reading of 'slightly below' (Sec. IV-A): the largest value that puts
    t below r in the (value, index) order -- r's value when r has the larger
    index, else the float just below it."""
    v = np.float32(v)
    return v if r > t else np.nextafter(v, np.float32(-np.inf), dtype=np.float32)


# fixture -> (lowered vertex, its reference vertex)
BELOW_CASES = {
    "fpmax_fig_fpmax.json": (1, 2),          # the false maximum falls below f's n_max (0.35 in f)
    "fnmax_c_loop.json": (13, 12),           # the spurious neighbour falls below the maximum i
    "fpmin_c_loop.json": (13, 12),           # f's n_min falls below i, which g makes a minimum
    "fnmin_c_loop.json": (12, 17),           # the minimum i falls below g's smaller neighbour
    "descending_fig_nonextrema_abc.json": (3, 5),   # the original minimum 0.1 falls below 0.08
    "ascending_fig_nonextrema_def.json": (5, 8),    # the spurious 0.4 falls to 0.3
}


@pytest.mark.parametrize("name", list(BELOW_CASES))
def test_below_reference_moves_just_under_the_reference(name):
    d, f, fhat, xi = load(name)
    t, r = BELOW_CASES[name]
    res = oracle.correct(f, fhat, xi, rule=oracle.RULE_BELOW, log_capacity=8)
    assert res.status == oracle.OK and res.sweeps == 1
    assert list(res.edit_idx) == [t]
    g = res.g.reshape(-1)
    assert g[t].view(np.uint32) == below(fhat.reshape(-1)[r], t, r).view(np.uint32)
    # t is below r, and the next float up would not be
    assert (float(g[t]), t) < (float(g[r]), r)
    up = np.nextafter(g[t], np.float32(np.inf), dtype=np.float32)
    assert (float(up), t) > (float(g[r]), r)
    assert np.array_equal(bf.brute_codes(res.g), bf.brute_codes(f))


def test_below_reference_worked_example_values():
    """Fig. nonextrema (d)-(f): 'decreased to 0.3 or slightly below' and the
    ascending path 0.15 -> 0.2 -> 0.3."""
    d, f, fhat, xi = load("ascending_fig_nonextrema_def.json")
    pf = d["paper_facts"]
    res = oracle.correct(f, fhat, xi, rule=oracle.RULE_BELOW)
    g = res.g.reshape(-1)
    assert g[pf["D"]] == np.float32(pf["C_value"])
    codes = oracle.codes(res.g).reshape(-1)
    path = [pf["P"]]
    while (codes[path[-1]] & 15) != 15:
        path.append(oracle.neighbour(f.shape, path[-1], int(codes[path[-1]] & 15)))
    assert [np.float32(g[p]) for p in path] == [np.float32(v) for v in pf["path"]]


def test_edit_below_clamps_at_the_floor_and_never_raises():
    assert oracle.edit_below(0.5, 0.2, 0.3) == (np.float32(0.3), True)
    assert oracle.edit_below(0.5, 0.35, 0.3) == (np.float32(0.35), True)   # clamped at the floor
    assert oracle.edit_below(0.35, 0.35, 0.3) == (np.float32(0.35), False)  # already at the floor
    g, ch = oracle.edit_below(0.0, -1.0, -0.0)
    assert not ch and g.view(np.uint32) == np.float32(0.0).view(np.uint32)  # -0 is not below +0 in value
