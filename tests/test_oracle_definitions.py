"""Pins of the oracle's definitions (Sec. III-A, Sec. IV-A) against things other
than itself: the Kuhn simplices, brute force under tuple order, and closed forms."""
import numpy as np
import pytest

import oracle
from tests import bruteforce as bf


@pytest.mark.parametrize("np_shape", [(4, 5), (3, 4, 5), (2, 2, 2), (1, 6), (5, 1), (3, 1, 4), (1, 1, 3),
                                      (4, 3, 1), (1, 1), (1, 1, 1)])
def test_neighbourhood_is_kuhn_triangulation(np_shape):
    """Every in-domain slot of every vertex is an edge of some Kuhn simplex and
    vice versa (reading of 'constant triangular/tetrahedral mesh', Sec. III-A)."""
    shape_xyz = bf.xyz_shape(np_shape)
    nb = bf.kuhn_neighbours(shape_xyz)
    n = int(np.prod(np_shape))
    ndim = len(np_shape)
    for i in range(n):
        c = bf.coords(i, shape_xyz)
        want = sorted(bf.lin(u, shape_xyz) for u in nb.get(c, ()))
        got = sorted(j for s in range(oracle.num_slots(ndim))
                     if (j := oracle.neighbour(np_shape, i, s)) is not None)
        assert got == want, (np_shape, c)


def test_interior_degree():
    """6 neighbours in 2D, 14 in 3D for interior vertices."""
    assert sum(oracle.neighbour((5, 5), 12, s) is not None for s in range(6)) == 6
    i = 2 + 5 * (2 + 5 * 2)
    assert sum(oracle.neighbour((5, 5, 5), i, s) is not None for s in range(14)) == 14


def test_slot_numbering_matches_public_table():
    for ndim, shape in ((2, (7, 7)), (3, (7, 7, 7))):
        xyz = bf.xyz_shape(shape)
        centre = tuple(3 for _ in range(ndim))
        i = bf.lin(centre, xyz)
        for s, d in enumerate(bf.slot_offsets(ndim)):
            j = oracle.neighbour(shape, i, s)
            assert bf.coords(j, xyz) == tuple(a + b for a, b in zip(centre, d))


@pytest.mark.parametrize("np_shape,levels,seed", [
    ((4, 5), 3, 0), ((6, 7), 2, 1), ((3, 4, 5), 3, 2), ((4, 4, 4), 2, 3), ((2, 3, 2), 1, 4),
    ((1, 7), 2, 5), ((3, 1, 4), 2, 6), ((5, 5, 5), 50, 7), ((1, 1, 1), 1, 8), ((2, 1, 1), 2, 9)])
def test_codes_brute_force_with_ties(np_shape, levels, seed):
    """Small integer values make ties everywhere: the index tie-break decides."""
    rng = np.random.default_rng(seed)
    v = rng.integers(0, levels, size=np_shape).astype(np.float32)
    assert np.array_equal(oracle.codes(v), bf.brute_codes(v))


def test_signed_zeros_compare_equal():
    v = np.array([[0.0, -0.0, 0.0], [-0.0, 0.0, -0.0]], dtype=np.float32)
    assert np.array_equal(oracle.codes(v), bf.brute_codes(np.zeros_like(v)))


def _extrema(codes):
    mx = np.flatnonzero((codes.reshape(-1) & 15) == 15)
    mn = np.flatnonzero((codes.reshape(-1) >> 4) == 15)
    return mn, mx


@pytest.mark.parametrize("np_shape", [(6, 7, 8), (9, 11)])
def test_linear_ramp_closed_form(np_shape):
    """a x + b y + c z with a > b > c > 0: one minimum (origin), one maximum (far
    corner), and every interior vertex ascends along (1,1,1) / descends along
    (-1,-1,-1) -- the diagonal edge gains a+b+c, more than any other edge."""
    ndim = len(np_shape)
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in np_shape], indexing="ij")
    if ndim == 3:
        z, y, x = grids
        v = (3.0 * x + 2.0 * y + 1.0 * z).astype(np.float32)
        up, dn = 6, 13
    else:
        y, x = grids
        v = (2.0 * x + 1.0 * y).astype(np.float32)
        up, dn = 2, 5
    c = oracle.codes(v)
    mn, mx = _extrema(c)
    assert list(mn) == [0] and list(mx) == [v.size - 1]
    inner = c[(slice(1, -1),) * ndim]
    assert np.all((inner & 15) == up) and np.all((inner >> 4) == dn)


def test_single_gaussian_bump_has_one_maximum():
    shape = (13, 15, 17)
    z, y, x = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    cz, cy, cx = 6.3, 7.2, 8.4
    v = np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * 3.0 ** 2)).astype(np.float32)
    c = oracle.codes(v)
    _, mx = _extrema(c)
    peak = 8 + 17 * (7 + 15 * 6)   # nearest grid point (8, 7, 6)
    assert list(mx) == [peak]
    _, max_label = oracle.labels(c)
    assert np.all(max_label == peak)


def test_constant_field_extrema_are_index_ends():
    v = np.full((4, 5, 6), 0.25, dtype=np.float32)
    c = oracle.codes(v)
    mn, mx = _extrema(c)
    assert list(mn) == [0] and list(mx) == [v.size - 1]
    min_label, max_label = oracle.labels(c)
    assert np.all(min_label == 0) and np.all(max_label == v.size - 1)


@pytest.mark.parametrize("np_shape,seed", [((5, 6), 0), ((4, 5, 6), 1), ((3, 3, 3), 2), ((1, 9), 3),
                                           ((2, 5, 1), 4)])
def test_labels_brute_force(np_shape, seed):
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 4, size=np_shape).astype(np.float32)
    c = oracle.codes(v)
    mn, mx = oracle.labels(c)
    bmn, bmx = bf.brute_labels(c)
    assert np.array_equal(mn, bmn) and np.array_equal(mx, bmx)
    # labels are extrema of the right kind
    flat = c.reshape(-1)
    assert np.all((flat[mx.reshape(-1)] & 15) == 15)
    assert np.all((flat[mn.reshape(-1)] >> 4) == 15)


def test_compare_counts_planted_differences():
    rng = np.random.default_rng(11)
    f = rng.random((6, 7, 8)).astype(np.float32)
    g = f.copy()
    cf = oracle.codes(f)
    assert oracle.compare(cf, cf, *oracle.labels(cf), *oracle.labels(cf)) == dict(
        wrong_labels=0, fp_max=0, fn_max=0, fp_min=0, fn_min=0)
    # plant a new maximum and a new minimum at interior points far from the originals
    g[3, 3, 3] = 10.0
    g[2, 4, 5] = -10.0
    cg = oracle.codes(g)
    res = oracle.compare(cf, cg, *oracle.labels(cf), *oracle.labels(cg))
    bmf, bMf = bf.brute_labels(cf)
    bmg, bMg = bf.brute_labels(cg)
    want_wrong = int(np.count_nonzero((bmf != bmg) | (bMf != bMg)))
    isM = lambda c: (c & 15) == 15
    ism = lambda c: (c >> 4) == 15
    assert res["wrong_labels"] == want_wrong > 0
    assert res["fp_max"] == int(np.count_nonzero(isM(cg) & ~isM(cf))) >= 1
    assert res["fn_max"] == int(np.count_nonzero(isM(cf) & ~isM(cg)))
    assert res["fp_min"] == int(np.count_nonzero(ism(cg) & ~ism(cf))) >= 1
    assert res["fn_min"] == int(np.count_nonzero(ism(cf) & ~ism(cg)))
