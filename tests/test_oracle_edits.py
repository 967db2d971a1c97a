"""Pins of the edit-list encoding oracle (oracle/edits.py).

What fixes it from outside itself: the ulp distance against repeated
np.nextafter steps, the value order of the key against numpy's float order, a
stream worked out by hand, the stream length from the widths alone, and the
defining property of a lossless encoding (decoding gives back g bit for bit)
on lists that cross block boundaries and use the extreme widths."""
import numpy as np
import pytest

from oracle import edits as E


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def test_ulp_distance_is_the_number_of_nextafter_steps():
    rng = np.random.default_rng(1)
    vals = np.concatenate([rng.uniform(-2, 2, 40), [0.0, -0.0, 1e-40, -1e-40, 1e-45, 1.0, -1.0, 3e38]])
    for v in vals.astype(np.float32):
        steps = int(rng.integers(1, 60))
        g = np.float32(v)
        for _ in range(steps):
            g = np.nextafter(g, np.float32(-np.inf), dtype=np.float32)
        fh = np.array([v], dtype=np.float32)
        idx, m = E.edits_of(fh, np.array([g], dtype=np.float32))
        # nextafter steps over -0 from a non-negative value to a negative one;
        # the key counts -0 as its own step
        extra = int(not np.signbit(v) and np.signbit(g))
        assert list(idx) == [0] and int(m[0]) == steps + extra


def test_key_follows_the_float_order():
    rng = np.random.default_rng(2)
    v = np.unique(np.concatenate([rng.standard_normal(500) * 10.0 ** rng.integers(-40, 38, 500),
                                  [np.inf, -np.inf, 1e-45, -1e-45]]).astype(np.float32))
    v = v[np.isfinite(v) | np.isinf(v)]
    k = E.ord_of(v)
    assert np.all(np.diff(k.astype(np.int64)) > 0)  # np.unique sorts by value
    assert E.ord_of(np.array([-0.0], np.float32))[0] + 1 == E.ord_of(np.array([0.0], np.float32))[0]
    assert np.array_equal(_bits(E.float_of(k)), _bits(v))


def test_stream_worked_by_hand():
    # edits at 3, 4, 9 with ulp distances 1, 2, 6: gaps d = 0, 0, 4 (3 bits),
    # m - 1 = 0, 1, 5 (3 bits); d packs to 4 << 6 = 0x100, m - 1 to
    # 1 << 3 | 5 << 6 = 0x148
    want = bytes.fromhex(
        "4d5a5345" "00010000" "0300000000000000"  # magic, B = 256, count = 3
        "03000000" "00000000"                     # first index 3, payload word 0
        "03" "03" "0000"                          # wd = 3, wm = 3, padding
        "00010000" "48010000")                    # d words, m - 1 words
    got = E.encode(np.array([3, 4, 9]), np.array([1, 2, 6]))
    assert got == want
    idx, m = E.decode(want)
    assert list(idx) == [3, 4, 9] and list(m) == [1, 2, 6]


def test_empty_list():
    s = E.encode(np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert len(s) == 16 and E.encoded_size(np.zeros(0), np.zeros(0)) == 16
    idx, m = E.decode(s)
    assert idx.size == 0 and m.size == 0


@pytest.mark.parametrize("count", [1, 2, 255, 256, 257, 600])
@pytest.mark.parametrize("kind", ["dense", "sparse", "extreme"])
def test_round_trip_and_length(count, kind):
    rng = np.random.default_rng(count * 7 + len(kind))
    if kind == "dense":
        gaps = rng.integers(1, 3, count)
        m = rng.integers(1, 5, count)
    elif kind == "sparse":
        gaps = rng.integers(1, 5000, count)
        m = rng.integers(1, 1 << 20, count)
    else:
        gaps = rng.integers(1, (1 << 31) // max(count, 1), count)
        m = rng.integers(1, 1 << 32, count, dtype=np.uint64)
        m[count // 2] = (1 << 32) - 1  # wm = 32
    idx = (np.cumsum(gaps) - 1).astype(np.uint64)
    assert idx[-1] < (1 << 31)
    s = E.encode(idx, m)
    assert len(s) == E.encoded_size(idx, m) and len(s) % 4 == 0
    i2, m2 = E.decode(s)
    assert np.array_equal(i2.astype(np.uint64), idx) and np.array_equal(m2.astype(np.uint64), m.astype(np.uint64))


def test_apply_recovers_g_bit_for_bit():
    rng = np.random.default_rng(3)
    fh = rng.uniform(-1, 1, 4000).astype(np.float32)
    fh[:4] = [0.0, -0.0, 1e-41, 5e-39]
    g = fh.copy()
    pick = rng.random(fh.size) < 0.3
    drop = rng.uniform(0, 1e-3, fh.size).astype(np.float32)
    g[pick] = (fh[pick] - drop[pick]).astype(np.float32)
    g[0] = -0.0   # +0 -> -0: equal values, different bits
    g[2] = -1e-42
    idx, m = E.edits_of(fh, g)
    assert np.all(m >= 1)
    out = E.apply(fh, *E.decode(E.encode(idx, m)))
    assert np.array_equal(_bits(out), _bits(g))


def test_length_of_a_uniform_list():
    # 3 blocks of 256 edits 3 apart with m = 1: d = 2 (wd = 2 bits, 16 words
    # a block), m - 1 = 0 (wm = 0, no words); the 30 table bytes pad to 32
    idx = np.arange(0, 3 * 256 * 3, 3, dtype=np.uint64)
    m = np.ones(idx.size, dtype=np.uint64)
    assert len(E.encode(idx, m)) == 16 + 32 + 3 * 16 * 4


def test_zero_distance_wraps_to_the_widest_field():
    # an index listed with g_i == fhat_i: m = 0, stored as (0 - 1) mod 2^32
    idx, m = np.array([5, 6]), np.array([0, 3])
    s = E.encode(idx, m)
    assert s[16 + 8 + 1] == 32  # wm
    i2, m2 = E.decode(s)
    assert list(i2) == [5, 6] and list(m2) == [0, 3]
