"""Pins of the error bound (Sec. III-B, |f - g| <= xi) and of Eq. 1's edit."""
from fractions import Fraction

import numpy as np
import pytest

import oracle

F32_MAX = np.float32(np.finfo(np.float32).max)


def _exact(x) -> Fraction:
    return Fraction(float(x))


def _check_floor(f, xi):
    """L is the smallest finite float32 >= f - xi (exact real arithmetic)."""
    L = oracle.floor_bound(f, xi)
    e = _exact(f) - _exact(xi)
    assert _exact(L) >= e or L == -F32_MAX, (f, xi, L)
    if L > -F32_MAX:
        below = np.nextafter(L, np.float32(-np.inf), dtype=np.float32)
        assert _exact(below) < e, (f, xi, L)


def _check_ceil(f, xi):
    """U is the largest finite float32 <= f + xi."""
    U = oracle.ceil_bound(f, xi)
    e = _exact(f) + _exact(xi)
    assert _exact(U) <= e or U == F32_MAX, (f, xi, U)
    if U < F32_MAX:
        above = np.nextafter(U, np.float32(np.inf), dtype=np.float32)
        assert _exact(above) > e, (f, xi, U)


ADVERSARIAL = [
    (1.0, 1e-4), (0.5, 1e-4), (1e-30, 1e-4), (-1e-30, 1e-4), (1e-45, 1e-45), (3e-45, 1e-45),
    (0.0, 1e-4), (-0.0, 1e-5), (1e-4, 1e-4), (2.0, 2.0 ** -24), (2.0, 2.0 ** -23), (1.0, 2.0 ** -25),
    (1.0, 2.0 ** -24), (1.0, 3 * 2.0 ** -26), (1e20, 1.0), (-3e38, 1e38), (3e38, 1e38), (1e-38, 1e-39),
    (0.25, 0.0), (16777216.0, 1.0), (16777217.0, 0.5), (7.0, 1e-30)]


@pytest.mark.parametrize("f,xi", ADVERSARIAL)
def test_floor_ceil_exact_adversarial(f, xi):
    f, xi = np.float32(f), np.float32(xi)
    _check_floor(f, xi)
    _check_ceil(f, xi)


def test_floor_ceil_exact_random():
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2 ** 32, size=4000, dtype=np.uint64).astype(np.uint32)
    fs = bits.view(np.float32)
    xis = np.abs(rng.integers(0, 2 ** 32, size=4000, dtype=np.uint64).astype(np.uint32).view(np.float32))
    for f, xi in zip(fs, xis):
        if not (np.isfinite(f) and np.isfinite(xi)):
            continue
        _check_floor(f, xi)
        _check_ceil(f, xi)


def test_validate():
    f = np.array([0.5, 0.25, 0.0], dtype=np.float32)
    xi = np.float32(1e-3)
    assert oracle.validate(f, f, xi) == oracle.OK
    ok = np.array([oracle.floor_bound(v, xi) for v in f], dtype=np.float32)
    assert oracle.validate(f, ok, xi) == oracle.OK
    bad = ok.copy()
    bad[1] = np.nextafter(bad[1], np.float32(-1), dtype=np.float32)
    assert oracle.validate(f, bad, xi) == oracle.ERR_INPUT_BOUND
    up = np.array([oracle.ceil_bound(v, xi) for v in f], dtype=np.float32)
    assert oracle.validate(f, up, xi) == oracle.OK
    up[0] = np.nextafter(up[0], np.float32(2), dtype=np.float32)
    assert oracle.validate(f, up, xi) == oracle.ERR_INPUT_BOUND
    nan = f.copy()
    nan[2] = np.nan
    assert oracle.validate(f, nan, xi) == oracle.ERR_INPUT_BOUND
    assert oracle.validate(f, f, np.float32(-1.0)) == oracle.ERR_INVALID_ARG


@pytest.mark.parametrize("g,L", [(0.5, 0.4999), (1.0, -1.0), (1e-3, -1e-3), (0.3, 0.29999998), (5e-45, 0.0),
                                 (1.0, 0.99999994), (-2.0, -2.5)])
def test_halve_properties(g, L):
    """Eq. 1 with the HALVE step: strictly decreasing, never below the floor,
    within an ulp of the exact midpoint, and at the floor after finitely many steps."""
    g, L = np.float32(g), np.float32(L)
    steps = 0
    while True:
        h, changed = oracle.edit(g, L, oracle.RULE_HALVE)
        if not changed:
            assert h == g == L
            break
        assert L <= h < g
        mid = (_exact(g) + _exact(L)) / 2
        if h != L:
            ulp = abs(_exact(np.spacing(np.float32(max(abs(g), abs(L))))))
            assert abs(_exact(h) - mid) <= 2 * ulp
        g = h
        steps += 1
        assert steps < 400
    assert steps >= 1


def test_edit_at_floor_is_noop_and_snap_reaches_floor():
    h, ch = oracle.edit(np.float32(0.1), np.float32(0.1))
    assert not ch and h == np.float32(0.1)
    h, ch = oracle.edit(np.float32(0.7), np.float32(0.2), oracle.RULE_SNAP)
    assert ch and h == np.float32(0.2)
