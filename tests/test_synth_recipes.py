"""The seeded synthetic inputs follow the recipes stated for them: fields
min-max scaled to [0, 1]; xi = float32(eb_rel * range) with the product in
double; fhat inside the exact bound (the oracle's check); prequantization to
multiples of 2 xi; uniform noise spanning +-xi; the peak density of the
1024 x 1024 x 512 workload; the 64-field batch's shapes and bounds; and
determinism (the same seed gives the same bytes, another seed other bytes)."""
import numpy as np
import pytest

import oracle
from paper_2601_01787_gb300 import synth


def _xi(f, eb_rel):
    return np.float32(eb_rel * (float(f.max()) - float(f.min())))


def test_perlin_prequantized():
    fl = synth.perlin3d_prequant((20, 33, 47), seed=2, eb_rel=1e-4)
    f, fh, xi = fl.f, fl.fhat, float(fl.xi)
    assert f.dtype == np.float32 and f.shape == (20, 33, 47) and fl.ndim == 3
    assert f.min() == 0.0 and f.max() == 1.0
    assert fl.xi == _xi(f, 1e-4)
    assert oracle.validate(f, fh, fl.xi) == oracle.OK
    # 2 xi * round(f / 2 xi) in double, ties to even; a value float32 rounding
    # pushed past the bound was moved back, so nearly all match exactly
    q = ((2.0 * xi) * np.rint(f.astype(np.float64) / (2.0 * xi))).astype(np.float32)
    assert np.mean(fh == q) > 0.999
    # plateaus: far fewer distinct values than f
    assert np.unique(fh).size * 4 < np.unique(f).size


@pytest.mark.parametrize("make, eb_rel", [
    (lambda: synth.peaks3d((16, 32, 48), seed=3), 1e-4),
    (lambda: synth.perlin2d((40, 56), seed=1), 1e-3),
])
def test_uniform_noise_spans_the_bound(make, eb_rel):
    fl = make()
    f, fh = fl.f, fl.fhat
    assert f.min() == 0.0 and f.max() == 1.0
    assert fl.xi == _xi(f, eb_rel)
    assert oracle.validate(f, fh, fl.xi) == oracle.OK
    d = (fh.astype(np.float64) - f) / float(fl.xi)
    assert d.min() < -0.99 and d.max() > 0.99        # U[-xi, xi], not a narrower band
    assert abs(d.mean()) < 0.05                       # centred
    assert 0.25 < np.mean(np.abs(d) < 0.5) < 0.75     # flat: half the mass within xi / 2


def test_peak_density():
    # 20,000 peaks at 1024 x 1024 x 512; 5,000 at 512^3; 78 per 128^3 training field
    assert round(synth.DEFAULT_PEAK_DENSITY * 1024 * 1024 * 512) == 20000
    assert round(synth.DEFAULT_PEAK_DENSITY * 512 ** 3) == 5000
    assert round(synth.DEFAULT_PEAK_DENSITY * 128 ** 3) == 78


def test_batch_recipe():
    bs = synth.batch_shapes(64)
    assert len(bs) == 64
    for k, (shape, eb, seed) in enumerate(bs):
        assert len(shape) == 3 and all(64 <= a <= 384 for a in shape)
        assert eb in (1e-3, 1e-4, 1e-5) and seed == 1000 + k
    assert {eb for _, eb, _ in bs} == {1e-3, 1e-4, 1e-5}
    # the workload the batch benchmark reports (747,917,344 vertices)
    assert sum(int(np.prod(s)) for s, _, _ in bs) == 747917344
    assert synth.batch_shapes(64) == bs


def test_determinism():
    a = synth.perlin((8, 16, 24), seed=5)
    assert a.tobytes() == synth.perlin((8, 16, 24), seed=5).tobytes()
    assert a.tobytes() != synth.perlin((8, 16, 24), seed=6).tobytes()
    p = synth.peaks((8, 16, 24), npeaks=3, seed=9)
    assert p.tobytes() == synth.peaks((8, 16, 24), npeaks=3, seed=9).tobytes()
    u = synth.uniform(100000, seed=1)
    assert np.array_equal(u, synth.uniform(100000, seed=1))
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    assert not np.array_equal(u, synth.uniform(100000, seed=1, stream=1))
