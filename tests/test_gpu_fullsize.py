"""The configurations at their full sizes, in the launch configuration that
bench.py times, checked where the oracle can check them at that size:

- the exact error bound at every vertex (the oracle's own bound check) and
  g <= fhat everywhere;
- the oracle's steepest-neighbour codes of g against those of f, one vertex
  at a time, on a sample of edited vertices, their neighbours and random
  vertices;
- the edit list, in full: exactly the changed vertices, ascending, with
  delta = float32(g - fhat) bit for bit;
- the GPU verifier's wrong-label and false-extremum counts over the whole
  field (all zero).

Smaller cases of the same workloads are checked element by element against
the oracle's whole correction in test_gpu_parity.py and test_gpu_batch.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_01787_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_01787_gb300 import api as a
    a.load()
    return a


def _sample(n, shape, edit_idx, seed, count=6000):
    rng = np.random.default_rng(seed)
    picks = [rng.integers(0, n, count)]
    if edit_idx.size:
        e = edit_idx[rng.integers(0, edit_idx.size, count)].astype(np.int64)
        nz, ny, nx = shape
        # the edited vertices and a neighbour of each (x+-1, y+-1 or z+-1, clipped)
        step = np.array([1, -1, nx, -nx, nx * ny, -nx * ny])[rng.integers(0, 6, count)]
        picks += [e, np.clip(e + step, 0, n - 1)]
    picks.append(np.array([0, n - 1, shape[2] - 1, n - shape[2]]))
    return np.unique(np.concatenate(picks))


def check_corrected(api, fl, f_dev, out, edit_idx, edit_delta, count, seed=0):
    n = fl.n
    g = out.cpu().numpy()
    assert oracle.validate(fl.f, g, fl.xi) == oracle.OK  # |g - f| <= xi, exactly, everywhere
    assert bool((g <= fl.fhat).all())
    gi = g.view(np.uint32).ravel()
    hi = fl.fhat.view(np.uint32).ravel()
    changed = np.flatnonzero(gi != hi)
    assert count == changed.size
    idx = edit_idx[:count].cpu().numpy().view(np.uint32)
    assert np.array_equal(idx, changed.astype(np.uint32))
    delta = (g.ravel()[changed] - fl.fhat.ravel()[changed]).astype(np.float32)
    assert np.array_equal(edit_delta[:count].cpu().numpy().view(np.uint32), delta.view(np.uint32))
    for i in _sample(n, fl.shape, changed, seed):
        assert oracle.code_at(g, int(i)) == oracle.code_at(fl.f, int(i)), int(i)
    v = api.verify(f_dev, out)
    assert v["codes_equal"]
    assert (v["wrong_labels"], v["fp_max"], v["fn_max"], v["fp_min"], v["fn_min"]) == (0, 0, 0, 0, 0)


def _run_plain(api, fl, cap_div=4):
    f = torch.from_numpy(fl.f).cuda()
    fh = torch.from_numpy(fl.fhat).cuda()
    cap = fl.n // cap_div
    out = torch.empty_like(f)
    eidx = torch.empty(cap, dtype=torch.int32, device=f.device)
    edel = torch.empty(cap, dtype=torch.float32, device=f.device)
    r = api.correct(f, fh, fl.xi, out=out, edit_idx=eidx, edit_delta=edel, edit_capacity=cap)
    return f, fh, out, eidx, edel, r


def test_perlin_512_prequantized(api):
    fl = synth.perlin3d_prequant((512, 512, 512), seed=2, eb_rel=1e-4)
    f, fh, out, eidx, edel, r = _run_plain(api, fl)
    assert r.status == api.OK
    assert r.stats["sweeps"] >= 1 and r.stats["first_distorted"] > 0
    check_corrected(api, fl, f, out, eidx, edel, r.edit_count, seed=2)


def test_peaks_1024x1024x512(api):
    fl = synth.peaks3d((512, 1024, 1024), seed=3, eb_rel=1e-4)
    f, fh, out, eidx, edel, r = _run_plain(api, fl, cap_div=2)
    assert r.status == api.OK, api.status_str(r.status)
    assert r.stats["sweeps"] > 10
    check_corrected(api, fl, f, out, eidx, edel, r.edit_count, seed=3)


def test_learned_peaks_512(api):
    from paper_2601_01787_gb300 import learned
    net, _ = learned.default_net()
    fl = synth.peaks3d((512, 512, 512), seed=7, eb_rel=1e-4, npeaks=5000)
    f = torch.from_numpy(fl.f).cuda()
    fh = torch.from_numpy(fl.fhat).cuda()
    cap = fl.n // 2
    out = torch.empty_like(f)
    eidx = torch.empty(cap, dtype=torch.int32, device=f.device)
    edel = torch.empty(cap, dtype=torch.float32, device=f.device)
    lr = learned.correct_learned(f, fh, fl.xi, net, out=out, edit_idx=eidx, edit_delta=edel, edit_capacity=cap)
    assert lr.result.status == api.OK, api.status_str(lr.result.status)
    check_corrected(api, fl, f, out, eidx, edel, lr.result.edit_count, seed=7)
