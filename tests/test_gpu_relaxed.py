"""msz_correct_relaxed (the relaxed synchronization of Sec. IV-B on one GPU)
against the CPU oracle orc_correct_relaxed with the same 8 x 8 x 32 tiles:
bit-exact corrected field and edit list, the same statuses and the same
iteration, local-sweep and tile-run counts."""
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


def _bits(a):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return np.ascontiguousarray(a).view(np.uint32)


CASES = {
    "peaks_ragged": lambda: synth.peaks3d((21, 37, 70), seed=41, eb_rel=1e-4),
    "peaks_dense": lambda: synth.peaks3d((24, 32, 96), seed=42, eb_rel=1e-4, npeaks=40),
    "perlin_prequant": lambda: synth.perlin3d_prequant((30, 44, 65), seed=43, eb_rel=1e-3, octaves=4),
    "thin": lambda: synth.peaks3d((3, 5, 33), seed=44, eb_rel=1e-3, npeaks=2),
}


@pytest.mark.parametrize("name", list(CASES))
def test_relaxed_matches_oracle(api, name):
    fl = CASES[name]()
    st_ref, g_ref, s_ref = oracle.correct_relaxed(fl.f, fl.fhat, fl.xi, api.RELAXED_TILE)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    r = api.correct_relaxed(f, fh, fl.xi, log_capacity=4096)
    assert r.status == st_ref
    assert np.array_equal(_bits(r.out), _bits(g_ref))
    st = r.stats
    assert (st["sweeps"], st["local_sweeps"], st["edited"], st["first_distorted"], st["left"], st["tile_runs"]) == \
        tuple(int(v) for v in (s_ref[0], s_ref[1], s_ref[2], s_ref[3], s_ref[4], s_ref[5]))
    changed = np.flatnonzero(_bits(g_ref).ravel() != _bits(fl.fhat).ravel())
    assert np.array_equal(r.edit_idx.cpu().numpy().view(np.uint32), changed.astype(np.uint32))
    delta = (g_ref.ravel()[changed] - fl.fhat.ravel()[changed]).astype(np.float32)
    assert np.array_equal(_bits(r.edit_delta), delta.view(np.uint32))
    assert r.sweep_log.shape[0] == st["sweeps"] + 1 and r.sweep_log[:, 0].sum() == st["tile_runs"]
    v = api.verify(f, r.out)
    assert v["codes_equal"] and v["wrong_labels"] == 0


def test_relaxed_caps_and_correct_input(api):
    fl = CASES["peaks_dense"]()
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    r = api.correct_relaxed(f, fh, fl.xi, max_iters=1)
    st_ref, g_ref, s_ref = oracle.correct_relaxed(fl.f, fl.fhat, fl.xi, api.RELAXED_TILE, max_iters=1)
    assert r.status == st_ref
    assert np.array_equal(_bits(r.out), _bits(g_ref))
    r = api.correct_relaxed(f, fh, fl.xi, local_cap=2)
    st_ref, g_ref, s_ref = oracle.correct_relaxed(fl.f, fl.fhat, fl.xi, api.RELAXED_TILE, local_cap=2)
    assert r.status == st_ref and r.stats["local_sweeps"] == s_ref[1] and r.stats["sweeps"] == s_ref[0]
    assert np.array_equal(_bits(r.out), _bits(g_ref))
    r = api.correct_relaxed(f, f, fl.xi)
    assert r.status == api.OK and r.stats["sweeps"] == 0 and r.edit_count == 0


def test_relaxed_plain_agree_on_invariants(api):
    """Both schedules end in fields with the codes and labels of f; the relaxed
    one in fewer global iterations than the synchronous loop has sweeps."""
    fl = synth.peaks3d((48, 64, 96), seed=45, eb_rel=1e-4)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    p = api.correct(f, fh, fl.xi)
    r = api.correct_relaxed(f, fh, fl.xi)
    assert p.ok and r.ok
    assert r.stats["sweeps"] < p.stats["sweeps"]
    for g in (p.out, r.out):
        v = api.verify(f, g)
        assert v["codes_equal"] and v["wrong_labels"] == 0
