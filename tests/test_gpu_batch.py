"""msz_correct_batch: every field of one persistent launch gets exactly what a
separate correction gives -- checked against the oracle (small uneven batch)
and against msz_correct plus the GPU verifier (the full 64-field batch)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_01787_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available()
    from paper_2601_01787_gb300 import api as a
    a.load()
    return a


def _bits(t):
    a = t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else t
    return np.ascontiguousarray(a).view(np.uint32)


def _small_batch():
    fields = []
    for k, (shape, eb) in enumerate([((33, 47, 61), 1e-4), ((20, 20, 20), 1e-3), ((64, 40, 70), 1e-5),
                                     ((7, 130, 9), 1e-3), ((45, 33, 129), 1e-4)]):
        fields.append(synth.perlin3d_prequant(shape, seed=900 + k, eb_rel=eb, octaves=4))
    fields.append(synth.peaks3d((24, 31, 40), seed=950, eb_rel=1e-3, npeaks=12))
    return fields


@pytest.mark.parametrize("dense_min", [-1, 0, 1])
def test_batch_matches_oracle_per_field(api, dense_min):
    fields = _small_batch()
    fs = [torch.from_numpy(fl.f).cuda() for fl in fields]
    fhs = [torch.from_numpy(fl.fhat).cuda() for fl in fields]
    res = api.correct_batch(fs, fhs, [fl.xi for fl in fields], dense_min_items=dense_min, log_capacity=4096)
    assert res.status == api.OK
    for fl, r in zip(fields, res.fields):
        ref = oracle.correct(fl.f, fl.fhat, fl.xi, log_capacity=4096)
        assert r.status == ref.status
        assert np.array_equal(_bits(r.out), _bits(ref.g))
        assert r.edit_count == ref.edit_count
        assert np.array_equal(r.edit_idx.cpu().numpy().view(np.uint32), ref.edit_idx)
        assert np.array_equal(_bits(r.edit_delta), _bits(ref.edit_delta))
        st = r.stats
        assert (st["sweeps"], st["edits"], st["edited"], st["first_distorted"], st["left"]) == \
            (ref.sweeps, ref.edits, ref.edited, ref.first_distorted, ref.left)
        assert np.array_equal(r.sweep_log[:, 1:], ref.sweep_log[:, 1:])
        if dense_min == -1:
            assert np.array_equal(r.sweep_log[:, 0], ref.sweep_log[:, 0])
            assert st["examined"] == ref.examined


def test_batch_with_done_and_stuck_fields(api):
    good = synth.perlin3d_prequant((30, 30, 30), seed=960, eb_rel=1e-4)
    f_st = np.array([[[1.0000001, 1.0]]], dtype=np.float32)
    xi_st = np.float32(1e8)
    lo = np.array([oracle.floor_bound(v, xi_st) for v in f_st.reshape(-1)], dtype=np.float32).reshape(f_st.shape)
    cases = [(good.f, good.fhat, good.xi), (good.f, good.f.copy(), good.xi), (f_st, lo, xi_st)]
    res = api.correct_batch([torch.from_numpy(a).cuda() for a, _, _ in cases],
                            [torch.from_numpy(b).cuda() for _, b, _ in cases], [c for _, _, c in cases])
    assert res.status == api.OK
    for (f, fh, xi), r in zip(cases, res.fields):
        ref = oracle.correct(f, fh, xi)
        assert r.status == ref.status
        assert np.array_equal(_bits(r.out), _bits(ref.g))
        assert r.stats["sweeps"] == ref.sweeps and r.stats["left"] == ref.left


def test_batch_input_bound_is_reported_per_field(api):
    a = synth.perlin3d_prequant((16, 16, 16), seed=970, eb_rel=1e-3)
    b = synth.perlin3d_prequant((16, 17, 18), seed=971, eb_rel=1e-3)
    bad = b.fhat.copy()
    bad[3, 4, 5] = b.f[3, 4, 5] + np.float32(4) * b.xi
    res = api.correct_batch([torch.from_numpy(a.f).cuda(), torch.from_numpy(b.f).cuda()],
                            [torch.from_numpy(a.fhat).cuda(), torch.from_numpy(bad).cuda()], [a.xi, b.xi])
    assert res.status == api.ERR_INPUT_BOUND
    assert res.fields[1].status == api.ERR_INPUT_BOUND


def test_full_uneven_batch_matches_single_corrections(api):
    """The 64-field batch (axes uniform in 64..384, eb_rel in {1e-3,1e-4,1e-5},
    prequantized Perlin): each field equals its own msz_correct call, which the
    parity tests tie to the oracle, and verifies on the GPU."""
    fields = synth.batch(64)
    fs = [torch.from_numpy(fl.f).cuda() for fl in fields]
    fhs = [torch.from_numpy(fl.fhat).cuda() for fl in fields]
    res = api.correct_batch(fs, fhs, [fl.xi for fl in fields], edit_capacities=[fl.n // 4 for fl in fields])
    assert res.status == api.OK
    for fl, f, fh, r in zip(fields, fs, fhs, res.fields):
        one = api.correct(f, fh, fl.xi, edit_capacity=fl.n // 4)
        assert r.status == one.status == api.OK
        assert torch.equal(r.out.view(torch.int32), one.out.view(torch.int32))
        assert torch.equal(r.edit_idx, one.edit_idx)
        for key in ("sweeps", "edits", "edited", "first_distorted", "uncertified"):
            assert r.stats[key] == one.stats[key], key
        v = api.verify(f, r.out)
        assert v["codes_equal"] and v["wrong_labels"] == 0


def test_batch_graph_replay_matches_oracle(api):
    """The batch launch captured in a CUDA graph: every replay rebuilds g, the
    edit lists and the statuses from fhat, equal to the oracle's per field."""
    fields = _small_batch()
    fs = [torch.from_numpy(fl.f).cuda() for fl in fields]
    fhs = [torch.from_numpy(fl.fhat).cuda() for fl in fields]
    plan = api.BatchPlan(fs, fhs, [fl.xi for fl in fields])
    graph = plan.graph()
    refs = [oracle.correct(fl.f, fl.fhat, fl.xi, log_capacity=4096) for fl in fields]
    for rep in range(3):
        for r in plan.outputs:
            r[0].fill_(float("nan"))  # the replay must rewrite every output
        graph.replay()
        res = plan.collect(log_capacity=4096)
        assert res.status == api.OK
        for ref, r in zip(refs, res.fields):
            assert r.status == ref.status
            assert np.array_equal(_bits(r.out), _bits(ref.g))
            assert r.edit_count == ref.edit_count
            assert np.array_equal(r.edit_idx.cpu().numpy().view(np.uint32), ref.edit_idx)
            assert np.array_equal(_bits(r.edit_delta), _bits(ref.edit_delta))
            assert r.stats["sweeps"] == ref.sweeps
            assert np.array_equal(r.sweep_log[:, 1:], ref.sweep_log[:, 1:])
    plan.close()


def test_batch_plan_launch_matches_one_call(api):
    fields = _small_batch()
    fs = [torch.from_numpy(fl.f).cuda() for fl in fields]
    fhs = [torch.from_numpy(fl.fhat).cuda() for fl in fields]
    one = api.correct_batch(fs, fhs, [fl.xi for fl in fields], log_capacity=64)
    plan = api.BatchPlan(fs, fhs, [fl.xi for fl in fields])
    plan.launch()
    two = plan.collect(log_capacity=64)
    assert one.status == two.status == api.OK
    for a, b in zip(one.fields, two.fields):
        assert a.status == b.status and a.edit_count == b.edit_count
        assert np.array_equal(_bits(a.out), _bits(b.out))
        assert np.array_equal(a.sweep_log, b.sweep_log)
        assert {k: v for k, v in a.stats.items() if not k.endswith("_ns")} == \
            {k: v for k, v in b.stats.items() if not k.endswith("_ns")}


def test_batch_timeline(api):
    """The batch's timeline: one row per sweep the launch reached (detection
    end, edit end), non-decreasing, inside the kernels' time; -1 beyond."""
    fields = _small_batch()
    fs = [torch.from_numpy(fl.f).cuda() for fl in fields]
    fhs = [torch.from_numpy(fl.fhat).cuda() for fl in fields]
    cap = 64
    res = api.correct_batch(fs, fhs, [fl.xi for fl in fields], timeline_capacity=cap)
    assert res.status == api.OK and res.timeline.shape == (cap, 2)
    S = max(r.stats["sweeps"] for r in res.fields)
    assert 0 < S < cap - 1
    tl = res.timeline
    # sweeps 0 .. S-1 detect and edit; sweep S detects only (nothing left)
    seq = [t for q in range(S) for t in tl[q]] + [tl[S, 0]]
    assert all(t > 0 for t in seq) and seq == sorted(seq)
    assert tl[S, 1] == -1 and (tl[S + 1:] == -1).all()
    assert seq[-1] <= res.fields[0].stats["kernel_ns"]
    plan = api.BatchPlan(fs, fhs, [fl.xi for fl in fields], timeline_capacity=cap)
    plan.launch()
    two = plan.collect()
    assert two.status == api.OK and ((two.timeline > 0) == (tl > 0)).all()
    assert api.correct_batch(fs, fhs, [fl.xi for fl in fields]).timeline.shape == (0, 2)


def test_batch_at_the_field_limit(api):
    """MSZ_BATCH_MAX_FIELDS tiny uneven fields in one launch, each equal to its
    own correction; one more field is rejected."""
    n = api.BATCH_MAX_FIELDS
    shapes = [(2 + k % 5, 3 + k % 7, 5 + k % 11) for k in range(n)]
    fields = [synth.perlin3d_prequant(s, seed=3000 + k, eb_rel=1e-3, octaves=2) for k, s in enumerate(shapes)]
    fs = [torch.from_numpy(fl.f).cuda() for fl in fields]
    fhs = [torch.from_numpy(fl.fhat).cuda() for fl in fields]
    res = api.correct_batch(fs, fhs, [fl.xi for fl in fields])
    assert res.status == api.OK
    for k in range(0, n, 17):
        one = api.correct(fs[k], fhs[k], fields[k].xi)
        assert res.fields[k].status == one.status
        assert np.array_equal(_bits(res.fields[k].out), _bits(one.out))
    with pytest.raises(api.MszError):
        api.correct_batch(fs + fs[:1], fhs + fhs[:1], [fl.xi for fl in fields] + [fields[0].xi])
