"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: bit-exact for codes, labels, counts, the corrected float field, the edit
list and every per-sweep count (the loop is deterministic Jacobi with IEEE
round-to-nearest arithmetic on both sides)."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bits(t):
    a = t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else t
    return np.ascontiguousarray(a).view(np.uint32)


# ----------------------------------------------------------------- codes
@pytest.mark.parametrize("shape,levels,seed", [
    ((37, 53), 4, 0), ((7, 9, 11), 3, 1), ((33, 65, 130), 1000, 2), ((1, 1, 1), 1, 3), ((1, 40), 3, 4),
    ((40, 1), 3, 5), ((5, 1, 7), 2, 6), ((1, 6, 9), 2, 7), ((64, 1, 1), 5, 8), ((17, 31, 129), 2, 9)])
def test_directions_bit_exact(api, shape, levels, seed):
    rng = np.random.default_rng(seed)
    v = (rng.integers(0, levels, size=shape) / max(levels - 1, 1)).astype(np.float32)
    got = api.directions(dev(v)).cpu().numpy()
    assert np.array_equal(got, oracle.codes(v))


def test_directions_signed_zero_and_extremes(api):
    v = np.array([[0.0, -0.0, 1e-45, -1e-45], [3.4e38, -3.4e38, 0.0, -0.0]], dtype=np.float32)
    assert np.array_equal(api.directions(dev(v)).cpu().numpy(), oracle.codes(v))


# ------------------------------------------------------------ correction
CASES = {
    "perlin2d_256": lambda: synth.perlin2d((256, 256), seed=1),
    "perlin2d_ragged": lambda: synth.perlin2d((71, 203), seed=31),
    "perlin3d_prequant_ragged": lambda: synth.perlin3d_prequant((45, 67, 133), seed=32, eb_rel=1e-4),
    "perlin3d_prequant_coarse": lambda: synth.perlin3d_prequant((40, 50, 60), seed=33, eb_rel=1e-3, octaves=4),
    "peaks3d_small": lambda: synth.peaks3d((33, 41, 57), seed=34, eb_rel=1e-4),
    "peaks3d_flat": lambda: synth.peaks3d((16, 16, 16), seed=35, eb_rel=1e-3, npeaks=2),
    # x extents that are multiples of 4 and at least 136 wide: the code pass
    # stages these by TMA (ragged last tiles in x and y; the smallest box)
    "perlin3d_tma_ragged": lambda: synth.perlin3d_prequant((37, 13, 140), seed=36, eb_rel=1e-4),
    "peaks3d_tma": lambda: synth.peaks3d((21, 26, 264), seed=37, eb_rel=1e-4),
    "perlin3d_tma_min": lambda: synth.perlin3d_prequant((5, 10, 136), seed=38, eb_rel=1e-3),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    fl = CASES[request.param]()
    ref = oracle.correct(fl.f, fl.fhat, fl.xi, log_capacity=100000)
    assert ref.status == oracle.OK
    return fl, ref


def _check_against(res, ref, fl, worklist_column: bool):
    assert res.status == ref.status
    assert np.array_equal(bits(res.out), bits(ref.g))
    assert res.edit_count == ref.edit_count
    assert np.array_equal(res.edit_idx.cpu().numpy().view(np.uint32), ref.edit_idx)
    assert np.array_equal(bits(res.edit_delta), bits(ref.edit_delta))
    st = res.stats
    assert (st["sweeps"], st["edits"], st["edited"], st["first_distorted"], st["left"]) == \
        (ref.sweeps, ref.edits, ref.edited, ref.first_distorted, ref.left)
    assert np.array_equal(res.sweep_log[:, 1:], ref.sweep_log[:, 1:])
    if worklist_column:
        assert np.array_equal(res.sweep_log[:, 0], ref.sweep_log[:, 0])
        assert st["examined"] == ref.examined


def test_correct_worklist_only_bit_exact(api, case):
    fl, ref = case
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, dense_min_items=-1, log_capacity=100000)
    _check_against(res, ref, fl, worklist_column=True)
    assert res.stats["dense_sweeps"] == 1


def test_correct_default_bit_exact(api, case):
    fl, ref = case
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, log_capacity=100000)
    _check_against(res, ref, fl, worklist_column=False)


def test_correct_always_dense_bit_exact(api, case):
    fl, ref = case
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, dense_min_items=1, log_capacity=100000)
    _check_against(res, ref, fl, worklist_column=False)
    assert res.stats["dense_sweeps"] == res.stats["sweeps"] + 1


def test_correct_mixed_dense_then_worklist_bit_exact(api, case):
    """Whole-grid scans while many vertices are distorted, then the worklist."""
    fl, ref = case
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, dense_min_items=max(1, fl.n // 16), log_capacity=100000)
    _check_against(res, ref, fl, worklist_column=False)


def test_correct_is_deterministic_across_calls(api, case):
    fl, ref = case
    f, fh = dev(fl.f), dev(fl.fhat)
    a = api.correct(f, fh, fl.xi)
    b = api.correct(f, fh, fl.xi)
    assert np.array_equal(bits(a.out), bits(b.out))
    assert torch.equal(a.edit_idx, b.edit_idx)


def test_corrected_field_verifies_on_gpu(api, case):
    """Sec. IV-A / Sec. V-C: after correction the GPU's own codes and labels of g
    equal those of f: zero wrong labels and zero false extrema."""
    fl, ref = case
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi)
    v = api.verify(dev(fl.f), res.out)
    assert v["codes_equal"]
    assert (v["wrong_labels"], v["fp_max"], v["fn_max"], v["fp_min"], v["fn_min"]) == (0, 0, 0, 0, 0)


def test_snap_rule_bit_exact(api):
    fl = synth.perlin3d_prequant((30, 31, 65), seed=40, eb_rel=1e-4)
    ref = oracle.correct(fl.f, fl.fhat, fl.xi, rule=oracle.RULE_SNAP, log_capacity=1000)
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, rule="snap", log_capacity=1000)
    _check_against(res, ref, fl, worklist_column=False)


@pytest.mark.parametrize("shape", [(24, 35, 47), (20, 17, 144)])
def test_g_init_bit_exact(api, shape):
    fl = synth.perlin3d_prequant(shape, seed=41, eb_rel=1e-4)
    lo = np.array([oracle.floor_bound(a, fl.xi) for a in fl.f.reshape(-1)], dtype=np.float32).reshape(fl.shape)
    r = synth.uniform(fl.n, seed=41).reshape(fl.shape)
    g0 = np.maximum(lo, (fl.fhat.astype(np.float64) - 0.5 * r * (fl.fhat - lo)).astype(np.float32))
    ref = oracle.correct(fl.f, fl.fhat, fl.xi, g_init=g0, log_capacity=1000)
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, g_init=dev(g0), log_capacity=1000)
    _check_against(res, ref, fl, worklist_column=False)


def _unaligned(a):
    # a copy whose data starts 4 bytes past a 16-byte boundary
    buf = torch.empty(a.size + 4, dtype=torch.float32, device="cuda")
    v = buf[1:1 + a.size].view(a.shape)
    v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    assert v.data_ptr() % 16 == 4
    return v


@pytest.mark.parametrize("dense", [-1, 1])
@pytest.mark.parametrize("shape", [(37, 13, 140), (9, 24, 392)])
def test_tma_and_cp_async_staging_agree(api, shape, dense):
    """16-byte aligned arrays take the TMA-staged passes, unaligned ones the
    cp.async code pass and gathered detection: under one detection schedule
    (worklists only, or whole-grid scans only) the same result, edit list and
    per-sweep records."""
    fl = synth.peaks3d(shape, seed=42, eb_rel=1e-4)
    a = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, log_capacity=1000, dense_min_items=dense)
    b = api.correct(_unaligned(fl.f), _unaligned(fl.fhat), fl.xi, log_capacity=1000, dense_min_items=dense)
    assert a.status == b.status == api.OK
    assert np.array_equal(bits(a.out), bits(b.out))
    assert np.array_equal(a.edit_idx.cpu().numpy(), b.edit_idx.cpu().numpy())
    assert np.array_equal(a.sweep_log, b.sweep_log)
    assert {k: v for k, v in a.stats.items() if not k.endswith("_ns")} == \
        {k: v for k, v in b.stats.items() if not k.endswith("_ns")}


# ----------------------------------------------------- edges and errors
@pytest.mark.parametrize("shape", [(1, 1), (1, 1, 1), (1, 2), (2, 1), (1, 1, 5), (1, 7, 1), (3, 1, 1), (2, 2, 2),
                                   (1, 33), (33, 1, 2),
                                   # thin grids staged by TMA: one or two planes, the smallest box
                                   (1, 12, 140), (2, 10, 136), (1, 10, 264)])
def test_degenerate_grids(api, shape):
    rng = np.random.default_rng(sum(shape))
    f = rng.integers(0, 3, size=shape).astype(np.float32) / np.float32(4)
    xi = np.float32(0.2)
    fhat = (f + rng.uniform(-0.19, 0.19, size=shape)).astype(np.float32)
    ref = oracle.correct(f, fhat, xi, log_capacity=1000)
    res = api.correct(dev(f), dev(fhat), xi, log_capacity=1000)
    _check_against(res, ref, None, worklist_column=False)


def test_constant_field_all_ties(api):
    f = np.full((9, 10, 11), 0.5, dtype=np.float32)
    xi = np.float32(1e-3)
    fhat = synth.perturb_uniform(f, xi, seed=3)
    ref = oracle.correct(f, fhat, xi, log_capacity=100000)
    res = api.correct(dev(f), dev(fhat), xi, log_capacity=100000)
    _check_against(res, ref, None, worklist_column=False)


def test_already_correct_needs_no_sweep(api):
    fl = synth.perlin2d((50, 60), seed=5)
    res = api.correct(dev(fl.f), dev(fl.f), fl.xi)
    assert res.status == api.OK and res.stats["sweeps"] == 0 and res.edit_count == 0


def test_stuck_reported(api):
    f = np.array([[1.0000001, 1.0]], dtype=np.float32)
    xi = np.float32(1e8)
    L = np.array([oracle.floor_bound(v, xi) for v in f.reshape(-1)], dtype=np.float32).reshape(f.shape)
    ref = oracle.correct(f, L.copy(), xi)
    res = api.correct(dev(f), dev(L), xi)
    assert ref.status == oracle.STUCK and res.status == api.STUCK
    assert res.stats["left"] == ref.left and res.stats["sweeps"] == ref.sweeps


def test_max_sweeps_and_capacity(api):
    fl = synth.perlin2d((64, 80), seed=6)
    ref = oracle.correct(fl.f, fl.fhat, fl.xi, max_sweeps=2)
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, max_sweeps=2)
    assert ref.status == oracle.ERR_MAX_SWEEPS == res.status
    assert np.array_equal(bits(res.out), bits(ref.g))
    assert res.stats["left"] == ref.left
    full = oracle.correct(fl.f, fl.fhat, fl.xi)
    small = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, edit_capacity=5)
    assert small.status == api.ERR_CAPACITY and small.edit_count == full.edit_count
    assert np.array_equal(small.edit_idx.cpu().numpy().view(np.uint32), full.edit_idx[:5])
    assert np.array_equal(bits(small.out), bits(full.g))
    none = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, edit_capacity=0)
    assert none.status == api.ERR_CAPACITY and none.edit_count == full.edit_count


@pytest.mark.parametrize("shape", [(20, 30), (6, 12, 60), (6, 12, 140)])  # 2D, cp.async, TMA staging
def test_input_bound_violations(api, shape):
    fl = synth.perlin2d(shape, seed=7) if len(shape) == 2 else synth.perlin3d_prequant(shape, seed=7, eb_rel=1e-3)
    at = (3, 4) if len(shape) == 2 else (2, 3, 4)
    bad = fl.fhat.copy()
    bad[at] = fl.f[at] + np.float32(3) * fl.xi
    assert api.correct(dev(fl.f), dev(bad), fl.xi).status == api.ERR_INPUT_BOUND
    for value in (np.nan, np.inf, -np.inf):
        odd = fl.fhat.copy()
        odd[at] = value
        assert api.correct(dev(fl.f), dev(odd), fl.xi).status == api.ERR_INPUT_BOUND
        if len(shape) == 3:
            g0 = fl.fhat.copy()
            g0[at] = value  # an unusable proposed start
            assert api.correct(dev(fl.f), dev(fl.fhat), fl.xi, g_init=dev(g0)).status == api.ERR_INPUT_BOUND
    inf = fl.f.copy()
    inf[at] = np.inf
    assert api.correct(dev(inf), dev(fl.fhat), fl.xi).status == api.ERR_INPUT_BOUND
    # exactly at the floor and ceiling is valid
    lo = np.array([oracle.floor_bound(a, fl.xi) for a in fl.f.reshape(-1)], dtype=np.float32).reshape(fl.shape)
    hi = np.array([oracle.ceil_bound(a, fl.xi) for a in fl.f.reshape(-1)], dtype=np.float32).reshape(fl.shape)
    mix = np.where(np.arange(fl.n).reshape(fl.shape) % 2 == 0, lo, hi).astype(np.float32)
    ref = oracle.correct(fl.f, mix, fl.xi)
    res = api.correct(dev(fl.f), dev(mix), fl.xi)
    assert ref.status == res.status == api.OK
    assert np.array_equal(bits(res.out), bits(ref.g))
    # a context that saw input errors keeps working
    ok = api.correct(dev(fl.f), dev(fl.fhat), fl.xi)
    assert ok.status == api.OK


def test_floor_matches_oracle_on_adversarial_values(api):
    """The device floor (one round-up subtraction) equals the oracle's exact floor:
    fhat at the oracle floor is accepted, one ulp below is rejected."""
    f = np.array([[1e-30, -1e-30, 1.0, 0.5, 3e-45, 7.0, 0.25, 1e20]], dtype=np.float32)
    xi = np.float32(1e-4)
    lo = np.array([oracle.floor_bound(a, xi) for a in f.reshape(-1)], dtype=np.float32).reshape(f.shape)
    assert api.correct(dev(f), dev(lo), xi).status in (api.OK, api.STUCK)
    for k in range(f.size):
        below = lo.copy()
        below.reshape(-1)[k] = np.nextafter(lo.reshape(-1)[k], np.float32(-np.inf))
        assert api.correct(dev(f), dev(below), xi).status == api.ERR_INPUT_BOUND


# ------------------------------------------------------------ labels
@pytest.mark.parametrize("shape,seed", [((45, 67, 133), 50), ((256, 256), 51), ((1, 1, 9), 52), ((3, 1, 4), 53)])
def test_segment_labels_and_compare(api, shape, seed):
    if len(shape) == 2:
        fl = synth.perlin2d(shape, seed=seed)
    else:
        fl = synth.perlin3d_prequant(shape, seed=seed, eb_rel=1e-4, octaves=3)
    cf, ch = oracle.codes(fl.f), oracle.codes(fl.fhat)
    mnf, mxf = oracle.labels(cf)
    mnh, mxh = oracle.labels(ch)
    gcf = api.directions(dev(fl.f))
    gch = api.directions(dev(fl.fhat))
    a, b = api.segment(gcf)
    c, d = api.segment(gch)
    assert np.array_equal(a.cpu().numpy(), mnf) and np.array_equal(b.cpu().numpy(), mxf)
    assert np.array_equal(c.cpu().numpy(), mnh) and np.array_equal(d.cpu().numpy(), mxh)
    got = api.compare(gcf, gch, a, b, c, d)
    assert got.pop("code_mismatches") == int((cf != ch).sum())
    assert got == oracle.compare(cf, ch, mnf, mxf, mnh, mxh)


def test_segment_rejects_codes_outside_grid(api):
    codes = torch.full((3, 4, 5), 0x00, dtype=torch.uint8, device="cuda")  # slot 0 at x = nx-1 leaves the grid
    with pytest.raises(api.MszError):
        api.segment(codes)


# ------------------------------------------------------- host buffers
@pytest.mark.parametrize("memory", ["pinned", "pageable"])
@pytest.mark.parametrize("shape", [(31, 47, 70), (53, 91)])
def test_correct_host_matches_oracle(api, memory, shape):
    """Host entry point with pinned and with pageable host buffers: both give
    the oracle's result."""
    fl = synth.perlin3d_prequant(shape, seed=60, eb_rel=1e-4) if len(shape) == 3 else \
        synth.perlin2d(shape, seed=61)
    ref = oracle.correct(fl.f, fl.fhat, fl.xi)
    if memory == "pinned":
        f = torch.from_numpy(fl.f).pin_memory()
        fh = torch.from_numpy(fl.fhat).pin_memory()
    else:
        f, fh = fl.f.copy(), fl.fhat.copy()
    res = api.correct_host(f, fh, fl.xi)
    assert res.status == ref.status
    assert np.array_equal(bits(res.out), bits(ref.g))
    assert np.array_equal(res.edit_idx, ref.edit_idx) and np.array_equal(bits(res.edit_delta), bits(ref.edit_delta))


@pytest.mark.parametrize("dense_min", [-1, 0, 1], ids=["worklist_only", "default", "always_dense"])
@pytest.mark.parametrize("name", list(CASES))
def test_below_reference_rule_bit_exact(api, name, dense_min):
    """BELOW_REFERENCE (Sec. IV-A 'to 0.3 or slightly below'): the whole loop,
    per-sweep counts included, against the oracle's BELOW rule."""
    fl = CASES[name]()
    ref = oracle.correct(fl.f, fl.fhat, fl.xi, rule=oracle.RULE_BELOW, log_capacity=100000)
    assert ref.status == oracle.OK
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, rule="below", dense_min_items=dense_min,
                      log_capacity=100000)
    _check_against(res, ref, fl, worklist_column=dense_min == -1)


def test_below_reference_needs_its_workspace(api):
    fl = synth.perlin3d_prequant((20, 21, 22), seed=41, eb_rel=1e-4)
    lib = api.load()
    need = lib.msz_workspace_size_rule(api.grid_of(fl.shape), 2)
    assert need > api.workspace_size(fl.shape)
    ws = torch.empty(api.workspace_size(fl.shape), dtype=torch.uint8, device="cuda")
    res = api.correct(dev(fl.f), dev(fl.fhat), fl.xi, rule="below", ws=ws)
    assert res.status == api.ERR_WORKSPACE


# ------------------------------------------------------ per-kernel events
@pytest.mark.parametrize("shape", [(24, 20, 136), (21, 30, 45), (67, 91)], ids=["tma", "cp_async", "2d"])
def test_phase_events_bracket_each_kernel(api, shape):
    """The three timing events of msz_options: recorded around sweep 0's
    kernel and the loop kernel, without changing the result; an entry left
    null is skipped."""
    fl = (synth.perlin3d_prequant(shape, seed=61, eb_rel=1e-4) if len(shape) == 3
          else synth.perlin2d(shape, seed=61))
    f, fh = dev(fl.f), dev(fl.fhat)
    ref = api.correct(f, fh, fl.xi)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    res = api.correct(f, fh, fl.xi, events=ev)
    torch.cuda.synchronize()
    assert res.status == ref.status == api.OK
    assert np.array_equal(bits(res.out), bits(ref.out))
    assert np.array_equal(res.edit_idx.cpu().numpy(), ref.edit_idx.cpu().numpy())
    t_codes, t_loop = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    assert t_loop > 0.0
    if len(shape) == 3:
        assert t_codes > 0.0
    else:
        assert 0.0 <= t_codes < t_loop  # one kernel: [0] and [1] both before it
    part = [None, torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
    res2 = api.correct(f, fh, fl.xi, events=part)
    torch.cuda.synchronize()
    assert res2.status == api.OK and part[1].elapsed_time(part[2]) > 0.0
