"""Failure detection without a GPU fault: every device-side wait of the
correction kernel is bounded.  Test hook 1 makes block 0 wait at the first
grid barrier without arriving, so every block's wait runs out (0.25 s); hook
2 makes block 0 of the TMA-staged code pass withhold a plane copy, so its
mbarrier wait runs out.  The kernel records the timeout and returns, the host
reports MSZ_ERR_TIMEOUT, and the same context then corrects exactly as
before."""
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


def _bits(t):
    return np.ascontiguousarray(t.detach().cpu().numpy()).view(np.uint32)


@pytest.mark.parametrize("case", ["3d", "2d"])
def test_timeout_is_reported_and_the_context_stays_usable(api, case):
    fl = synth.perlin3d_prequant((40, 50, 60), seed=33, eb_rel=1e-3, octaves=4) if case == "3d" else \
        synth.perlin2d((71, 203), seed=31)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    bad = api.correct(f, fh, fl.xi, test_fault=1)
    assert bad.status == api.ERR_TIMEOUT
    # the context still works: a plain correction right after is exact
    good = api.correct(f, fh, fl.xi)
    ref = oracle.correct(fl.f, fl.fhat, fl.xi)
    assert good.status == ref.status
    assert np.array_equal(_bits(good.out), np.ascontiguousarray(ref.g).view(np.uint32))
    assert good.edit_count == ref.edit_count
    assert float(torch.ones(4, device="cuda").sum().item()) == 4.0


def test_static_entry_point_reports_the_timeout_too(api):
    fl = synth.perlin3d_prequant((20, 30, 40), seed=34, eb_rel=1e-3, octaves=4)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    out = torch.empty_like(f)
    lib = api.load()
    import ctypes
    opt, _ = api._options("halve", 0, 0, None, 0, 0, 1)
    cnt = ctypes.c_int64()
    st = lib.msz_correct_static(api._dptr(f), api._dptr(fh), ctypes.c_float(fl.xi), api.grid_of(f.shape),
                                api._dptr(out), None, None, 0, ctypes.byref(cnt), ctypes.byref(opt), None,
                                api._stream(None))
    assert st == api.ERR_TIMEOUT
    opt, _ = api._options("halve", 0, 0, None, 0)
    st = lib.msz_correct_static(api._dptr(f), api._dptr(fh), ctypes.c_float(fl.xi), api.grid_of(f.shape),
                                api._dptr(out), None, None, 0, ctypes.byref(cnt), ctypes.byref(opt), None,
                                api._stream(None))
    assert st in (api.OK, api.ERR_CAPACITY)
    ref = oracle.correct(fl.f, fl.fhat, fl.xi)
    assert np.array_equal(_bits(out), np.ascontiguousarray(ref.g).view(np.uint32))


def test_withheld_plane_copy_times_out_the_tma_ring(api):
    """Hook 2: block 0 of the TMA-staged code pass never issues its first plane
    copy, so its mbarrier wait runs out (0.25 s): the block records the
    timeout, waits for its other copies and leaves; the call reports
    MSZ_ERR_TIMEOUT and the next correction on the same context is exact."""
    fl = synth.perlin3d_prequant((256, 256, 256), seed=35, eb_rel=1e-4)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    bad = api.correct(f, fh, fl.xi, test_fault=2, edit_capacity=0)
    assert bad.status == api.ERR_TIMEOUT
    small = synth.perlin3d_prequant((24, 20, 140), seed=36, eb_rel=1e-4)  # also staged by TMA
    g = api.correct(torch.from_numpy(small.f).cuda(), torch.from_numpy(small.fhat).cuda(), small.xi)
    ref = oracle.correct(small.f, small.fhat, small.xi)
    assert g.status == ref.status == api.OK
    assert np.array_equal(_bits(g.out), np.ascontiguousarray(ref.g).view(np.uint32))
    again = api.correct(f, fh, fl.xi, edit_capacity=0)
    assert again.status in (api.OK, api.ERR_CAPACITY)
