"""msz_correct_static: the correction for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Checked through the
C ABI against msz_correct, on two calls in a row.  This file is collected last
on purpose, and it depends on no other test module's state."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2601_01787_gb300 import synth

pytestmark = pytest.mark.gpu


def _static_call(lib, api, f, fh, xi, cap):
    out = torch.empty_like(f)
    idx = torch.empty(max(cap, 1), dtype=torch.int32, device=f.device)
    dl = torch.empty(max(cap, 1), dtype=torch.float32, device=f.device)
    cnt = ctypes.c_int64()
    stats = api.Stats()
    opt = api.Options(0, 0, 0, 0, None, None, 0, None)
    st = lib.msz_correct_static(f.data_ptr(), fh.data_ptr(), ctypes.c_float(np.float32(xi)), api.grid_of(f.shape),
                                out.data_ptr(), idx.data_ptr(), dl.data_ptr(), cap, ctypes.byref(cnt),
                                ctypes.byref(opt), ctypes.byref(stats), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    m = min(int(cnt.value), cap)
    return st, out, idx[:m], dl[:m], int(cnt.value), stats.as_dict()


@pytest.mark.parametrize("make", [
    lambda: synth.perlin3d_prequant((96, 100, 120), seed=71, eb_rel=1e-4),
    lambda: synth.peaks3d((40, 64, 64), seed=72, eb_rel=1e-3, npeaks=20),
    lambda: synth.perlin2d((300, 500), seed=73),
], ids=["perlin3d", "peaks3d", "perlin2d"])
def test_static_matches_workspace_entry_point(make):
    assert torch.cuda.is_available()
    from paper_2601_01787_gb300 import api
    lib = api.load()
    fl = make()
    f = torch.from_numpy(fl.f).cuda()
    fh = torch.from_numpy(fl.fhat).cuda()
    ref = api.correct(f, fh, fl.xi)
    assert ref.status == api.OK
    for _ in range(2):   # the shared array keeps the previous call's contents
        st, out, idx, dl, cnt, stats = _static_call(lib, api, f, fh, fl.xi, fl.n)
        assert st == api.OK, api.status_str(st)
        assert torch.equal(out.view(torch.int32), ref.out.view(torch.int32))
        assert cnt == ref.edit_count
        assert torch.equal(idx, ref.edit_idx)
        assert torch.equal(dl.view(torch.int32), ref.edit_delta.view(torch.int32))
        for key in ("sweeps", "edits", "edited", "first_distorted", "left", "examined", "dense_sweeps"):
            assert stats[key] == ref.stats[key], key


def test_static_rejects_grids_above_its_limit():
    from paper_2601_01787_gb300 import api
    lib = api.load()
    f = torch.zeros(1, dtype=torch.float32, device="cuda")
    cnt = ctypes.c_int64()
    big = api.Grid(3, 0, 256, 256, 65)   # 4,259,840 > MSZ_STATIC_MAX_VERTICES vertices
    st = lib.msz_correct_static(f.data_ptr(), f.data_ptr(), ctypes.c_float(0.1), big, f.data_ptr(), None, None, 0,
                                ctypes.byref(cnt), None, None, None)
    assert st == api.ERR_WORKSPACE
