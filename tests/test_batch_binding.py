"""Host-side marshalling of the batch entry points (no GPU): the msz_field
array points every field at its own tensors and at its own slice of the
shared edit-list buffers, and the results read back each field's status,
edit count, statistics and sweep log from that array."""
import numpy as np
import pytest
import torch

from paper_2601_01787_gb300 import api


@pytest.fixture
def host_ptrs(monkeypatch):
    # CPU tensors stand in for device tensors: only their addresses are used
    monkeypatch.setattr(api, "_dptr", lambda t: None if t is None else t.data_ptr())


def test_fields_point_at_their_buffers(host_ptrs):
    fs = [torch.zeros((3 + k % 4, 5, 9 + k)) for k in range(40)]
    fhs = [torch.ones_like(f) for f in fs]
    caps = [0 if k == 3 else 11 * k for k in range(40)]
    arr, (outs, idx_all, dl_all, offs, cps) = api._batch_fields(fs, fhs, [0.25 + k for k in range(40)], caps, None,
                                                               [k % 3 for k in range(40)])
    assert cps == caps and len(outs) == 40
    # every field's slice is disjoint from the next one, a zero capacity included
    assert offs == list(np.cumsum([0] + [max(c, 1) for c in caps[:-1]]))
    assert idx_all.numel() == dl_all.numel() == offs[-1] + max(caps[-1], 1)
    for k, fk in enumerate(arr):
        nz, ny, nx = fs[k].shape
        assert (fk.grid.ndim, fk.grid.nx, fk.grid.ny, fk.grid.nz) == (3, nx, ny, nz)
        assert (fk.d_f, fk.d_fhat, fk.d_out) == (fs[k].data_ptr(), fhs[k].data_ptr(), outs[k].data_ptr())
        assert fk.d_edit_idx == idx_all.data_ptr() + 4 * offs[k]
        assert fk.d_edit_delta == dl_all.data_ptr() + 4 * offs[k]
        assert fk.xi == np.float32(0.25 + k) and fk.status == -1 and fk.edit_capacity == caps[k]
        assert fk.tile_z == k % 3 and fk.edit_count == 0 and fk.stats.sweeps == 0


def test_results_read_each_field(host_ptrs):
    fs = [torch.zeros((4, 4, 4 + k)) for k in range(20)]
    caps = [5 * k for k in range(20)]
    arr, keep = api._batch_fields(fs, fs, [1.0] * 20, caps, None, None)
    for k, fk in enumerate(arr):  # what msz_batch_collect writes
        fk.status = api.OK if k % 3 else api.ERR_MAX_SWEEPS
        fk.edit_count = 7 * k  # above the capacity for k > 0: the list is cut there
        for j, name in enumerate(api._STATS_NAMES):
            setattr(fk.stats, name, 1000 * k + j)
        fk.stats.sweeps = k % 5
    cap = 6
    log = np.arange(4 * 20 * cap, dtype=np.int64)
    res = api._batch_results(arr, keep, log, cap, api.OK)
    assert res.status == api.OK and len(res.fields) == 20
    for k, r in enumerate(res.fields):
        assert r.status == arr[k].status and r.edit_count == 7 * k
        assert r.stats == arr[k].stats.as_dict()
        assert r.edit_idx.numel() == r.edit_delta.numel() == min(7 * k, caps[k])
        assert r.out is keep[0][k]
        if r.edit_idx.numel():  # (an empty slice has no address)
            assert r.edit_idx.data_ptr() == arr[k].d_edit_idx and r.edit_delta.data_ptr() == arr[k].d_edit_delta
        nlog = min(k % 5 + 1, cap)
        assert np.array_equal(r.sweep_log, log[4 * k * cap:4 * (k * cap + nlog)].reshape(-1, 4))
    # no log asked for: empty logs
    assert all(r.sweep_log.shape == (0, 4) for r in api._batch_results(arr, keep, log, 0, api.OK).fields)
