"""The pipelined host-buffer entry points (msz_pipeline_*): a sequence of
fields whose copies overlap gives each field exactly the oracle's corrected
field, edit list and counts; the in-flight limit and an empty collect are
rejected; a field whose edit list does not fit reports MSZ_ERR_CAPACITY with
the needed count."""
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


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("shape", [(19, 23, 140), (12, 17, 45)])
def test_sequence_matches_the_oracle(api, shape):
    fields = [synth.perlin3d_prequant(shape, seed=60 + k, eb_rel=(1e-3, 1e-4)[k % 2]) if k % 3 else
              synth.peaks3d(shape, seed=60 + k, eb_rel=1e-4) for k in range(5)]
    refs = [oracle.correct(fl.f, fl.fhat, fl.xi) for fl in fields]
    pl = api.Pipeline(shape)
    bufs = []
    for k, fl in enumerate(fields):
        # result buffers: pinned (the device writes g and the edit list into
        # them) and, for one field, pageable (copied by the host API)
        if k == 1:
            res_bufs = (np.zeros(shape, np.float32), np.zeros(fl.n, np.uint32), np.zeros(fl.n, np.float32))
        else:
            res_bufs = (torch.empty(shape, dtype=torch.float32).pin_memory(),
                        torch.empty(fl.n, dtype=torch.int32).pin_memory(),
                        torch.empty(fl.n, dtype=torch.float32).pin_memory())
        bufs.append((_pinned(fl.f), _pinned(fl.fhat)) + res_bufs)
    got = []
    for k, (fl, b) in enumerate(zip(fields, bufs)):
        if k >= 2:
            got.append(pl.collect())
        pl.submit(b[0], b[1], fl.xi, b[2], b[3], b[4])
    got += [pl.collect(), pl.collect()]
    pl.close()
    def host(a):
        return a.numpy() if torch.is_tensor(a) else np.asarray(a)

    for fl, ref, res in zip(fields, refs, got):
        assert res.status == ref.status == api.OK
        assert np.array_equal(host(res.out).view(np.uint32), ref.g.view(np.uint32))
        assert res.edit_count == ref.edit_count
        assert np.array_equal(host(res.edit_idx).view(np.uint32), ref.edit_idx[:ref.edit_count])
        assert np.array_equal(host(res.edit_delta).view(np.uint32), ref.edit_delta[:ref.edit_count].view(np.uint32))
        assert (res.stats["sweeps"], res.stats["edits"], res.stats["first_distorted"]) == \
            (ref.sweeps, ref.edits, ref.first_distorted)


def test_in_flight_limit_and_empty_collect(api):
    shape = (8, 9, 10)
    fl = synth.perlin3d_prequant(shape, seed=70, eb_rel=1e-3)
    pl = api.Pipeline(shape)
    outs = [torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(3)]
    f, fh = _pinned(fl.f), _pinned(fl.fhat)
    pl.submit(f, fh, fl.xi, outs[0])
    pl.submit(f, fh, fl.xi, outs[1])
    with pytest.raises(api.MszError) as e:
        pl.submit(f, fh, fl.xi, outs[2])
    assert e.value.status == api.ERR_INVALID_ARG
    a, b = pl.collect(), pl.collect()
    assert a.status == b.status == api.OK
    assert torch.equal(outs[0].view(torch.int32), outs[1].view(torch.int32))
    with pytest.raises(api.MszError):
        pl.collect()
    pl.close()


def test_capacity_reported(api):
    shape = (16, 16, 16)
    fl = synth.peaks3d(shape, seed=71, eb_rel=1e-4)
    ref = oracle.correct(fl.f, fl.fhat, fl.xi)
    assert ref.edit_count > 4
    pl = api.Pipeline(shape, edit_capacity=4)
    out = torch.empty(shape, dtype=torch.float32).pin_memory()
    pl.submit(_pinned(fl.f), _pinned(fl.fhat), fl.xi, out)
    r = pl.collect()
    pl.close()
    assert r.status == api.ERR_CAPACITY and r.edit_count == ref.edit_count
    assert np.array_equal(out.numpy().view(np.uint32), ref.g.view(np.uint32))


def test_encoded_sequence_matches_the_oracle(api):
    """The encoded pipeline returns each field's edit list as a stream: byte
    for byte the oracle's encoding of the oracle's edits, and applied to fhat
    it gives the oracle's g."""
    from oracle import edits as E
    shape = (18, 21, 140)
    fields = [synth.perlin3d_prequant(shape, seed=80 + k, eb_rel=1e-4) if k % 2 else
              synth.peaks3d(shape, seed=80 + k, eb_rel=1e-4) for k in range(4)]
    refs = [oracle.correct(fl.f, fl.fhat, fl.xi) for fl in fields]
    pl = api.Pipeline(shape, encoded=True)
    # stream buffers: pinned (the device writes the stream into them) and
    # pageable (copied at collect)
    bufs = [(_pinned(fl.f), _pinned(fl.fhat),
             torch.empty(pl.stream_bound(), dtype=torch.uint8).pin_memory() if k % 3 != 1 else
             np.zeros(pl.stream_bound(), dtype=np.uint8))
            for k, fl in enumerate(fields)]
    got = []
    for k, (fl, b) in enumerate(zip(fields, bufs)):
        if k >= 2:
            got.append(pl.collect())
        pl.submit(b[0], b[1], fl.xi, b[2])
    got += [pl.collect(), pl.collect()]
    for fl, ref, res in zip(fields, refs, got):
        assert res.status == api.OK and res.edit_count == ref.edit_count
        want = E.encode(*E.edits_of(fl.fhat, ref.g))
        stream = res.stream if torch.is_tensor(res.stream) else torch.from_numpy(np.array(res.stream))
        assert stream.numpy().tobytes() == want
        field = torch.from_numpy(fl.fhat.copy()).cuda().reshape(-1)
        assert api.decode_edits(stream.cuda(), field) == ref.edit_count
        assert np.array_equal(field.cpu().numpy().view(np.uint32), ref.g.reshape(-1).view(np.uint32))
    # a field-mode call on an encoded pipeline is rejected
    import ctypes
    assert api.load().msz_pipeline_collect(pl._h, ctypes.byref(ctypes.c_int64()), None) == api.ERR_INVALID_ARG
    pl.close()


def test_encoded_stream_capacity(api):
    shape = (12, 14, 136)
    fl = synth.peaks3d(shape, seed=90, eb_rel=1e-4)
    ref = oracle.correct(fl.f, fl.fhat, fl.xi)
    assert ref.edit_count > 100
    pl = api.Pipeline(shape, encoded=True)
    for small in (torch.empty(64, dtype=torch.uint8).pin_memory(), np.zeros(64, dtype=np.uint8)):
        pl.submit(_pinned(fl.f), _pinned(fl.fhat), fl.xi, small)
        r = pl.collect()
        assert r.status == api.ERR_CAPACITY and r.edit_count == ref.edit_count
    pl.close()
