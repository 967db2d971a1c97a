"""GPU parity of the edit-list encoding (msz_edits_encode / msz_edits_decode)
with the oracle's format (oracle/edits.py): the stream byte for byte, and the
field decoding gives back bit for bit.

- the oracle's own correction of small fields: its edits encoded by the
  oracle, those of the GPU correction encoded by the GPU -- equal streams;
- synthetic edit lists over several blocks with a ragged last block, gaps up
  to 2^30, ulp distances up to 2^32 - 1 and 0 (an index listed with g = fhat),
  signed zeros and subnormals;
- malformed streams and edit lists rejected before anything is written;
- the 512^3 Perlin correction: the whole stream round-trips and sampled blocks
  equal the oracle's packing of the same edits.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import edits as E
from paper_2601_01787_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_01787_gb300 import api as a
    a.load()
    return a


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bits(t):
    a = t.cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


@pytest.mark.parametrize("make", [
    lambda: synth.perlin3d_prequant((24, 40, 72), seed=11, eb_rel=1e-3),
    lambda: synth.peaks3d((20, 33, 47), seed=12, eb_rel=1e-4),
    lambda: synth.perlin2d((96, 130), seed=13, eb_rel=1e-3),
])
def test_correction_edits_encode_like_the_oracle(api, make):
    fl = make()
    ref = oracle.correct(fl.f, fl.fhat, fl.xi)
    assert ref.status == oracle.OK and ref.edit_count > 0
    idx_o, m_o = E.edits_of(fl.fhat, ref.g)
    assert np.array_equal(idx_o, ref.edit_idx[:ref.edit_count])
    want = E.encode(idx_o, m_o)
    res = api.correct(_dev(fl.f), _dev(fl.fhat), fl.xi)
    got = api.encode_edits(_dev(fl.fhat).reshape(-1), res.out.reshape(-1), res.edit_idx)
    assert got.cpu().numpy().tobytes() == want
    field = _dev(fl.fhat).reshape(-1).clone()
    assert api.decode_edits(got, field) == ref.edit_count
    assert np.array_equal(_bits(field), _bits(ref.g).ravel())


def _synthetic(count, kind, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "dense":
        gaps = rng.integers(1, 3, count)
        m = rng.integers(1, 9, count)
    elif kind == "sparse":
        gaps = rng.integers(1, 4000, count)
        m = rng.integers(1, 1 << 22, count)
    else:  # the widest ulp distances: 2^32 - 1, and 0 (an index listed with g = fhat)
        gaps = rng.integers(1, 200, count)
        m = rng.integers(0, 1 << 32, count, dtype=np.uint64)
        m[: count // 3] = (1 << 32) - 1
        m[count // 3: count // 2] = 0
    idx = (np.cumsum(gaps) - 1).astype(np.int64)
    return idx, m.astype(np.uint64)


@pytest.mark.parametrize("count", [0, 1, 255, 256, 257, 3001])
@pytest.mark.parametrize("kind", ["dense", "sparse", "wide"])
def test_synthetic_lists_match_the_oracle(api, count, kind):
    idx, m = _synthetic(count, kind, seed=count + len(kind))
    n = max(int(idx[-1]) + 6 if count else 0, 16)
    rng = np.random.default_rng(count)
    fhat = rng.uniform(-1, 1, n).astype(np.float32)
    fhat[:8] = [0.0, -0.0, 1e-42, -1e-42, 1.0, -1.0, 3e38, -3e38]
    g = fhat.copy()
    key = (E.ord_of(fhat[idx]).astype(np.int64) - m.astype(np.int64)) % (1 << 32)
    g[idx] = E.float_of(key.astype(np.uint32))
    want = E.encode(idx, m)
    got = api.encode_edits(_dev(fhat), _dev(g), _dev(idx.astype(np.int32)))
    assert got.cpu().numpy().tobytes() == want
    field = _dev(fhat)
    assert api.decode_edits(got, field) == count
    assert np.array_equal(_bits(field), _bits(E.apply(fhat, idx, m)))


def test_widest_gaps_and_distances(api):
    # gaps of 2^30 and more need a field of 2^31 - 1 floats; the index gaps
    # are exercised on a field of 2^27 (512 MB per copy), distances of
    # 2^32 - 1 and 0 everywhere
    n = 1 << 27
    idx = np.array([0, 1, (1 << 26) + 3, (1 << 27) - 1], dtype=np.int64)
    m = np.array([(1 << 32) - 1, 0, 1, 1 << 31], dtype=np.uint64)
    fhat = torch.zeros(n, dtype=torch.float32, device="cuda")
    fh_np = np.zeros(4, dtype=np.float32)
    key = (E.ord_of(fh_np).astype(np.int64) - m.astype(np.int64)) % (1 << 32)
    g = fhat.clone()
    g[_dev(idx)] = _dev(E.float_of(key.astype(np.uint32)))
    want = E.encode(idx, m)
    got = api.encode_edits(fhat, g, _dev(idx.astype(np.int32)))
    assert got.cpu().numpy().tobytes() == want
    field = fhat.clone()
    assert api.decode_edits(got, field) == 4
    assert torch.equal(field.view(torch.int32), g.view(torch.int32))


def test_malformed_streams_are_rejected_untouched(api):
    fhat = np.linspace(-1, 1, 5000, dtype=np.float32)
    idx = np.arange(3, 4900, 7, dtype=np.int64)
    m = np.arange(1, idx.size + 1, dtype=np.uint64)
    good = np.frombuffer(E.encode(idx, m), dtype=np.uint8).copy()

    def rejected(stream, n=fhat.size):
        field = _dev(fhat)
        with pytest.raises(api.MszError) as e:
            api.decode_edits(_dev(stream), field[:n] if n <= fhat.size else field)
        assert e.value.status == api.ERR_INVALID_ARG
        assert torch.equal(field.view(torch.int32), _dev(fhat).view(torch.int32))

    bad = good.copy(); bad[0] ^= 1
    rejected(bad)                                 # magic
    rejected(good[:-4])                           # payload cut short
    rejected(good[:20])                           # table cut short
    nb = (idx.size + 255) // 256
    bad = good.copy(); bad[16 + 8 * nb] = 40      # a width above 32
    rejected(bad)
    bad = good.copy(); bad[16 + 4:16 + 8] = np.frombuffer(np.uint32(5).tobytes(), np.uint8)
    rejected(bad)                                 # block 1 starts before block 0 ends
    rejected(good, n=int(idx[-1]))                # last index not below n
    # the encoder: indices not strictly ascending, or not below n
    g = fhat.copy(); g[idx] -= 0.25
    for wrong in (np.array([5, 5, 9]), np.array([9, 5]), np.array([1, 5000])):
        with pytest.raises(api.MszError) as e:
            api.encode_edits(_dev(fhat), _dev(g), _dev(wrong.astype(np.int32)))
        assert e.value.status == api.ERR_INVALID_ARG


def test_capacity_reported(api):
    import ctypes
    lib = api.load()
    fhat = _dev(np.linspace(0, 1, 4096, dtype=np.float32))
    g = fhat.clone(); g[::3] -= 1e-3
    idx = torch.arange(0, 4096, 3, dtype=torch.int32, device="cuda")
    need = api.encode_edits(fhat, g, idx).numel()
    out = torch.empty(need, dtype=torch.uint8, device="cuda")
    ws = api.workspace(lib.msz_edits_workspace_size(idx.numel()))
    nbytes = ctypes.c_size_t(0)
    st = lib.msz_edits_encode(fhat.data_ptr(), g.data_ptr(), 4096, idx.data_ptr(), idx.numel(), out.data_ptr(),
                              need - 4, ctypes.byref(nbytes), ws.data_ptr(), ws.numel(), None)
    assert st == api.ERR_CAPACITY and nbytes.value == need
    st = lib.msz_edits_encode(fhat.data_ptr(), g.data_ptr(), 4096, idx.data_ptr(), idx.numel(), out.data_ptr(),
                              need, ctypes.byref(nbytes), ws.data_ptr(), ws.numel(), None)
    assert st == api.OK and nbytes.value == need


def test_perlin_512_edit_stream(api):
    fl = synth.perlin3d_prequant((512, 512, 512), seed=2, eb_rel=1e-4)
    f, fh = _dev(fl.f), _dev(fl.fhat)
    cap = fl.n // 4
    eidx = torch.empty(cap, dtype=torch.int32, device="cuda")
    res = api.correct(f, fh, fl.xi, edit_idx=eidx, edit_capacity=cap)
    assert res.status == api.OK
    cnt = res.edit_count
    s = api.encode_edits(fh.reshape(-1), res.out.reshape(-1), eidx[:cnt])
    assert s.numel() < 4 * cnt  # well under the 8 bytes of a raw (index, delta) pair
    field = fh.reshape(-1).clone()
    assert api.decode_edits(s, field) == cnt
    assert torch.equal(field.view(torch.int32), res.out.reshape(-1).view(torch.int32))
    # sampled blocks against the oracle's packing of the same edits
    stream = s.cpu().numpy().tobytes()
    idx = eidx[:cnt].cpu().numpy().view(np.uint32).astype(np.int64)
    g = res.out.cpu().numpy().ravel()
    nb = (cnt + 255) // 256
    rng = np.random.default_rng(5)
    for k in sorted(set(rng.integers(0, nb, 12).tolist()) | {0, nb - 1}):
        bi = idx[k * 256:(k + 1) * 256]
        fh_b, g_b = fl.fhat.ravel()[bi], g[bi]
        m = (E.ord_of(fh_b).astype(np.int64) - E.ord_of(g_b).astype(np.int64)) % (1 << 32)
        one = E.encode(bi, m.astype(np.uint64))  # this block alone: a one-block stream
        words_one = np.frombuffer(one[16 + 12:], dtype="<u4")
        off = 16 + 10 * nb + (-(10 * nb) % 4)
        start = int(np.frombuffer(stream[16 + 4 * nb + 4 * k:16 + 4 * nb + 4 * k + 4], "<u4")[0])
        words = np.frombuffer(stream[off + 4 * start: off + 4 * (start + words_one.size)], dtype="<u4")
        assert np.array_equal(words, words_one), k
        assert int(np.frombuffer(stream[16 + 4 * k:16 + 4 * k + 4], "<u4")[0]) == int(bi[0])
