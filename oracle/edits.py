"""Oracle of the edit-list encoding (storage of the edits).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline leg are the only callers.  The product path never imports it.

The corrected field is stored as the decompressed field fhat plus a list of
edits (Sec. V, computation and storage overhead: the extra storage is the
edits).  The paper fixes no format; this module writes out, plainly and one
block at a time, the exact format the library's encoder produces, so that
its bytes can be compared with the GPU's one for one.

An edit is a pair (i, m): the vertex index i and its ulp distance
    m = (ord(fhat_i) - ord(g_i)) mod 2^32,
where ord maps a float32's bits to an unsigned integer in value order
(positive: bits | 0x80000000, negative: ~bits).  ord is a bijection on bit
patterns, so g_i = ord^-1(ord(fhat_i) - m) recovers g_i bit for bit, -0 and
subnormals included.  The edits of a field are the vertices where g and fhat
differ bitwise, in ascending index order (m >= 1).

Stream (little-endian), B = 256 edits per block, nb = ceil(count / B):
    bytes 0..3    magic 0x45535A4D
    bytes 4..7    B
    bytes 8..15   count
    nb x u32      first index of each block
    nb x u32      start of each block's payload, in 32-bit words from the
                  start of the payload
    nb x u8       wd: bit width of the block's index gaps
    nb x u8       wm: bit width of the block's ulp distances minus one
    zero bytes    up to a multiple of 4
    payload       per block of c edits: the c values d_j packed wd bits each,
                  LSB first into 32-bit words (value j at bit j*wd of the
                  section), the section padded to whole words; then the c
                  values (m_j - 1) mod 2^32 packed wm bits each the same way
                  (an index listed with g_i = fhat_i, m = 0, stays exact).
with d_0 = 0 and d_j = i_j - i_{j-1} - 1, and the width of a section the bit
length of its largest value (0 when every value is 0: the section is empty).
"""
from __future__ import annotations

import numpy as np

MAGIC = 0x45535A4D
BLOCK = 256


def ord_of(v: np.ndarray) -> np.ndarray:
    """Value-order key of float32 values as uint32 (see the module docstring)."""
    b = np.ascontiguousarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    neg = (b >> 31) == 1
    out = np.where(neg, (~b) & 0xFFFFFFFF, b | 0x80000000)
    return out.astype(np.uint32)


def float_of(key: np.ndarray) -> np.ndarray:
    """Inverse of ord_of."""
    k = np.asarray(key, dtype=np.uint64)
    pos = (k >> 31) == 1
    b = np.where(pos, k & 0x7FFFFFFF, (~k) & 0xFFFFFFFF)
    return b.astype(np.uint32).view(np.float32)


def edits_of(fhat: np.ndarray, g: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """The edit list of a corrected field: indices where g and fhat differ
    bitwise (ascending) and their ulp distances m."""
    fb = np.ascontiguousarray(fhat, dtype=np.float32).reshape(-1)
    gb = np.ascontiguousarray(g, dtype=np.float32).reshape(-1)
    idx = np.flatnonzero(fb.view(np.uint32) != gb.view(np.uint32)).astype(np.uint32)
    m = (ord_of(fb[idx]).astype(np.int64) - ord_of(gb[idx]).astype(np.int64)) % (1 << 32)
    return idx, m.astype(np.uint32)


def bit_width(x: int) -> int:
    """Number of bits of the largest value of a section (0 for 0)."""
    return int(x).bit_length()


def pack(values: np.ndarray, width: int) -> list[int]:
    """values packed `width` bits each, LSB first, into 32-bit words."""
    nbits = len(values) * width
    words = [0] * ((nbits + 31) // 32)
    for j, v in enumerate(values.tolist()):
        for b in range(width):
            if (v >> b) & 1:
                pos = j * width + b
                words[pos >> 5] |= 1 << (pos & 31)
    return words


def unpack(words: list[int], count: int, width: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint64)
    for j in range(count):
        v = 0
        for b in range(width):
            pos = j * width + b
            v |= ((words[pos >> 5] >> (pos & 31)) & 1) << b
        out[j] = v
    return out


def encode(idx: np.ndarray, m: np.ndarray) -> bytes:
    """The stream of an edit list (ascending indices, ulp distances >= 1)."""
    idx = np.asarray(idx, dtype=np.uint64)
    m = np.asarray(m, dtype=np.uint64)
    count = len(idx)
    nb = (count + BLOCK - 1) // BLOCK
    first, start, wd, wm, payload = [], [], [], [], []
    for k in range(nb):
        bi = idx[k * BLOCK:(k + 1) * BLOCK]
        bm = m[k * BLOCK:(k + 1) * BLOCK]
        d = np.zeros(len(bi), dtype=np.uint64)
        d[1:] = bi[1:] - bi[:-1] - 1
        w1 = bit_width(int(d.max()))
        mq = (bm + 0xFFFFFFFF) & 0xFFFFFFFF  # (m - 1) mod 2^32
        w2 = bit_width(int(mq.max()))
        first.append(int(bi[0]))
        start.append(len(payload))
        wd.append(w1)
        wm.append(w2)
        payload += pack(d, w1)
        payload += pack(mq, w2)
    head = np.array([MAGIC, BLOCK], dtype="<u4").tobytes() + np.array([count], dtype="<u8").tobytes()
    table = (np.array(first, dtype="<u4").tobytes() + np.array(start, dtype="<u4").tobytes()
             + np.array(wd, dtype="u1").tobytes() + np.array(wm, dtype="u1").tobytes())
    table += b"\0" * (-len(table) % 4)
    return head + table + np.array(payload, dtype="<u4").tobytes()


def decode(stream: bytes) -> tuple[np.ndarray, np.ndarray]:
    """(indices, ulp distances) of a stream."""
    magic, block = np.frombuffer(stream[:8], dtype="<u4")
    if magic != MAGIC or block != BLOCK:
        raise ValueError("not an edit-list stream")
    count = int(np.frombuffer(stream[8:16], dtype="<u8")[0])
    nb = (count + BLOCK - 1) // BLOCK
    o = 16
    first = np.frombuffer(stream[o:o + 4 * nb], dtype="<u4"); o += 4 * nb
    start = np.frombuffer(stream[o:o + 4 * nb], dtype="<u4"); o += 4 * nb
    wd = np.frombuffer(stream[o:o + nb], dtype="u1"); o += nb
    wm = np.frombuffer(stream[o:o + nb], dtype="u1"); o += nb
    o += -o % 4
    words = np.frombuffer(stream[o:], dtype="<u4").tolist()
    idx = np.zeros(count, dtype=np.uint64)
    m = np.zeros(count, dtype=np.uint64)
    for k in range(nb):
        c = min(BLOCK, count - k * BLOCK)
        s = int(start[k])
        nd = (c * int(wd[k]) + 31) // 32
        nm = (c * int(wm[k]) + 31) // 32
        d = unpack(words[s:s + nd], c, int(wd[k]))
        mm = (unpack(words[s + nd:s + nd + nm], c, int(wm[k])) + 1) & 0xFFFFFFFF
        i = int(first[k])
        for j in range(c):
            if j:
                i += int(d[j]) + 1
            idx[k * BLOCK + j] = i
        m[k * BLOCK:k * BLOCK + c] = mm
    return idx.astype(np.uint32), m.astype(np.uint32)


def apply(fhat: np.ndarray, idx: np.ndarray, m: np.ndarray) -> np.ndarray:
    """g from fhat and an edit list: g_i = ord^-1(ord(fhat_i) - m_i)."""
    g = np.array(fhat, dtype=np.float32, copy=True).reshape(-1)
    key = (ord_of(g[idx]).astype(np.int64) - np.asarray(m, dtype=np.int64)) % (1 << 32)
    g[idx] = float_of(key.astype(np.uint32))
    return g.reshape(np.shape(fhat))


def encoded_size(idx: np.ndarray, m: np.ndarray) -> int:
    """Length of the stream from the widths alone (no packing)."""
    idx = np.asarray(idx, dtype=np.uint64)
    m = np.asarray(m, dtype=np.uint64)
    count = len(idx)
    nb = (count + BLOCK - 1) // BLOCK
    words = 0
    for k in range(nb):
        bi = idx[k * BLOCK:(k + 1) * BLOCK]
        bm = m[k * BLOCK:(k + 1) * BLOCK]
        c = len(bi)
        w1 = bit_width(int((bi[1:] - bi[:-1] - 1).max())) if c > 1 else 0
        w2 = bit_width(int(((bm + 0xFFFFFFFF) & 0xFFFFFFFF).max()))
        words += (c * w1 + 31) // 32 + (c * w2 + 31) // 32
    table = 8 * nb + 2 * nb
    return 16 + table + (-table % 4) + 4 * words
