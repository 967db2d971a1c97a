"""ctypes binding of the CPU oracle (msz_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference arm are the only callers.  The product path never
imports this package.

Every function takes numpy arrays in (nz, ny, nx) or (ny, nx) C order, i.e. x
fastest, matching the linear index i = x + nx*(y + ny*z) of the paper's grid.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msz_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libmsz_oracle.so")
_lock = threading.Lock()
_lib = None

SELF = 15
OK, ERR_INVALID_ARG, ERR_INPUT_BOUND, ERR_CAPACITY, ERR_OOM, ERR_MAX_SWEEPS, STUCK = 0, 1, 2, 3, 4, 6, 8
RULE_HALVE, RULE_SNAP, RULE_BELOW = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (plain C99, no FMA contraction, no fast-math)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _configure(lib):
    """Declare the argument and result types of the oracle's C functions."""
    P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.orc_neighbour.argtypes = [I, I64, I64, I64, I64, I, ctypes.POINTER(I64)]
    lib.orc_neighbour.restype = I
    lib.orc_code_at.argtypes = [P, I, I64, I64, I64, I64]
    lib.orc_code_at.restype = ctypes.c_uint8
    lib.orc_codes.argtypes = [P, I, I64, I64, I64, P]
    lib.orc_floor.argtypes = [ctypes.c_float, ctypes.c_float]
    lib.orc_floor.restype = ctypes.c_float
    lib.orc_ceil.argtypes = [ctypes.c_float, ctypes.c_float]
    lib.orc_ceil.restype = ctypes.c_float
    lib.orc_validate.argtypes = [P, P, I64, ctypes.c_float]
    lib.orc_validate.restype = I
    lib.orc_edit.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_float, I]
    lib.orc_edit.restype = I
    lib.orc_edit_below.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float]
    lib.orc_edit_below.restype = I
    lib.orc_correct.argtypes = [P, P, ctypes.c_float, I, I64, I64, I64, I, I, I64, P, P,
                                P, P, I64, ctypes.POINTER(I64), P, P, I64]
    lib.orc_correct.restype = I
    lib.orc_correct_relaxed.argtypes = [P, P, ctypes.c_float, I, I64, I64, I64, I64, I64, I64, I, I64,
                                        I64, P, P]
    lib.orc_correct_relaxed.restype = I
    lib.orc_labels.argtypes = [P, I, I64, I64, I64, P, P]
    lib.orc_labels.restype = I
    lib.orc_compare.argtypes = [P, P, P, P, P, P, I64, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
    return a.ctypes.data


def grid_of(shape):
    """(ndim, nx, ny, nz) for a numpy shape (ny, nx) or (nz, ny, nx)."""
    if len(shape) == 2:
        return 2, int(shape[1]), int(shape[0]), 1
    if len(shape) == 3:
        return 3, int(shape[2]), int(shape[1]), int(shape[0])
    raise ValueError("grid must be 2D or 3D")


def neighbour(shape, i: int, slot: int):
    ndim, nx, ny, nz = grid_of(shape)
    j = ctypes.c_int64()
    ok = _load().orc_neighbour(ndim, nx, ny, nz, i, slot, ctypes.byref(j))
    return int(j.value) if ok else None


def num_slots(ndim: int) -> int:
    return 6 if ndim == 2 else 14


def code_at(v: np.ndarray, i: int) -> int:
    v = np.ascontiguousarray(v, dtype=np.float32)
    ndim, nx, ny, nz = grid_of(v.shape)
    return int(_load().orc_code_at(_p(v), ndim, nx, ny, nz, i))


def codes(v: np.ndarray) -> np.ndarray:
    """Packed steepest-neighbour codes: low nibble n_max slot, high nibble n_min slot, 15 = SELF."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    ndim, nx, ny, nz = grid_of(v.shape)
    out = np.empty(v.shape, dtype=np.uint8)
    _load().orc_codes(_p(v), ndim, nx, ny, nz, _p(out))
    return out


def floor_bound(f: float, xi: float) -> np.float32:
    return np.float32(_load().orc_floor(np.float32(f), np.float32(xi)))


def ceil_bound(f: float, xi: float) -> np.float32:
    return np.float32(_load().orc_ceil(np.float32(f), np.float32(xi)))


def validate(f: np.ndarray, fhat: np.ndarray, xi: float) -> int:
    f = np.ascontiguousarray(f, dtype=np.float32)
    fhat = np.ascontiguousarray(fhat, dtype=np.float32)
    return int(_load().orc_validate(_p(f), _p(fhat), f.size, np.float32(xi)))


def edit(g: float, L: float, rule: int = RULE_HALVE):
    """One application of Eq. 1: returns (new g, changed)."""
    c = ctypes.c_float(np.float32(g))
    ch = _load().orc_edit(ctypes.byref(c), np.float32(L), rule)
    return np.float32(c.value), bool(ch)


def edit_below(g: float, L: float, cand: float):
    """One BELOW-REFERENCE edit towards the candidate value: (new g, changed)."""
    c = ctypes.c_float(np.float32(g))
    ch = _load().orc_edit_below(ctypes.byref(c), np.float32(L), np.float32(cand))
    return np.float32(c.value), bool(ch)


class Result:
    def __init__(self, status, g, edit_idx, edit_delta, edit_count, stats, sweep_log):
        self.status = status
        self.g = g
        self.edit_idx = edit_idx
        self.edit_delta = edit_delta
        self.edit_count = edit_count
        self.stats = stats
        self.sweep_log = sweep_log

    @property
    def sweeps(self):
        return int(self.stats[0])

    @property
    def edits(self):
        return int(self.stats[1])

    @property
    def edited(self):
        return int(self.stats[2])

    @property
    def first_distorted(self):
        return int(self.stats[3])

    @property
    def left(self):
        return int(self.stats[4])

    @property
    def examined(self):
        return int(self.stats[5])


def correct(f, fhat, xi, *, worklist: bool = True, rule: int = RULE_HALVE, max_sweeps: int = 100000,
            g_init=None, edit_capacity: int | None = None, log_capacity: int = 0) -> Result:
    """Run the correction loop to zero distortion (or STUCK / MAX_SWEEPS)."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    fhat = np.ascontiguousarray(fhat, dtype=np.float32)
    assert f.shape == fhat.shape
    ndim, nx, ny, nz = grid_of(f.shape)
    n = f.size
    g = np.empty_like(f)
    cap = n if edit_capacity is None else int(edit_capacity)
    eidx = np.zeros(max(cap, 1), dtype=np.uint32)
    edel = np.zeros(max(cap, 1), dtype=np.float32)
    cnt = ctypes.c_int64()
    stats = np.zeros(8, dtype=np.int64)
    log = np.zeros(max(4 * log_capacity, 4), dtype=np.int64)
    gi = None if g_init is None else np.ascontiguousarray(g_init, dtype=np.float32)
    st = _load().orc_correct(_p(f), _p(fhat), np.float32(xi), ndim, nx, ny, nz, int(worklist), rule,
                             max_sweeps, _p(gi), _p(g), _p(eidx), _p(edel), cap, ctypes.byref(cnt),
                             _p(stats), _p(log), log_capacity)
    m = min(int(cnt.value), cap)
    nlog = min(int(stats[0]) + 1, log_capacity)
    return Result(int(st), g, eidx[:m].copy(), edel[:m].copy(), int(cnt.value), stats,
                  log[:4 * nlog].reshape(-1, 4).copy())


def correct_relaxed(f, fhat, xi, tile, *, rule: int = RULE_HALVE, local_cap: int = 0, max_iters: int = 100000):
    """Relaxed synchronization (Sec. IV-B) with tiles of tile = (tz, ty, tx)
    vertices (2D: (ty, tx)): returns (status, g, stats[8])."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    fhat = np.ascontiguousarray(fhat, dtype=np.float32)
    assert f.shape == fhat.shape
    ndim, nx, ny, nz = grid_of(f.shape)
    t = tuple(int(v) for v in tile)
    tz, ty, tx = t if len(t) == 3 else (1,) + t
    g = np.empty_like(f)
    stats = np.zeros(8, dtype=np.int64)
    st = _load().orc_correct_relaxed(_p(f), _p(fhat), np.float32(xi), ndim, nx, ny, nz, tx, ty, tz, rule,
                                     int(local_cap), int(max_iters), _p(g), _p(stats))
    return int(st), g, stats


def labels(codes_arr: np.ndarray):
    """(min_label, max_label): index of the extremum each vertex's integral line reaches."""
    c = np.ascontiguousarray(codes_arr, dtype=np.uint8)
    ndim, nx, ny, nz = grid_of(c.shape)
    mn = np.empty(c.shape, dtype=np.int32)
    mx = np.empty(c.shape, dtype=np.int32)
    st = _load().orc_labels(_p(c), ndim, nx, ny, nz, _p(mn), _p(mx))
    if st != OK:
        raise RuntimeError(f"orc_labels status {st}")
    return mn, mx


def compare(codes_f, codes_g, min_f, max_f, min_g, max_g) -> dict:
    """Wrong labels and false extrema between the segmentations of f and g (Sec. V-C)."""
    arrs = [np.ascontiguousarray(a) for a in (codes_f, codes_g, min_f, max_f, min_g, max_g)]
    out = np.zeros(5, dtype=np.int64)
    _load().orc_compare(*[_p(a) for a in arrs], arrs[0].size, _p(out))
    return dict(wrong_labels=int(out[0]), fp_max=int(out[1]), fn_max=int(out[2]),
                fp_min=int(out[3]), fn_min=int(out[4]))
