"""Python binding of the C ABI in include/msz.h (ctypes).

Argument marshalling only: every step of the correction runs in the CUDA
kernels of libmsz.so.  PyTorch provides device memory and the stream.  There
is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os
import struct
import threading
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _build

OK, ERR_INVALID_ARG, ERR_INPUT_BOUND, ERR_CAPACITY, ERR_WORKSPACE, ERR_CUDA = 0, 1, 2, 3, 4, 5
ERR_MAX_SWEEPS, ERR_TIMEOUT, STUCK, ERR_UNSUPPORTED = 6, 7, 8, 9
RULES = {"halve": 0, "snap": 1, "below": 2}
SELF = 15
MAX_SWEEPS_LIMIT = 65536
SMALL_WORKSPACE = 65536


class MszError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_str(status)}")


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64)]


class Options(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("test_fault", ctypes.c_int32), ("max_sweeps", ctypes.c_int64),
                ("dense_min_items", ctypes.c_int64), ("d_g_init", ctypes.c_void_p),
                ("h_sweep_log", ctypes.c_void_p), ("log_capacity", ctypes.c_int64),
                ("h_timeline", ctypes.c_void_p), ("tile_z", ctypes.c_int32), ("local_cap", ctypes.c_int32),
                ("phase_events", ctypes.c_void_p * 3)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("sweeps", "edits", "edited", "first_distorted", "left",
                                              "examined", "dense_sweeps", "kernel_ns", "codes_ns",
                                              "uncertified", "local_sweeps", "tile_runs")]

    def as_dict(self) -> dict:
        return dict(zip(_STATS_NAMES, _STATS_LAYOUT.unpack(bytes(self))))


_STATS_NAMES = tuple(n for n, _ in Stats._fields_)
_STATS_LAYOUT = struct.Struct(f"={len(_STATS_NAMES)}q")


class Field(ctypes.Structure):
    """msz_field: one field of a batch (inputs, then outputs written by the call)."""
    _fields_ = [("d_f", ctypes.c_void_p), ("d_fhat", ctypes.c_void_p), ("xi", ctypes.c_float),
                ("status", ctypes.c_int32), ("grid", Grid), ("d_out", ctypes.c_void_p),
                ("d_edit_idx", ctypes.c_void_p), ("d_edit_delta", ctypes.c_void_p),
                ("edit_capacity", ctypes.c_int64), ("edit_count", ctypes.c_int64), ("stats", Stats),
                ("tile_z", ctypes.c_int32), ("reserved", ctypes.c_int32)]


BATCH_MAX_FIELDS = 256
BATCH_MAX_SWEEPS = 4096

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmsz.so (building it first when asked).  Raises if it cannot load."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libmsz.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, I64, SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
        st = ctypes.c_int
        lib.msz_workspace_size.argtypes = [Grid]
        lib.msz_workspace_size.restype = SZ
        lib.msz_workspace_size_rule.argtypes = [Grid, ctypes.c_int32]
        lib.msz_workspace_size_rule.restype = SZ
        lib.msz_host_workspace_size.argtypes = [Grid, I64]
        lib.msz_host_workspace_size.restype = SZ
        lib.msz_directions.argtypes = [P, Grid, P, P]
        lib.msz_directions.restype = st
        lib.msz_correct.argtypes = [P, P, ctypes.c_float, Grid, P, P, P, I64, ctypes.POINTER(I64),
                                    ctypes.POINTER(Options), ctypes.POINTER(Stats), P, SZ, P]
        lib.msz_correct.restype = st
        lib.msz_correct_host.argtypes = lib.msz_correct.argtypes
        lib.msz_correct_host.restype = st
        lib.msz_segment.argtypes = [P, Grid, P, P, P, SZ, P]
        lib.msz_segment.restype = st
        lib.msz_compare.argtypes = [P, P, P, P, P, P, I64, ctypes.POINTER(I64), P, SZ, P]
        lib.msz_compare.restype = st
        lib.msz_correct_static.argtypes = [P, P, ctypes.c_float, Grid, P, P, P, I64, ctypes.POINTER(I64),
                                           ctypes.POINTER(Options), ctypes.POINTER(Stats), P]
        lib.msz_correct_static.restype = st
        lib.msz_batch_workspace_size.argtypes = [ctypes.c_int32, ctypes.POINTER(Field), I64]
        lib.msz_batch_workspace_size.restype = SZ
        lib.msz_correct_batch.argtypes = [ctypes.c_int32, ctypes.POINTER(Field), ctypes.POINTER(Options), P, I64, P,
                                          SZ, P]
        lib.msz_correct_batch.restype = st
        lib.msz_batch_plan_create.argtypes = [ctypes.c_int32, ctypes.POINTER(Field), ctypes.POINTER(Options), P, SZ,
                                              P, ctypes.POINTER(P)]
        lib.msz_batch_plan_create.restype = st
        lib.msz_batch_launch.argtypes = [P, P]
        lib.msz_batch_launch.restype = st
        lib.msz_batch_collect.argtypes = [P, ctypes.POINTER(Field), P, I64, P]
        lib.msz_batch_collect.restype = st
        lib.msz_batch_plan_destroy.argtypes = [P]
        lib.msz_batch_plan_destroy.restype = None
        lib.msz_relaxed_workspace_size.argtypes = [Grid]
        lib.msz_relaxed_workspace_size.restype = SZ
        lib.msz_correct_relaxed.argtypes = lib.msz_correct.argtypes
        lib.msz_correct_relaxed.restype = st
        lib.msz_edits_encoded_bound.argtypes = [I64]
        lib.msz_edits_encoded_bound.restype = SZ
        lib.msz_edits_workspace_size.argtypes = [I64]
        lib.msz_edits_workspace_size.restype = SZ
        lib.msz_edits_encode.argtypes = [P, P, I64, P, I64, P, SZ, ctypes.POINTER(SZ), P, SZ, P]
        lib.msz_edits_encode.restype = st
        lib.msz_edits_decode.argtypes = [P, SZ, P, I64, ctypes.POINTER(I64), P, SZ, P]
        lib.msz_edits_decode.restype = st
        lib.msz_pipeline_workspace_size.argtypes = [Grid, I64]
        lib.msz_pipeline_workspace_size.restype = SZ
        lib.msz_pipeline_create.argtypes = [Grid, I64, P, SZ, ctypes.POINTER(P)]
        lib.msz_pipeline_create.restype = st
        lib.msz_pipeline_submit.argtypes = [P, P, P, ctypes.c_float, P, P, P, ctypes.POINTER(Options)]
        lib.msz_pipeline_submit.restype = st
        lib.msz_pipeline_collect.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(Stats)]
        lib.msz_pipeline_collect.restype = st
        lib.msz_pipeline_destroy.argtypes = [P]
        lib.msz_pipeline_destroy.restype = None
        lib.msz_pipeline_workspace_size_encoded.argtypes = [Grid, I64]
        lib.msz_pipeline_workspace_size_encoded.restype = SZ
        lib.msz_pipeline_create_encoded.argtypes = [Grid, I64, P, SZ, ctypes.POINTER(P)]
        lib.msz_pipeline_create_encoded.restype = st
        lib.msz_pipeline_submit_encoded.argtypes = [P, P, P, ctypes.c_float, P, SZ, ctypes.POINTER(Options)]
        lib.msz_pipeline_submit_encoded.restype = st
        lib.msz_pipeline_collect_encoded.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(SZ), ctypes.POINTER(Stats)]
        lib.msz_pipeline_collect_encoded.restype = st
        lib.msz_status_str.argtypes = [st]
        lib.msz_status_str.restype = ctypes.c_char_p
        _lib = lib
        return lib


def status_str(status: int) -> str:
    return load().msz_status_str(int(status)).decode()


def grid_of(shape) -> Grid:
    """C grid for a tensor shape (ny, nx) or (nz, ny, nx), x fastest."""
    if len(shape) == 2:
        return Grid(2, 0, int(shape[1]), int(shape[0]), 1)
    if len(shape) == 3:
        return Grid(3, 0, int(shape[2]), int(shape[1]), int(shape[0]))
    raise ValueError("grid must be 2D or 3D")


def _dptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


_ws_cache: dict = {}


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A cached device byte buffer of at least nbytes (256-byte aligned)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
    key = dev.index
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        _ws_cache.pop(key, None)
        buf = torch.empty(max(int(nbytes), SMALL_WORKSPACE), dtype=torch.uint8, device=dev)
        assert buf.data_ptr() % 256 == 0
        _ws_cache[key] = buf
    return buf


def workspace_size(shape) -> int:
    return int(load().msz_workspace_size(grid_of(shape)))


def directions(v: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Packed steepest-neighbour codes of a float32 CUDA field (msz_directions)."""
    assert v.dtype == torch.float32
    if out is None:
        out = torch.empty(v.shape, dtype=torch.uint8, device=v.device)
    st = load().msz_directions(_dptr(v), grid_of(v.shape), _dptr(out), _stream(stream))
    if st != OK:
        raise MszError(st, "msz_directions")
    return out


@dataclass
class CorrectResult:
    status: int
    out: object
    edit_idx: object
    edit_delta: object
    edit_count: int
    stats: dict
    sweep_log: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), np.int64))

    @property
    def ok(self) -> bool:
        return self.status == OK


def _event_handle(ev):
    """The cudaEvent_t of a torch.cuda.Event (None: None); torch creates the
    event at its first record, so an event never recorded is recorded once."""
    if ev is None:
        return None
    if not ev.cuda_event:
        ev.record()
    return ev.cuda_event


_NO_LOG = np.zeros(4, dtype=np.int64)
_NO_TIMELINE = np.full(2, -1, dtype=np.int64)


def _options(rule, max_sweeps, dense_min_items, g_init, log_capacity, tile_z=0, test_fault=0, local_cap=0):
    # without a log the library writes no record: shared (empty-sliced) stand-ins
    log = np.zeros(4 * log_capacity, dtype=np.int64) if log_capacity else _NO_LOG
    tl = np.full(2 * log_capacity, -1, dtype=np.int64) if log_capacity else _NO_TIMELINE
    opt = Options(RULES[rule] if isinstance(rule, str) else int(rule), int(test_fault), int(max_sweeps),
                  int(dense_min_items),
                  _dptr(g_init), log.ctypes.data if log_capacity else None, int(log_capacity),
                  tl.ctypes.data if log_capacity else None, int(tile_z), int(local_cap))
    opt._keep = (log, tl)
    return opt, log


def correct(f: torch.Tensor, fhat: torch.Tensor, xi: float, *, rule="halve", max_sweeps: int = 0,
            dense_min_items: int = 0, g_init: torch.Tensor | None = None, edit_capacity: int | None = None,
            log_capacity: int = 0, out: torch.Tensor | None = None, edit_idx: torch.Tensor | None = None,
            edit_delta: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None,
            check: bool = False, tile_z: int = 0, test_fault: int = 0, events=None) -> CorrectResult:
    """Run the correction loop on device tensors (msz_correct).  events:
    three torch.cuda.Event (entries may be None) recorded before sweep 0's
    pass, between it and the loop kernel, and after the loop kernel."""
    assert f.dtype == torch.float32 and fhat.dtype == torch.float32 and f.shape == fhat.shape
    lib = load()
    g = grid_of(f.shape)
    n = f.numel()
    cap = n if edit_capacity is None else int(edit_capacity)
    if out is None:
        out = torch.empty_like(f)
    if edit_idx is None or edit_idx.numel() < cap:
        edit_idx = torch.empty(max(cap, 1), dtype=torch.int32, device=f.device)
    if edit_delta is None or edit_delta.numel() < cap:
        edit_delta = torch.empty(max(cap, 1), dtype=torch.float32, device=f.device)
    if ws is None:
        ws = workspace(int(lib.msz_workspace_size_rule(g, RULES[rule] if isinstance(rule, str) else int(rule))),
                       f.device)
    opt, log = _options(rule, max_sweeps, dense_min_items, g_init, log_capacity, tile_z, test_fault)
    if events is not None:
        for i, ev in enumerate(events):
            opt.phase_events[i] = _event_handle(ev)
    stats = Stats()
    count = ctypes.c_int64()
    st = lib.msz_correct(_dptr(f), _dptr(fhat), ctypes.c_float(np.float32(xi)), g, _dptr(out),
                         _dptr(edit_idx), _dptr(edit_delta), cap, ctypes.byref(count), ctypes.byref(opt),
                         ctypes.byref(stats), _dptr(ws), ws.numel(), _stream(stream))
    if check and st not in (OK,):
        raise MszError(st, "msz_correct")
    m = min(int(count.value), cap)
    nlog = min(stats.sweeps + 1, log_capacity)
    res = CorrectResult(int(st), out, edit_idx[:m], edit_delta[:m], int(count.value), stats.as_dict(),
                        log[:4 * nlog].reshape(-1, 4).copy())
    res.timeline = opt._keep[1][:2 * nlog].reshape(-1, 2).copy()
    return res


RELAXED_TILE = (8, 8, 32)  # (z, y, x) vertices per tile of msz_correct_relaxed


def correct_relaxed(f: torch.Tensor, fhat: torch.Tensor, xi: float, *, rule="halve", max_iters: int = 0,
                    local_cap: int = 0, edit_capacity: int | None = None, log_capacity: int = 0,
                    out: torch.Tensor | None = None, edit_idx: torch.Tensor | None = None,
                    edit_delta: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None,
                    tile_z: int = 0) -> CorrectResult:
    """The relaxed synchronization of Sec. IV-B on one GPU (msz_correct_relaxed)."""
    assert f.dtype == torch.float32 and fhat.dtype == torch.float32 and f.shape == fhat.shape and f.dim() == 3
    lib = load()
    g = grid_of(f.shape)
    cap = f.numel() if edit_capacity is None else int(edit_capacity)
    if out is None:
        out = torch.empty_like(f)
    if edit_idx is None or edit_idx.numel() < cap:
        edit_idx = torch.empty(max(cap, 1), dtype=torch.int32, device=f.device)
    if edit_delta is None or edit_delta.numel() < cap:
        edit_delta = torch.empty(max(cap, 1), dtype=torch.float32, device=f.device)
    if ws is None:
        ws = workspace(int(lib.msz_relaxed_workspace_size(g)), f.device)
    opt, log = _options(rule, max_iters, 0, None, log_capacity, tile_z, 0, local_cap)
    stats = Stats()
    count = ctypes.c_int64()
    st = lib.msz_correct_relaxed(_dptr(f), _dptr(fhat), ctypes.c_float(np.float32(xi)), g, _dptr(out),
                                 _dptr(edit_idx), _dptr(edit_delta), cap, ctypes.byref(count), ctypes.byref(opt),
                                 ctypes.byref(stats), _dptr(ws), ws.numel(), _stream(stream))
    m = min(int(count.value), cap)
    nlog = min(stats.sweeps + 1, log_capacity)
    res = CorrectResult(int(st), out, edit_idx[:m], edit_delta[:m], int(count.value), stats.as_dict(),
                        log[:4 * nlog].reshape(-1, 4).copy())
    res.timeline = opt._keep[1][:2 * nlog].reshape(-1, 2).copy()
    return res


def host_workspace_size(shape, edit_capacity: int) -> int:
    return int(load().msz_host_workspace_size(grid_of(shape), int(edit_capacity)))


def correct_host(f: np.ndarray | torch.Tensor, fhat, xi: float, *, out=None, edit_idx=None, edit_delta=None,
                 edit_capacity: int | None = None, rule="halve", max_sweeps: int = 0, dense_min_items: int = 0,
                 ws: torch.Tensor | None = None, stream=None) -> CorrectResult:
    """msz_correct_host: host buffers in, host buffers out (copies inside the call)."""
    def host_ptr(a):
        if isinstance(a, torch.Tensor):
            assert not a.is_cuda and a.is_contiguous()
            return a.data_ptr()
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data

    lib = load()
    shape = tuple(f.shape)
    n = int(np.prod(shape))
    cap = n if edit_capacity is None else int(edit_capacity)
    if out is None:
        out = np.empty(shape, dtype=np.float32)
    if edit_idx is None:
        edit_idx = np.empty(max(cap, 1), dtype=np.uint32)
    if edit_delta is None:
        edit_delta = np.empty(max(cap, 1), dtype=np.float32)
    g = grid_of(shape)
    need = int(lib.msz_host_workspace_size(g, cap))
    if ws is None:
        ws = workspace(need)
    opt, log = _options(rule, max_sweeps, dense_min_items, None, 0)
    stats = Stats()
    count = ctypes.c_int64()
    st = lib.msz_correct_host(host_ptr(f), host_ptr(fhat), ctypes.c_float(np.float32(xi)), g, host_ptr(out),
                              host_ptr(edit_idx), host_ptr(edit_delta), cap, ctypes.byref(count),
                              ctypes.byref(opt), ctypes.byref(stats), _dptr(ws), ws.numel(), _stream(stream))
    m = min(int(count.value), cap)
    return CorrectResult(int(st), out, edit_idx[:m], edit_delta[:m], int(count.value), stats.as_dict())


def _host_ptr(a):
    if isinstance(a, torch.Tensor):
        assert not a.is_cuda and a.is_contiguous()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclass
class EncodedResult:
    status: int
    stream: object  # the host buffer, cut to the stream's length
    edit_count: int
    stats: dict


class Pipeline:
    """msz_pipeline_*: a sequence of fields of one shape corrected from host
    buffers with the copies of consecutive fields overlapped.  submit()
    returns at once (at most two fields in flight); collect() returns the
    oldest field's result once it is in its host buffers: a CorrectResult (g
    and the edit list), or with encoded=True an EncodedResult holding the edit
    list's stream (msz_edits_encode format) instead.  Pinned host buffers
    (torch pin_memory) let the copies overlap."""

    def __init__(self, shape, edit_capacity: int | None = None, device=None, encoded: bool = False):
        lib = load()
        self.shape = tuple(int(v) for v in shape)
        self.n = int(np.prod(self.shape))
        self.cap = self.n if edit_capacity is None else int(edit_capacity)
        self.encoded = bool(encoded)
        g = grid_of(self.shape)
        size = lib.msz_pipeline_workspace_size_encoded if encoded else lib.msz_pipeline_workspace_size
        need = int(size(g, self.cap))
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
        self.ws = torch.empty(need, dtype=torch.uint8, device=dev)  # owned: the pipeline's two slots
        h = ctypes.c_void_p()
        create = lib.msz_pipeline_create_encoded if encoded else lib.msz_pipeline_create
        st = create(g, self.cap, _dptr(self.ws), self.ws.numel(), ctypes.byref(h))
        if st != OK:
            raise MszError(st, "msz_pipeline_create")
        self._h = h
        self._fifo = []

    def stream_bound(self) -> int:
        """Bytes a host stream buffer needs for any field (encoded pipelines)."""
        return int(load().msz_edits_encoded_bound(self.cap))

    def submit(self, f, fhat, xi: float, out, edit_idx=None, edit_delta=None, *, rule="halve",
               max_sweeps: int = 0, dense_min_items: int = 0):
        """One field; `out` is g's host buffer, or for an encoded pipeline the
        stream's host buffer (uint8, stream_bound() bytes suffice)."""
        opt, _ = _options(rule, max_sweeps, dense_min_items, None, 0)
        lib = load()
        if self.encoded:
            nbytes = out.numel() if isinstance(out, torch.Tensor) else out.nbytes
            st = lib.msz_pipeline_submit_encoded(self._h, _host_ptr(f), _host_ptr(fhat),
                                                 ctypes.c_float(np.float32(xi)), _host_ptr(out), nbytes,
                                                 ctypes.byref(opt))
            if st != OK:
                raise MszError(st, "msz_pipeline_submit_encoded")
            self._fifo.append((out,))
            return
        if edit_idx is None:
            edit_idx = np.empty(max(self.cap, 1), dtype=np.uint32)
        if edit_delta is None:
            edit_delta = np.empty(max(self.cap, 1), dtype=np.float32)
        st = lib.msz_pipeline_submit(self._h, _host_ptr(f), _host_ptr(fhat), ctypes.c_float(np.float32(xi)),
                                     _host_ptr(out), _host_ptr(edit_idx), _host_ptr(edit_delta), ctypes.byref(opt))
        if st != OK:
            raise MszError(st, "msz_pipeline_submit")
        self._fifo.append((out, edit_idx, edit_delta))

    def collect(self):
        stats = Stats()
        count = ctypes.c_int64()
        lib = load()
        if self.encoded:
            nbytes = ctypes.c_size_t(0)
            st = lib.msz_pipeline_collect_encoded(self._h, ctypes.byref(count), ctypes.byref(nbytes),
                                                  ctypes.byref(stats))
            if not self._fifo:
                raise MszError(st, "msz_pipeline_collect_encoded")
            (buf,) = self._fifo.pop(0)
            return EncodedResult(int(st), buf[:nbytes.value], int(count.value), stats.as_dict())
        st = lib.msz_pipeline_collect(self._h, ctypes.byref(count), ctypes.byref(stats))
        if not self._fifo:
            raise MszError(st, "msz_pipeline_collect")
        out, idx, dl = self._fifo.pop(0)
        m = min(int(count.value), self.cap)
        return CorrectResult(int(st), out, idx[:m], dl[:m], int(count.value), stats.as_dict())

    def close(self):
        if getattr(self, "_h", None):
            load().msz_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def segment(codes: torch.Tensor, ws: torch.Tensor | None = None, stream=None):
    """(min_label, max_label) int32 tensors by pointer jumping (msz_segment)."""
    assert codes.dtype == torch.uint8
    mn = torch.empty(codes.shape, dtype=torch.int32, device=codes.device)
    mx = torch.empty(codes.shape, dtype=torch.int32, device=codes.device)
    if ws is None:
        ws = workspace(SMALL_WORKSPACE, codes.device)
    st = load().msz_segment(_dptr(codes), grid_of(codes.shape), _dptr(mn), _dptr(mx), _dptr(ws), ws.numel(),
                            _stream(stream))
    if st != OK:
        raise MszError(st, "msz_segment")
    return mn, mx


def compare(codes_f, codes_g, min_f, max_f, min_g, max_g, ws: torch.Tensor | None = None, stream=None) -> dict:
    """Wrong labels, false extrema and code mismatches between two fields'
    codes and segmentations (msz_compare)."""
    counts = (ctypes.c_int64 * 6)()
    if ws is None:
        ws = workspace(SMALL_WORKSPACE, codes_f.device)
    st = load().msz_compare(_dptr(codes_f), _dptr(codes_g), _dptr(min_f), _dptr(max_f), _dptr(min_g),
                            _dptr(max_g), codes_f.numel(), counts, _dptr(ws), ws.numel(), _stream(stream))
    if st != OK:
        raise MszError(st, "msz_compare")
    return dict(wrong_labels=counts[0], fp_max=counts[1], fn_max=counts[2], fp_min=counts[3], fn_min=counts[4],
                code_mismatches=counts[5])


def verify(f: torch.Tensor, g: torch.Tensor) -> dict:
    """Codes, labels and the verification counts of g against f, all on the GPU."""
    cf, cg = directions(f), directions(g)
    mf, Mf = segment(cf)
    mg, Mg = segment(cg)
    res = compare(cf, cg, mf, Mf, mg, Mg)
    res["codes_equal"] = res["code_mismatches"] == 0
    return res


@dataclass
class BatchResult:
    status: int
    fields: list  # CorrectResult per field
    # device ns from the code pass's start to the end of sweep k's detection
    # (column 0) and edit phase (column 1), -1 for none; empty unless asked for
    timeline: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int64))


def _batch_fields(fs, fhats, xis, edit_capacities, outs, tile_z):
    """The msz_field array of a batch and the output buffers it points to:
    (outs, edit_idx, edit_delta, offsets, capacities), the edit lists of all
    fields in one pair of buffers (field k's at offsets[k])."""
    n = len(fs)
    arr = (Field * n)()  # zero-filled: stats, edit_count and reserved start at 0
    caps = [fs[k].numel() if edit_capacities is None else int(edit_capacities[k]) for k in range(n)]
    offs, tot = [], 0
    for c in caps:
        offs.append(tot)
        tot += max(c, 1)
    dev = fs[0].device
    idx_all = torch.empty(tot, dtype=torch.int32, device=dev)
    dl_all = torch.empty(tot, dtype=torch.float32, device=dev)
    ib, db = _dptr(idx_all), _dptr(dl_all)
    outs = [torch.empty_like(f) for f in fs] if outs is None else list(outs)
    for k in range(n):
        f, fh = fs[k], fhats[k]
        assert f.dtype == torch.float32 and fh.dtype == torch.float32 and f.shape == fh.shape and f.dim() == 3
        fk = arr[k]
        fk.d_f = _dptr(f)
        fk.d_fhat = _dptr(fh)
        fk.xi = float(np.float32(xis[k]))
        fk.status = -1
        nz, ny, nx = f.shape
        g = fk.grid
        g.ndim, g.nx, g.ny, g.nz = 3, int(nx), int(ny), int(nz)
        fk.d_out = _dptr(outs[k])
        fk.d_edit_idx = ib + 4 * offs[k]
        fk.d_edit_delta = db + 4 * offs[k]
        fk.edit_capacity = caps[k]
        fk.tile_z = 0 if tile_z is None else int(tile_z[k])
    return arr, (outs, idx_all, dl_all, offs, caps)


def _batch_workspace(lib, arr, max_sweeps, ws, device):
    need = int(lib.msz_batch_workspace_size(len(arr), arr, int(max_sweeps)))
    if need == 0:
        raise MszError(ERR_INVALID_ARG, "msz_batch_workspace_size")
    return workspace(need, device) if ws is None else ws


_NO_SWEEP_LOG = np.zeros((0, 4), np.int64)
# the outputs of an msz_field array read as one numpy record each (offsets
# from the ctypes layout)
_FIELD_OUT = np.dtype({"names": ["status", "edit_count", "stats"],
                       "formats": [np.int32, np.int64, (np.int64, len(_STATS_NAMES))],
                       "offsets": [Field.status.offset, Field.edit_count.offset, Field.stats.offset],
                       "itemsize": ctypes.sizeof(Field)})


def _batch_results(arr, keep, log, log_capacity, status, timeline=None) -> "BatchResult":
    outs, idx_all, dl_all, offs, caps = keep
    rec = np.frombuffer(arr, dtype=_FIELD_OUT)
    counts = rec["edit_count"].tolist()
    statuses = rec["status"].tolist()
    stats = rec["stats"].tolist()
    results = []
    for k in range(len(arr)):
        m = min(counts[k], caps[k])
        st = dict(zip(_STATS_NAMES, stats[k]))
        if log_capacity:
            nlog = min(st["sweeps"] + 1, log_capacity)
            lg = log[4 * k * log_capacity:4 * (k * log_capacity + nlog)].reshape(-1, 4).copy()
        else:
            lg = _NO_SWEEP_LOG
        o = offs[k]
        results.append(CorrectResult(statuses[k], outs[k], idx_all[o:o + m], dl_all[o:o + m], counts[k], st, lg))
    tl = timeline.reshape(-1, 2).copy() if timeline is not None else np.zeros((0, 2), np.int64)
    return BatchResult(int(status), results, tl)


class BatchPlan:
    """A prepared batch (msz_batch_plan_create): launch() is asynchronous and
    can be captured in a CUDA graph; collect() synchronizes and returns the
    per-field results.  The plan keeps every buffer it points to alive."""

    def __init__(self, fs, fhats, xis, *, rule="halve", max_sweeps: int = 0, dense_min_items: int = 0,
                 edit_capacities=None, outs=None, ws: torch.Tensor | None = None, stream=None, tile_z=None,
                 timeline_capacity: int = 0):
        lib = load()
        arr, keep = _batch_fields(fs, fhats, xis, edit_capacities, outs, tile_z)
        ws = _batch_workspace(lib, arr, max_sweeps, ws, fs[0].device)
        opt, _ = _options(rule, max_sweeps, dense_min_items, None, int(timeline_capacity))
        handle = ctypes.c_void_p()
        st = lib.msz_batch_plan_create(len(arr), arr, ctypes.byref(opt), _dptr(ws), ws.numel(), _stream(stream),
                                       ctypes.byref(handle))
        if st != OK:
            raise MszError(st, "msz_batch_plan_create")
        self._lib, self._h, self.n, self.arr = lib, handle, len(arr), arr
        self._keep = (list(fs), list(fhats), keep, ws, opt)

    @property
    def outputs(self):
        """(out, edit_idx, edit_delta, capacity) of every field."""
        outs, idx_all, dl_all, offs, caps = self._keep[2]
        return [(outs[k], idx_all[offs[k]:offs[k] + max(caps[k], 1)], dl_all[offs[k]:offs[k] + max(caps[k], 1)],
                 caps[k]) for k in range(len(outs))]

    def launch(self, stream=None) -> None:
        st = self._lib.msz_batch_launch(self._h, _stream(stream))
        if st != OK:
            raise MszError(st, "msz_batch_launch")

    def collect(self, log_capacity: int = 0, stream=None) -> "BatchResult":
        log = np.zeros(max(4 * self.n * log_capacity, 4), dtype=np.int64)
        st = self._lib.msz_batch_collect(self._h, self.arr, log.ctypes.data if log_capacity else None,
                                         int(log_capacity), _stream(stream))
        tl = self._keep[4]._keep[1] if self._keep[4].log_capacity else None
        return _batch_results(self.arr, self._keep[2], log, log_capacity, st, tl)

    def graph(self, stream=None) -> "torch.cuda.CUDAGraph":
        """Capture one launch in a CUDA graph; replay() then reruns the whole
        batch correction (read the results with collect())."""
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream() if stream is None else stream
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=side):
            self.launch(torch.cuda.current_stream())
        torch.cuda.current_stream().wait_stream(side)
        return g

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.msz_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def correct_batch(fs, fhats, xis, *, rule="halve", max_sweeps: int = 0, dense_min_items: int = 0,
                  edit_capacities=None, log_capacity: int = 0, outs=None, ws: torch.Tensor | None = None,
                  stream=None, tile_z=None, timeline_capacity: int = 0) -> BatchResult:
    """msz_correct_batch: many 3D fields (CUDA tensors) in one persistent
    launch.  timeline_capacity > 0: the result's timeline holds the device
    times of the first that many sweeps."""
    lib = load()
    arr, keep = _batch_fields(fs, fhats, xis, edit_capacities, outs, tile_z)
    ws = _batch_workspace(lib, arr, max_sweeps, ws, fs[0].device)
    opt, _ = _options(rule, max_sweeps, dense_min_items, None, int(timeline_capacity))
    log = np.zeros(max(4 * len(arr) * log_capacity, 4), dtype=np.int64)
    st = lib.msz_correct_batch(len(arr), arr, ctypes.byref(opt), log.ctypes.data if log_capacity else None,
                               log_capacity, _dptr(ws), ws.numel(), _stream(stream))
    return _batch_results(arr, keep, log, log_capacity, st, opt._keep[1] if timeline_capacity else None)


# ------------------------------------------------------------ edit encoding
EDIT_MAGIC = 0x45535A4D
EDIT_BLOCK = 256


def encode_edits(fhat: torch.Tensor, g: torch.Tensor, edit_idx: torch.Tensor, stream=None) -> torch.Tensor:
    """Stream of the edit list edit_idx (ascending int32/uint32 vertex indices,
    as correct() returns them) of g against fhat (msz_edits_encode): a uint8
    CUDA tensor of the stream's length."""
    lib = load()
    n = fhat.numel()
    if g.numel() != n or fhat.dtype != torch.float32 or g.dtype != torch.float32:
        raise ValueError("fhat and g must be float32 tensors of one size")
    if edit_idx.dtype not in (torch.int32, torch.uint32):
        raise ValueError("edit_idx must be int32 or uint32")
    count = edit_idx.numel()
    cap = int(lib.msz_edits_encoded_bound(count))
    out = torch.empty(cap, dtype=torch.uint8, device=fhat.device)
    ws = workspace(int(lib.msz_edits_workspace_size(count)), fhat.device)
    nbytes = ctypes.c_size_t(0)
    st = lib.msz_edits_encode(_dptr(fhat), _dptr(g), n, _dptr(edit_idx) if count else None, count, _dptr(out), cap,
                              ctypes.byref(nbytes), _dptr(ws), ws.numel(), _stream(stream))
    if st != OK:
        raise MszError(st, "msz_edits_encode")
    return out[:nbytes.value]


def decode_edits(stream_bytes: torch.Tensor, field: torch.Tensor, stream=None) -> int:
    """Applies an edit stream to `field` in place (fhat in, g out;
    msz_edits_decode) and returns its edit count."""
    lib = load()
    if stream_bytes.dtype != torch.uint8 or field.dtype != torch.float32:
        raise ValueError("expected a uint8 stream and a float32 field")
    if stream_bytes.numel() < 16:
        raise MszError(ERR_INVALID_ARG, "msz_edits_decode")
    count = int(stream_bytes[8:16].cpu().view(torch.int64)[0])
    if count < 0 or count > field.numel():
        raise MszError(ERR_INVALID_ARG, "msz_edits_decode")
    ws = workspace(int(lib.msz_edits_workspace_size(max(count, 0))), field.device)
    got = ctypes.c_int64(0)
    st = lib.msz_edits_decode(_dptr(stream_bytes), stream_bytes.numel(), _dptr(field), field.numel(),
                              ctypes.byref(got), _dptr(ws), ws.numel(), _stream(stream))
    if st != OK:
        raise MszError(st, "msz_edits_decode")
    return int(got.value)
