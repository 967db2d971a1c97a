"""Seeded synthetic inputs for the correction loop (its own module).

Holds none of the correction method's arithmetic: it only makes fields ``f``,
their compressor stand-ins ``fhat`` and the error bound ``xi``.  The CPU oracle
and the CUDA path both read what it returns.  The heavy lifting is in
``synth.c`` (OpenMP, counter-based random numbers, so results do not depend on
the thread count).

Workloads (the paper's scaling data is Perlin noise, Sec. V-B; a Gaussian-peak
field stands in for the diffraction-peak data of Fig. "distortion"; uniform
noise and 2*xi scalar quantization stand in for ZFP/SZ3 output, Sec. V):

=====================  =========================================================
name                   recipe
=====================  =========================================================
``perlin2d``           2D Perlin, 4 octaves, period 64; fhat = f + U[-xi, xi];
                       xi = 1e-3 * range (default 256 x 256, seed 1)
``perlin3d_prequant``  3D Perlin, 5 octaves, period 64; fhat = 2 xi round(f/2xi);
                       xi = 1e-4 * range (default 512^3, seed 2)
``peaks3d``            Poisson(5) background + Gaussian peaks (20,000 at
                       1024 x 1024 x 512, same density at other sizes);
                       fhat = f + U[-xi, xi]; xi = 1e-4 * range (seed 3)
``batch``              64 Perlin fields, axes ~ U{64..384}, eb_rel in
                       {1e-3, 1e-4, 1e-5}, prequantized (seeds 1000 + k)
``peaks3d_learned``    512^3 peak field, 5,000 peaks, noise +-xi, 1e-4 (seed 7)
=====================  =========================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

DEFAULT_PEAK_DENSITY = 20000.0 / (1024 * 1024 * 512)


def build(force: bool = False) -> str:
    """Compile synth.c into _build/libsynth.so when missing or stale."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.syn_perlin.argtypes = [P, I64, I64, I64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64]
            lib.syn_peaks.argtypes = [P, I64, I64, I64, I64, ctypes.c_double, ctypes.c_uint64]
            lib.syn_perturb_uniform.argtypes = [P, P, I64, ctypes.c_float, ctypes.c_uint64]
            lib.syn_prequantize.argtypes = [P, P, I64, ctypes.c_float]
            lib.syn_minmax.argtypes = [P, I64, P, P]
            lib.syn_uniform.argtypes = [P, I64, ctypes.c_uint64, ctypes.c_uint64]
            lib.syn_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.syn_rand.restype = ctypes.c_uint64
            lib.syn_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _dims(shape):
    if len(shape) == 2:
        ny, nx = shape
        return nx, ny, 1
    nz, ny, nx = shape
    return nx, ny, nz


def perlin(shape, octaves: int = 5, period: float = 64.0, seed: int = 0) -> np.ndarray:
    """Fractal Perlin noise scaled to [0, 1]; shape (ny, nx) or (nz, ny, nx)."""
    out = np.empty(shape, dtype=np.float32)
    nx, ny, nz = _dims(shape)
    _load().syn_perlin(_ptr(out), nx, ny, nz, octaves, period, seed)
    return out


def peaks(shape, npeaks: int | None = None, lam: float = 5.0, seed: int = 0) -> np.ndarray:
    """Poisson(lam) background plus isotropic Gaussian peaks, scaled to [0, 1]."""
    out = np.empty(shape, dtype=np.float32)
    nx, ny, nz = _dims(shape)
    if npeaks is None:
        npeaks = max(1, int(round(DEFAULT_PEAK_DENSITY * nx * ny * nz)))
    _load().syn_peaks(_ptr(out), nx, ny, nz, npeaks, lam, seed)
    return out


def perturb_uniform(f: np.ndarray, xi: float, seed: int) -> np.ndarray:
    """fhat = f + U[-xi, xi] (double), rounded to float32 and kept inside the bound."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    out = np.empty_like(f)
    _load().syn_perturb_uniform(_ptr(f), _ptr(out), f.size, np.float32(xi), seed)
    return out


def prequantize(f: np.ndarray, xi: float) -> np.ndarray:
    """fhat = 2 xi * round(f / 2 xi) (ties to even, double), kept inside the bound."""
    f = np.ascontiguousarray(f, dtype=np.float32)
    out = np.empty_like(f)
    _load().syn_prequantize(_ptr(f), _ptr(out), f.size, np.float32(xi))
    return out


def uniform(n: int, seed: int, stream: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().syn_uniform(_ptr(out), n, seed, stream)
    return out


def rand_u64(key: int, i: int) -> int:
    return int(_load().syn_rand(key, i))


def threads() -> int:
    return int(_load().syn_threads())


def xi_from_relative(f: np.ndarray, eb_rel: float) -> np.float32:
    """xi = float32(eb_rel * (max f - min f)), the product taken in double."""
    lo = ctypes.c_float()
    hi = ctypes.c_float()
    f = np.ascontiguousarray(f, dtype=np.float32)
    _load().syn_minmax(_ptr(f), f.size, ctypes.byref(lo), ctypes.byref(hi))
    return np.float32(float(eb_rel) * (float(hi.value) - float(lo.value)))


class Field:
    """One correction problem: f, fhat, xi and the grid dimensionality."""

    def __init__(self, name: str, f: np.ndarray, fhat: np.ndarray, xi: np.float32, eb_rel: float):
        self.name = name
        self.f = f
        self.fhat = fhat
        self.xi = np.float32(xi)
        self.eb_rel = eb_rel
        self.ndim = f.ndim

    @property
    def shape(self):
        return self.f.shape

    @property
    def n(self) -> int:
        return int(self.f.size)

    def __repr__(self):
        return f"Field({self.name}, shape={self.shape}, xi={float(self.xi):.3g})"


def perlin2d(shape=(256, 256), seed: int = 1, eb_rel: float = 1e-3) -> Field:
    f = perlin(shape, octaves=4, period=64.0, seed=seed)
    xi = xi_from_relative(f, eb_rel)
    return Field(f"perlin2d_{shape[1]}x{shape[0]}", f, perturb_uniform(f, xi, seed), xi, eb_rel)


def perlin3d_prequant(shape=(512, 512, 512), seed: int = 2, eb_rel: float = 1e-4, octaves: int = 5) -> Field:
    f = perlin(shape, octaves=octaves, period=64.0, seed=seed)
    xi = xi_from_relative(f, eb_rel)
    nz, ny, nx = shape
    return Field(f"perlin3d_prequant_{nx}x{ny}x{nz}", f, prequantize(f, xi), xi, eb_rel)


def peaks3d(shape=(512, 1024, 1024), seed: int = 3, eb_rel: float = 1e-4, npeaks: int | None = None) -> Field:
    f = peaks(shape, npeaks=npeaks, lam=5.0, seed=seed)
    xi = xi_from_relative(f, eb_rel)
    nz, ny, nx = shape
    return Field(f"peaks3d_{nx}x{ny}x{nz}", f, perturb_uniform(f, xi, seed), xi, eb_rel)


def batch_shapes(count: int = 64, lo: int = 64, hi: int = 384, seed: int = 1000):
    """Per-field (shape, eb_rel, seed) of the uneven batch: axes ~ U{lo..hi}."""
    ebs = (1e-3, 1e-4, 1e-5)
    out = []
    key = 0x5EED0000 + seed
    for k in range(count):
        ax = [lo + rand_u64(key, 4 * k + c) % (hi - lo + 1) for c in range(3)]
        eb = ebs[rand_u64(key, 4 * k + 3) % 3]
        out.append(((int(ax[2]), int(ax[1]), int(ax[0])), eb, seed + k))
    return out


def batch(count: int = 64, lo: int = 64, hi: int = 384, seed: int = 1000) -> list[Field]:
    fields = []
    for shape, eb, s in batch_shapes(count, lo, hi, seed):
        fields.append(perlin3d_prequant(shape, seed=s, eb_rel=eb))
    return fields
