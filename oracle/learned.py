"""CPU oracle of the learned proposal network (numpy, float64).

TEST INFRASTRUCTURE ONLY: only tests/ and bench.py's CPU arms call it.

The network of the learned initial-edit proposal: four 3x3x3
cross-correlations with zero padding (channels 16 -> 32 -> 32 -> 32 -> 16),
ReLU between; the 16 outputs are the logits of the edit-count classes
k = 0..15, trained with softmax cross-entropy.  Tensors are channels-last
([z][y][x][C]); weights w[o][cout][cin] with kernel offset
o = (dz+1)*9 + (dy+1)*3 + (dx+1) applied to input voxel (x+dx, y+dy, z+dz).

Every sum is taken in float64.  `bf16_points=True` rounds to bfloat16 (round
to nearest even) where the GPU stores BFloat16: the input features, the
weights, the activations after each ReLU and the gradients between layers --
so that the GPU (FP32 accumulation) and this oracle differ only by the order
and precision of the sums.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
CHANNELS = (16, 32, 32, 32, 16)
CLASSES = 16


def bf16(a) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def conv3d(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """y[v, co] = sum_o sum_ci w[o, co, ci] * x[v + d_o, ci] (zero outside)."""
    nz, ny, nx, _ = x.shape
    xp = np.zeros((nz + 2, ny + 2, nx + 2, x.shape[3]))
    xp[1:-1, 1:-1, 1:-1] = x
    y = np.zeros((nz, ny, nx, w.shape[1]))
    for o, (dx, dy, dz) in enumerate(OFFSETS):
        y += xp[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx] @ w[o].T
    return y


def conv3d_transpose(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3d in x: dx[v + d_o, ci] += sum_co dy[v, co] * w[o, co, ci]."""
    nz, ny, nx, _ = dy.shape
    dxp = np.zeros((nz + 2, ny + 2, nx + 2, w.shape[2]))
    for o, (dx, dyy, dz) in enumerate(OFFSETS):
        dxp[1 + dz:1 + dz + nz, 1 + dyy:1 + dyy + ny, 1 + dx:1 + dx + nx] += dy @ w[o]
    return dxp[1:-1, 1:-1, 1:-1]


def conv3d_wgrad(x: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """dw[o, co, ci] = sum_v dy[v, co] * x[v + d_o, ci]."""
    nz, ny, nx, _ = x.shape
    xp = np.zeros((nz + 2, ny + 2, nx + 2, x.shape[3]))
    xp[1:-1, 1:-1, 1:-1] = x
    dw = np.zeros((27, dy.shape[3], x.shape[3]))
    dyf = dy.reshape(-1, dy.shape[3])
    for o, (dx, dyy, dz) in enumerate(OFFSETS):
        xs = xp[1 + dz:1 + dz + nz, 1 + dyy:1 + dyy + ny, 1 + dx:1 + dx + nx].reshape(-1, x.shape[3])
        dw[o] = dyf.T @ xs
    return dw


def softmax(z):
    e = np.exp(z - z.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def cross_entropy(z, k):
    """Softmax cross-entropy of logits z [..., C] against classes k [...]."""
    m = z.max(axis=-1)
    lse = m + np.log(np.exp(z - m[..., None]).sum(axis=-1))
    return lse - np.take_along_axis(z, k[..., None].astype(np.int64), axis=-1)[..., 0]


def forward(feat: np.ndarray, params, bf16_points: bool = True) -> dict:
    """params: [(w1, b1), .., (w4, b4)] with w_l [27, cout, cin].  Returns the
    activations x0 (features) .. x3, the logits z and the class probabilities p."""
    rd = bf16 if bf16_points else (lambda a: np.asarray(a, dtype=np.float64))
    acts = {"x0": rd(feat)}
    x = acts["x0"]
    for l in range(3):
        w, b = params[l]
        x = rd(np.maximum(conv3d(x, rd(w)) + b, 0.0))
        acts[f"x{l + 1}"] = x
    w, b = params[3]
    z = conv3d(x, rd(w)) + b
    acts["z"] = z
    acts["p"] = softmax(z)
    return acts


def backward(acts: dict, k: np.ndarray, params, scale: float, bf16_points: bool = True):
    """Gradients of scale * sum CE(z, k) with respect to every weight and bias:
    [(dw1, db1), .., (dw4, db4)], and the loss sum CE(z, k)."""
    rd = bf16 if bf16_points else (lambda a: np.asarray(a, dtype=np.float64))
    onehot = np.eye(acts["z"].shape[-1])[k.astype(np.int64)]
    dz = rd(scale * (acts["p"] - onehot))
    grads = [None] * 4
    grads[3] = (conv3d_wgrad(acts["x3"], dz), dz.sum(axis=(0, 1, 2)))
    for l in (2, 1, 0):
        w_next = rd(params[l + 1][0])
        dx = conv3d_transpose(dz, w_next)
        dz = rd(np.where(acts[f"x{l + 1}"] > 0, dx, 0.0))
        grads[l] = (conv3d_wgrad(acts[f"x{l}"], dz), dz.sum(axis=(0, 1, 2)))
    return grads, float(cross_entropy(acts["z"], k).sum())


def edit_count(fhat: float, g: float, L: float, halve, cap: int = CLASSES - 1) -> int:
    """Number of applications of the edit `halve(g, L) -> (g', changed)` that
    take fhat down to g (capped)."""
    h, k = np.float32(fhat), 0
    while k < cap and h > g:
        h, changed = halve(h, L)
        if not changed:
            break
        k += 1
    return k
