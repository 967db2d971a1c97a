"""Learned initial-edit proposal: binding, network, training and inference.

A 4-layer 3D conv net (3x3x3 kernels, zero padding, 16 -> 32 -> 32 -> 32 -> 16
channels, ReLU between) classifies each vertex by k = 0..15, the number of
HALVE edits the plain correction loop applies to it (15: fifteen or more).
The start g0 = fhat edited k times by that same rule goes to msz_correct as
its initial field and the exact loop finishes from there, so the result is
checked by the same loop and the same invariant check as the plain method; a
vertex whose class is right starts at exactly the plain loop's final value.

Every tensor operation of the network -- features, the conv layers on tcgen05,
the loss head, backward-data, weight gradients and Adam -- runs in the kernels
of msz_learned.cu through the C ABI; PyTorch only holds device memory.
Activations are channels-last BF16 tensors of shape [N, C]; weights are FP32
masters w[27][cout][cin] (kernel offset o = (dz+1)*9 + (dy+1)*3 + (dx+1)
applied to input voxel (x+dx, y+dy, z+dz)) from which BF16 images are built
before each use.
"""
from __future__ import annotations

import ctypes
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api

# (cin_real, cout_real, cin, cout): real channel counts and the padded ones the
# conv kernels run with
LAYERS = ((16, 32, 16, 32), (32, 32, 32, 32), (32, 32, 32, 32), (32, 16, 32, 16))
MODE_RELU, MODE_HEAD, MODE_DGRAD, MODE_RAW = 0, 1, 2, 3
FEATURES = 16  # input channels per vertex
CLASSES = 16   # edit-count classes of the head
SHIFT = 2      # added to nonzero classes at inference: a slight overshoot settles distortions sooner
_typed = False


def lib():
    """libmsz.so with the learned entry points typed."""
    global _typed
    L = api.load()
    if not _typed:
        P, I32, I64, F, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
        st = ctypes.c_int
        L.msz_learned_features.argtypes = [P, P, F, api.Grid, P, P, P, P]
        L.msz_learned_weight_image_size.argtypes = [I32, I32]
        L.msz_learned_weight_image_size.restype = SZ
        L.msz_learned_weight_image.argtypes = [P, I32, I32, I32, I32, I32, P, P]
        L.msz_learned_conv.argtypes = [P, I32, I32, I32, api.Grid, P, P, P, P, P, P, P, F, I32, P, P, P]
        L.msz_learned_head_grad.argtypes = [P, P, I64, F, P, P, P]
        L.msz_learned_target.argtypes = [P, P, P, F, I64, P, P]
        L.msz_learned_wgrad.argtypes = [P, I32, P, I32, api.Grid, I32, I32, P, P, P, ctypes.c_size_t, P]
        L.msz_learned_wgrad_workspace_size.argtypes = [I32, I32]
        L.msz_learned_wgrad_workspace_size.restype = ctypes.c_size_t
        L.msz_learned_adam.argtypes = [P, P, P, P, I64, F, F, F, F, I64, P]
        for name in ("features", "weight_image", "conv", "head_grad", "target", "wgrad", "adam"):
            getattr(L, "msz_learned_" + name).restype = st
        _typed = True
    return L


def _check(status: int, what: str) -> None:
    if status != api.OK:
        raise api.MszError(status, what)


def _p(t):
    return api._dptr(t)


def _s(stream):
    return api._stream(stream)


def _grid(shape) -> api.Grid:
    if len(shape) != 3:
        raise ValueError("the learned proposal works on 3D grids")
    return api.grid_of(shape)


# ----------------------------------------------------------------- kernels

def features(f: torch.Tensor, fhat: torch.Tensor, xi: float, codes_f=None, codes_h=None, out=None,
             stream=None) -> torch.Tensor:
    """[N, 16] BF16 input channels of the network (msz_learned_features)."""
    if codes_f is None:
        codes_f = api.directions(f, stream=stream)
    if codes_h is None:
        codes_h = api.directions(fhat, stream=stream)
    if out is None:
        out = torch.empty(f.numel(), FEATURES, dtype=torch.bfloat16, device=f.device)
    _check(lib().msz_learned_features(_p(f), _p(fhat), ctypes.c_float(np.float32(xi)), _grid(f.shape),
                                      _p(codes_f), _p(codes_h), _p(out), _s(stream)), "msz_learned_features")
    return out


def weight_image(w: torch.Tensor, cin: int, cout: int, mirror: bool = False, out=None, stream=None) -> torch.Tensor:
    """BF16 weight image of FP32 weights w [27, cout_real, cin_real]."""
    nbytes = int(lib().msz_learned_weight_image_size(cin, cout))
    if out is None:
        out = torch.empty(nbytes // 2, dtype=torch.bfloat16, device=w.device)
    _check(lib().msz_learned_weight_image(_p(w), int(w.shape[1]), int(w.shape[2]), cin, cout, int(mirror), _p(out),
                                          _s(stream)), "msz_learned_weight_image")
    return out


def conv(x: torch.Tensor, cin: int, cout: int, mode: int, shape, img: torch.Tensor, err: torch.Tensor, *,
         bias=None, out_bf16=None, out_f32=None, mask=None, f=None, fhat=None, xi: float = 0.0,
         shift: int = 0, g0=None, stream=None) -> None:
    """One 3x3x3 conv layer on the tensor cores (msz_learned_conv)."""
    _check(lib().msz_learned_conv(_p(x), cin, cout, mode, _grid(shape), _p(img), _p(bias), _p(out_bf16),
                                  _p(out_f32), _p(mask), _p(f), _p(fhat), ctypes.c_float(np.float32(xi)),
                                  int(shift), _p(g0), _p(err), _s(stream)), "msz_learned_conv")


def head_grad(z: torch.Tensor, target: torch.Tensor, scale: float, dz16: torch.Tensor, loss: torch.Tensor,
              stream=None) -> None:
    _check(lib().msz_learned_head_grad(_p(z), _p(target), target.numel(), ctypes.c_float(scale), _p(dz16),
                                       _p(loss), _s(stream)), "msz_learned_head_grad")


def target(f: torch.Tensor, fhat: torch.Tensor, g: torch.Tensor, xi: float, out=None, stream=None) -> torch.Tensor:
    """Training classes: HALVE edits from fhat to g, capped at 15 (msz_learned_target)."""
    if out is None:
        out = torch.empty_like(f)
    _check(lib().msz_learned_target(_p(f), _p(fhat), _p(g), ctypes.c_float(np.float32(xi)), f.numel(), _p(out),
                                    _s(stream)), "msz_learned_target")
    return out


_wgrad_ws: dict = {}


def wgrad(x: torch.Tensor, cin: int, dz: torch.Tensor, cout: int, shape, dw: torch.Tensor, db: torch.Tensor,
          stream=None) -> None:
    """dw += sum_v dz[v] x[v + d_o]^T, db += sum_v dz[v] (msz_learned_wgrad;
    deterministic: partial sums in a cached workspace, added in a fixed order)."""
    need = int(lib().msz_learned_wgrad_workspace_size(cin, cout))
    key = x.device.index
    ws = _wgrad_ws.get(key)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=x.device)
        _wgrad_ws[key] = ws
    _check(lib().msz_learned_wgrad(_p(x), cin, _p(dz), cout, _grid(shape), int(dw.shape[2]), int(dw.shape[1]),
                                   _p(dw), _p(db), _p(ws), ws.numel(), _s(stream)), "msz_learned_wgrad")


def adam(p, g, m, v, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    _check(lib().msz_learned_adam(_p(p), _p(g), _p(m), _p(v), p.numel(), ctypes.c_float(lr), ctypes.c_float(beta1),
                                  ctypes.c_float(beta2), ctypes.c_float(eps), int(step), _s(stream)),
           "msz_learned_adam")


# ----------------------------------------------------------------- network

class ProposalNet:
    """FP32 master parameters in one flat buffer (weights and padded biases of
    the four layers), their gradients and Adam moments, and the BF16 images."""

    def __init__(self, seed: int = 0, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        sizes = []
        for cin_r, cout_r, cin, cout in LAYERS:
            sizes += [27 * cout_r * cin_r, cout]
        self.sizes = sizes
        total = sum(sizes)
        self.flat = torch.zeros(total, dtype=torch.float32, device=self.device)
        self.grad = torch.zeros_like(self.flat)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        self.w, self.b, self.dw, self.db = [], [], [], []
        off = 0
        for (cin_r, cout_r, cin, cout) in LAYERS:
            nw = 27 * cout_r * cin_r
            self.w.append(self.flat[off:off + nw].view(27, cout_r, cin_r))
            self.dw.append(self.grad[off:off + nw].view(27, cout_r, cin_r))
            off += nw
            self.b.append(self.flat[off:off + cout])
            self.db.append(self.grad[off:off + cout])
            off += cout
        gen = torch.Generator().manual_seed(int(seed))
        for l, (cin_r, cout_r, _, _) in enumerate(LAYERS):
            std = math.sqrt(2.0 / (27 * cin_r)) * (0.1 if l == 3 else 1.0)
            self.w[l].copy_(torch.randn(27, cout_r, cin_r, generator=gen) * std)
        self.steps = 0
        self.err = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._img = [None] * 4
        self._mimg = [None] * 4
        self._bufs = {}

    # -- parameters
    def state(self) -> dict:
        return {"flat": self.flat.cpu().numpy().copy(), "layers": np.array(LAYERS), "steps": self.steps}

    def load_state(self, st: dict) -> "ProposalNet":
        flat = np.asarray(st["flat"], dtype=np.float32)
        if flat.size != self.flat.numel() or not np.array_equal(np.asarray(st["layers"]), np.array(LAYERS)):
            raise ValueError("parameter layout mismatch")
        self.flat.copy_(torch.from_numpy(flat))
        self.steps = int(st.get("steps", 0))
        return self

    def save(self, path: str) -> None:
        np.savez(path, **self.state())

    @classmethod
    def from_file(cls, path: str, device=None) -> "ProposalNet":
        with np.load(path) as z:
            return cls(device=device).load_state({k: z[k] for k in z.files})

    def params_numpy(self):
        """[(w, b)] as float64 numpy arrays with the real channel counts."""
        out = []
        for l, (cin_r, cout_r, _, _) in enumerate(LAYERS):
            out.append((self.w[l].double().cpu().numpy(), self.b[l][:cout_r].double().cpu().numpy()))
        return out

    def build_images(self, mirror: bool = False, stream=None) -> None:
        for l, (_, _, cin, cout) in enumerate(LAYERS):
            self._img[l] = weight_image(self.w[l], cin, cout, False, self._img[l], stream)
            if mirror and l > 0:
                self._mimg[l] = weight_image(self.w[l], cout, cin, True, self._mimg[l], stream)

    def check(self) -> None:
        if int(self.err.item()) != 0:
            raise api.MszError(api.ERR_TIMEOUT, "msz_learned_conv (bounded wait)")

    def _buf(self, name, n, c, dtype):
        t = self._bufs.get(name)
        if t is None or t.shape[0] < n or t.shape[1] != c or t.dtype != dtype:
            t = torch.empty(n, c, dtype=dtype, device=self.device)
            self._bufs[name] = t
        return t[:n]

    def release(self) -> None:
        self._bufs.clear()

    # -- forward / backward
    def forward(self, x0: torch.Tensor, shape, keep: bool = True, stream=None):
        """Activations [x0, x1, x2, x3] (BF16) and the head logits z ([N, 16]
        FP32).  keep=False reuses two buffers."""
        n = x0.shape[0]
        acts = [x0]
        for l in range(3):
            name = f"x{l + 1}" if keep else f"p{l % 2}"
            out = self._buf(name, n, 32, torch.bfloat16)
            _, _, cin, cout = LAYERS[l]
            conv(acts[-1], cin, cout, MODE_RELU, shape, self._img[l], self.err, bias=self.b[l], out_bf16=out,
                 stream=stream)
            acts.append(out)
        z = self._buf("z", n, 16, torch.float32)
        conv(acts[3], 32, 16, MODE_RAW, shape, self._img[3], self.err, bias=self.b[3], out_f32=z, stream=stream)
        return acts, z

    def backward(self, acts, z, tgt: torch.Tensor, shape, scale: float, stream=None) -> torch.Tensor:
        """Accumulate the gradients of scale * sum CE(z, k) into self.grad
        (k: classes as float); returns the device scalar sum CE (float64)."""
        n = tgt.numel()
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        dz4 = self._buf("dz4", n, 16, torch.bfloat16)
        head_grad(z, tgt, scale, dz4, loss, stream)
        wgrad(acts[3], 32, dz4, 16, shape, self.dw[3], self.db[3], stream)
        cur, cin_cur = dz4, 16
        for l in (3, 2, 1):
            nxt = self._buf(f"d{l % 2}", n, 32, torch.bfloat16)
            conv(cur, cin_cur, 32, MODE_DGRAD, shape, self._mimg[l], self.err, out_bf16=nxt, mask=acts[l],
                 stream=stream)
            cin_l = LAYERS[l - 1][2]
            wgrad(acts[l - 1], cin_l, nxt, 32, shape, self.dw[l - 1], self.db[l - 1], stream)
            cur, cin_cur = nxt, 32
        return loss

    def train_step(self, x0, tgt, shape, lr: float, stream=None) -> torch.Tensor:
        self.build_images(mirror=True, stream=stream)
        self.grad.zero_()
        acts, z = self.forward(x0, shape, keep=True, stream=stream)
        loss = self.backward(acts, z, tgt, shape, 1.0 / tgt.numel(), stream)
        self.steps += 1
        adam(self.flat, self.grad, self.m, self.v, lr, self.steps, stream=stream)
        return loss

    # -- inference
    def propose(self, f: torch.Tensor, fhat: torch.Tensor, xi: float, shift: int = SHIFT, out=None, k_out=None,
                stream=None) -> torch.Tensor:
        """The proposed start g0 (FP32, shape of f) for msz_correct's g_init;
        k_out (optional, FP32 [N]) receives the class used per vertex."""
        shape = tuple(f.shape)
        n = f.numel()
        x0 = features(f, fhat, xi, out=self._buf("x0", n, FEATURES, torch.bfloat16), stream=stream)
        self.build_images(stream=stream)
        acts = [x0]
        for l in range(3):
            out_l = self._buf(f"p{l % 2}", n, 32, torch.bfloat16)
            _, _, cin, cout = LAYERS[l]
            conv(acts[-1], cin, cout, MODE_RELU, shape, self._img[l], self.err, bias=self.b[l], out_bf16=out_l,
                 stream=stream)
            acts.append(out_l)
        if out is None:
            out = torch.empty_like(f)
        conv(acts[3], 32, 16, MODE_HEAD, shape, self._img[3], self.err, bias=self.b[3], out_f32=k_out, f=f,
             fhat=fhat, xi=xi, shift=shift, g0=out, stream=stream)
        return out


# ----------------------------------------------------------------- training

@dataclass
class Sample:
    f: torch.Tensor
    fhat: torch.Tensor
    xi: float
    target: torch.Tensor  # class per vertex (FP32)
    sweeps: int
    edited: int


def make_sample(fl, device=None) -> Sample:
    """One training triple: the plain loop's result on (f, fhat) as targets."""
    f = torch.from_numpy(fl.f).to(device or "cuda")
    fh = torch.from_numpy(fl.fhat).to(f.device)
    res = api.correct(f, fh, float(fl.xi), edit_capacity=0)
    if res.status not in (api.OK, api.ERR_CAPACITY):
        raise api.MszError(res.status, "training triple")
    t = target(f, fh, res.out, float(fl.xi))
    return Sample(f, fh, float(fl.xi), t, res.stats["sweeps"], res.stats["edited"])


def training_set(count: int = 200, shape=(128, 128, 128), eb_rel: float = 1e-4, seed0: int = 5000,
                 device=None) -> list[Sample]:
    """`count` seeded Gaussian-peak fields with uniform noise (the peak density
    of the large peak workload) and the plain loop's results."""
    from . import synth
    return [make_sample(synth.peaks3d(tuple(shape), seed=seed0 + k, eb_rel=eb_rel), device) for k in range(count)]


@dataclass
class TrainLog:
    epochs: list = field(default_factory=list)  # (epoch, mean loss, seconds)


def train(net: ProposalNet, data: list[Sample], epochs: int = 4, lr: float = 1e-3, seed: int = 0,
          lr_final: float | None = None, log: TrainLog | None = None, verbose: bool = False) -> TrainLog:
    """Adam on the per-sample mean softmax cross-entropy, one sample per step,
    in a seeded order; linear warm-up over the first 5% of the steps, then
    cosine decay from lr to lr_final."""
    log = log or TrainLog()
    rng = np.random.default_rng(seed)
    total = epochs * len(data)
    lr_final = lr * 0.05 if lr_final is None else lr_final
    it = 0
    for ep in range(epochs):
        t0 = time.perf_counter()
        losses = []
        for k in rng.permutation(len(data)):
            s = data[k]
            x0 = features(s.f, s.fhat, s.xi, out=net._buf("x0", s.f.numel(), FEATURES, torch.bfloat16))
            warm = min(1.0, (it + 1) / max(1, total // 20))
            cur = warm * (lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / max(total - 1, 1))))
            losses.append(net.train_step(x0, s.target.view(-1), tuple(s.f.shape), cur))
            it += 1
        mean = float(torch.cat(losses).sum().item()) / sum(s.f.numel() for s in data)
        net.check()
        log.epochs.append((ep, mean, time.perf_counter() - t0))
        if verbose:
            print(f"epoch {ep}: loss {mean:.6f} ({log.epochs[-1][2]:.1f} s)", flush=True)
    return log


# recipe of the default network: 200 seeded 128^3 Gaussian-peak fields (the
# peak density of the 1024 x 1024 x 512 workload), relative bound 1e-4, uniform
# noise, the plain loop's classes as targets
RECIPE = {"count": 200, "shape": (128, 128, 128), "eb_rel": 1e-4, "seed0": 5000, "epochs": 12, "lr": 2e-3,
          "init_seed": 1, "order_seed": 0}


def _cache_path(recipe: dict) -> str:
    import hashlib
    import json
    import os

    from . import _build
    key = hashlib.sha256((_build.source_hash() + json.dumps(recipe, sort_keys=True)).encode()).hexdigest()[:16]
    return os.path.join(os.path.dirname(_build.LIB), f"proposal_{key}.npz")


def default_net(device=None, train_if_missing: bool = True, recipe: dict | None = None, verbose: bool = False):
    """The network trained by `recipe` (default RECIPE) with the compiled
    library's kernels, cached next to the library; returns (net, info)."""
    import os
    recipe = dict(RECIPE if recipe is None else recipe)
    path = _cache_path(recipe)
    if os.path.exists(path):
        net = ProposalNet.from_file(path, device=device)
        with np.load(path) as z:
            info = {"cached": True, "train_s": float(z["train_s"]) if "train_s" in z.files else None,
                    "final_loss": float(z["final_loss"]) if "final_loss" in z.files else None}
        return net, info
    if not train_if_missing:
        raise FileNotFoundError(path)
    t0 = time.perf_counter()
    data = training_set(recipe["count"], recipe["shape"], recipe["eb_rel"], recipe["seed0"], device)
    t1 = time.perf_counter()
    net = ProposalNet(seed=recipe["init_seed"], device=device)
    log = train(net, data, epochs=recipe["epochs"], lr=recipe["lr"], seed=recipe["order_seed"], verbose=verbose)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del data
    info = {"cached": False, "data_s": t1 - t0, "train_s": t2 - t1, "final_loss": log.epochs[-1][1]}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, **net.state(), train_s=info["train_s"], final_loss=info["final_loss"])
    return net, info


# ----------------------------------------------------------------- inference

@dataclass
class LearnedResult:
    result: api.CorrectResult   # the exact loop's result (from g0, or from fhat after a fallback)
    fallback: bool              # the loop from g0 ended STUCK / capped and was rerun from fhat
    from_g0: api.CorrectResult  # the run from g0
    propose_ms: float


def correct_learned(f: torch.Tensor, fhat: torch.Tensor, xi: float, net: ProposalNet, shift: int = SHIFT,
                    **kw) -> LearnedResult:
    """Proposal, then the exact correction loop from it; when that loop ends
    without a correct field (STUCK or at its sweep cap) the plain loop from
    fhat runs instead, so the outcome is always the exact method's."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g0 = net.propose(f, fhat, xi, shift=shift)
    e1.record()
    r = api.correct(f, fhat, xi, g_init=g0, **kw)
    net.check()
    ms = e0.elapsed_time(e1)
    if r.status in (api.STUCK, api.ERR_MAX_SWEEPS):
        return LearnedResult(api.correct(f, fhat, xi, **kw), True, r, ms)
    return LearnedResult(r, False, r, ms)
