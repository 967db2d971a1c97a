"""The learned proposal's kernels against the CPU oracle (oracle/learned.py).

Every conv is checked in isolation on the GPU's own BF16 inputs: the FP32
tensor-core result against the float64 oracle within the accumulation bound
derived below, and the fused epilogues (bias + ReLU, ReLU mask, the head)
bit for bit against the RAW result.  Weight gradients, the loss head and Adam
follow, then the whole backward pass against the oracle's, and training.

Tolerance of an FP32 sum of K products of BF16 numbers (each product exact in
FP32): |error| <= K * 2^-23 * sum|terms|.  With K = 27 * 32 = 864 that is
1.03e-4 of sum|terms|; the tests use 2e-4, while one dropped or misplaced term
of average size is 1/864 = 1.16e-3 of it.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import learned as OL
from paper_2601_01787_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(3, 5, 130), (4, 4, 256), (2, 3, 300)]  # (nz, ny, nx): ragged tiles in x, y and z


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2601_01787_gb300 import learned
    learned.lib()
    return learned


def bf16_tensor(a, c_pad=None):
    """Host array [N, C] -> device BF16 (values rounded to BF16)."""
    a = np.asarray(a, dtype=np.float32)
    if c_pad is not None and a.shape[1] < c_pad:
        a = np.concatenate([a, np.zeros((a.shape[0], c_pad - a.shape[1]), np.float32)], axis=1)
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16).cuda()


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def err_word():
    return torch.zeros(1, dtype=torch.int32, device="cuda")


def weights(cout_r, cin_r, seed, scale=None):
    rng = np.random.default_rng(seed)
    s = scale if scale is not None else math.sqrt(2.0 / (27 * cin_r))
    return (rng.standard_normal((27, cout_r, cin_r)) * s).astype(np.float32)


def acts(shape, c, seed, relu=False):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((int(np.prod(shape)), c)).astype(np.float32)
    return np.maximum(a, 0) if relu else a


def close(got, ref, bound, factor=2e-4, what=""):
    err = np.abs(got - ref)
    lim = factor * bound + 1e-30
    bad = err > lim
    assert not bad.any(), f"{what}: {bad.sum()} entries off, worst {err[bad].max()} vs {lim[bad].min()}"


# ------------------------------------------------------------------ conv
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("cin_r,cout_r,cin,cout", [(8, 32, 16, 32), (32, 32, 32, 32), (32, 16, 32, 16), (32, 1, 32, 16)])
def test_conv_raw_matches_oracle(L, shape, cin_r, cout_r, cin, cout):
    n = int(np.prod(shape))
    x = bf16_tensor(acts(shape, cin, 100 + cin), cin)
    w = weights(cout_r, cin_r, 200 + cout_r)
    b = np.random.default_rng(3).standard_normal(cout).astype(np.float32)
    b[cout_r:] = 0
    wt = torch.from_numpy(w).cuda()
    img = L.weight_image(wt, cin, cout)
    out = torch.empty(n, cout, dtype=torch.float32, device="cuda")
    err = err_word()
    L.conv(x, cin, cout, L.MODE_RAW, shape, img, err, bias=torch.from_numpy(b).cuda(), out_f32=out)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    xh = host(x).reshape(*shape, cin)[..., :cin_r]
    wb = OL.bf16(w)
    ref = OL.conv3d(xh, wb) + b[:cout_r]
    bound = OL.conv3d(np.abs(xh), np.abs(wb)) + np.abs(b[:cout_r])
    got = host(out).reshape(*shape, cout)
    close(got[..., :cout_r], ref, bound, what="conv raw")
    assert np.all(got[..., cout_r:] == 0.0)


@pytest.mark.parametrize("cin", [16, 32])
def test_conv_relu_epilogue_bitwise(L, cin):
    shape = (3, 5, 130)
    n = int(np.prod(shape))
    x = bf16_tensor(acts(shape, cin, 7), cin)
    wt = torch.from_numpy(weights(32, cin, 8)).cuda()
    bias = torch.from_numpy(np.random.default_rng(9).standard_normal(32).astype(np.float32)).cuda()
    img = L.weight_image(wt, cin, 32)
    raw = torch.empty(n, 32, dtype=torch.float32, device="cuda")
    out = torch.empty(n, 32, dtype=torch.bfloat16, device="cuda")
    err = err_word()
    L.conv(x, cin, 32, L.MODE_RAW, shape, img, err, bias=bias, out_f32=raw)
    L.conv(x, cin, 32, L.MODE_RELU, shape, img, err, bias=bias, out_bf16=out)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = torch.clamp(raw, min=0.0).to(torch.bfloat16)
    assert torch.equal(out.view(torch.int16), ref.view(torch.int16))


@pytest.mark.parametrize("shape", SHAPES[:2])
@pytest.mark.parametrize("cout_r,cin_r,cin_img,cout_img", [(32, 32, 32, 32), (16, 32, 16, 32), (1, 32, 16, 32)])
def test_conv_dgrad_matches_oracle(L, shape, cout_r, cin_r, cin_img, cout_img):
    """Backward-data of a forward conv with cin_r inputs and cout_r outputs:
    dx = conv_transpose(dy, w), masked by the forward input's ReLU."""
    n = int(np.prod(shape))
    dy = bf16_tensor(acts(shape, cin_img, 11), cin_img)
    mask = bf16_tensor(acts(shape, cout_img, 12), cout_img)
    w = weights(cout_r, cin_r, 13)
    wt = torch.from_numpy(w).cuda()
    img = L.weight_image(wt, cin_img, cout_img, mirror=True)
    raw = torch.empty(n, cout_img, dtype=torch.float32, device="cuda")
    out = torch.empty(n, cout_img, dtype=torch.bfloat16, device="cuda")
    err = err_word()
    L.conv(dy, cin_img, cout_img, L.MODE_RAW, shape, img, err, out_f32=raw)
    L.conv(dy, cin_img, cout_img, L.MODE_DGRAD, shape, img, err, out_bf16=out, mask=mask)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    dyh = host(dy).reshape(*shape, cin_img)[..., :cout_r]
    wb = OL.bf16(w)
    ref = OL.conv3d_transpose(dyh, wb)
    bound = OL.conv3d_transpose(np.abs(dyh), np.abs(wb))
    close(host(raw).reshape(*shape, cout_img)[..., :cin_r], ref, bound, what="dgrad raw")
    expect = torch.where(mask > 0, raw, torch.zeros_like(raw)).to(torch.bfloat16)
    assert torch.equal(out.view(torch.int16), expect.view(torch.int16))


# --------------------------------------------------------- weight grads
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("cin_r,cout_r,cin,cout", [(8, 32, 16, 32), (32, 32, 32, 32), (32, 16, 32, 16), (32, 1, 32, 16)])
def test_wgrad_matches_oracle(L, shape, cin_r, cout_r, cin, cout):
    x = bf16_tensor(acts(shape, cin, 21, relu=True), cin)
    dz = bf16_tensor(acts(shape, cout, 22), cout)
    dw = torch.zeros(27, cout_r, cin_r, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    dw.add_(0.5)  # accumulates into what is there
    L.wgrad(x, cin, dz, cout, shape, dw, db)
    torch.cuda.synchronize()
    xh = host(x).reshape(*shape, cin)[..., :cin_r]
    dzh = host(dz).reshape(*shape, cout)[..., :cout_r]
    ref = OL.conv3d_wgrad(xh, dzh) + 0.5
    bound = OL.conv3d_wgrad(np.abs(xh), np.abs(dzh)) + 0.5
    close(host(dw), ref, bound, factor=1e-4, what="wgrad")
    close(host(db)[:cout_r], dzh.sum(axis=(0, 1, 2)), np.abs(dzh).sum(axis=(0, 1, 2)), factor=1e-4, what="db")
    assert np.all(host(db)[cout_r:] == 0)


# ------------------------------------------------------ head, target, adam
def test_head_grad_matches_oracle(L):
    n = 5000
    rng = np.random.default_rng(31)
    z = (rng.standard_normal((n, 16)) * 4).astype(np.float32)
    z[:20, 3] = 80.0  # a dominant logit
    k = rng.integers(0, 16, n)
    k[:10] = 3
    dz = torch.empty(n, 16, dtype=torch.bfloat16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    scale = 1.0 / n
    L.head_grad(torch.from_numpy(z).cuda(), torch.from_numpy(k.astype(np.float32)).cuda(), scale, dz, loss)
    torch.cuda.synchronize()
    zz = z.astype(np.float64)
    ref = scale * (OL.softmax(zz) - np.eye(16)[k])
    got = host(dz)
    # one BF16 rounding (2^-9 relative) of a value computed in FP32
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6 * scale)
    assert float(loss.item()) == pytest.approx(float(OL.cross_entropy(zz, k).sum()), rel=1e-5)


def halve_chain(fhat, f, xi, k):
    lo = oracle.floor_bound(f, xi)
    g = np.float32(fhat)
    for _ in range(int(k)):
        g, changed = oracle.edit(g, lo)
        if not changed:
            break
    return g


@pytest.mark.parametrize("shift", [0, 2, -3])
def test_head_mode_g0(L, shift):
    shape = (3, 5, 130)
    n = int(np.prod(shape))
    fl = synth.peaks3d(shape, seed=41, eb_rel=1e-3)
    x = bf16_tensor(acts(shape, 32, 42, relu=True), 32)
    w = weights(16, 32, 43, scale=0.05)
    img = L.weight_image(torch.from_numpy(w).cuda(), 32, 16)
    bias = torch.from_numpy(np.random.default_rng(44).standard_normal(16).astype(np.float32) * 0.3).cuda()
    f = torch.from_numpy(fl.f).cuda()
    fh = torch.from_numpy(fl.fhat).cuda()
    kk = torch.empty(n, dtype=torch.float32, device="cuda")
    raw = torch.empty(n, 16, dtype=torch.float32, device="cuda")
    g0 = torch.empty_like(f)
    err = err_word()
    L.conv(x, 32, 16, L.MODE_RAW, shape, img, err, bias=bias, out_f32=raw)
    L.conv(x, 32, 16, L.MODE_HEAD, shape, img, err, bias=bias, out_f32=kk, f=f, fhat=fh, xi=float(fl.xi),
           shift=shift, g0=g0)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    k_ref = raw.cpu().numpy().argmax(axis=1)  # argmax returns the first maximum, as the kernel does
    k_ref = np.where(k_ref > 0, np.clip(k_ref + shift, 1, 15), 0)
    got_k = kk.cpu().numpy().astype(np.int64)
    assert np.array_equal(got_k, k_ref)
    assert len(np.unique(k_ref)) > 4
    g_ref = np.array([halve_chain(a, b, fl.xi, c) for a, b, c in zip(fl.fhat.ravel(), fl.f.ravel(), k_ref)],
                     np.float32)
    assert np.array_equal(g0.cpu().numpy().ravel().view(np.uint32), g_ref.view(np.uint32))


def test_target_classes(L):
    shape = (6, 7, 33)
    fl = synth.peaks3d(shape, seed=44, eb_rel=1e-4)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    from paper_2601_01787_gb300 import api
    res = api.correct(f, fh, float(fl.xi))
    assert res.status == api.OK
    t = L.target(f, fh, res.out, float(fl.xi)).cpu().numpy().ravel()
    g = res.out.cpu().numpy().ravel()
    ref = np.array([OL.edit_count(a, c, oracle.floor_bound(b, fl.xi), oracle.edit)
                    for a, b, c in zip(fl.fhat.ravel(), fl.f.ravel(), g)], np.float32)
    assert np.array_equal(t, ref)
    assert np.array_equal(t == 0, g == fl.fhat.ravel())
    # the chain of t[i] edits from fhat lands on g exactly (below the cap)
    for i in np.flatnonzero((t > 0) & (t < 15))[:300]:
        assert halve_chain(fl.fhat.ravel()[i], fl.f.ravel()[i], fl.xi, t[i]) == g[i]


def test_adam_matches_torch_optim(L):
    rng = np.random.default_rng(51)
    p0 = rng.standard_normal(1000).astype(np.float32)
    grads = [rng.standard_normal(1000).astype(np.float32) for _ in range(5)]
    p = torch.from_numpy(p0.copy()).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    ref = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([ref], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for k, g in enumerate(grads, 1):
        L.adam(p, torch.from_numpy(g).cuda(), m, v, 1e-2, k)
        ref.grad = torch.from_numpy(g)
        opt.step()
    torch.cuda.synchronize()
    np.testing.assert_allclose(p.cpu().numpy(), ref.detach().numpy(), rtol=1e-5, atol=1e-6)


def features_reference(fl):
    """The 16 input channels written out from their definitions with the
    oracle's codes and neighbour table (float32 arithmetic as on the GPU)."""
    shape = fl.f.shape
    inv = np.float32(1) / np.float32(fl.xi)
    inv4 = np.float32(0.25) / np.float32(fl.xi)

    def cl(a, s):
        return np.clip(a.astype(np.float32) * s, -1, 1).astype(np.float32)

    ff, hh = fl.f, fl.fhat
    ch = np.zeros((*shape, 16), np.float32)
    ch[..., 0] = cl(hh - ff, inv)
    for c, src in ((1, ff), (12, hh)):
        ch[:, :, :-1, c] = cl(src[:, :, 1:] - src[:, :, :-1], inv4)
        ch[:, :-1, :, c + 1] = cl(src[:, 1:, :] - src[:, :-1, :], inv4)
        ch[:-1, :, :, c + 2] = cl(src[1:] - src[:-1], inv4)
    cf, cg = oracle.codes(ff), oracle.codes(hh)
    ch[..., 4] = (cf & 15) == 15
    ch[..., 5] = (cf >> 4) == 15
    ch[..., 6] = (cf & 15) != (cg & 15)
    ch[..., 7] = (cf >> 4) != (cg >> 4)
    ch[..., 10] = (cg & 15) == 15
    ch[..., 11] = (cg >> 4) == 15
    flat = ch.reshape(-1, 16)
    cfv, cgv, fv = cf.ravel(), cg.ravel(), ff.ravel()
    for j in range(fv.size):
        a_f, a_g, d_f, d_g = cfv[j] & 15, cgv[j] & 15, cfv[j] >> 4, cgv[j] >> 4
        if a_f != a_g:  # ascending mismatch: itself when fhat makes it a maximum, else fhat's steepest ascent
            flat[j if a_g == 15 else oracle.neighbour(shape, j, int(a_g)), 8] = 1
        if d_f != d_g:  # descending mismatch: itself when f makes it a minimum, else f's steepest descent
            flat[j if d_f == 15 else oracle.neighbour(shape, j, int(d_f)), 9] = 1
        ties = 0
        for sl in range(14):
            k = oracle.neighbour(shape, j, sl)
            ties += k is not None and fv[k] == fv[j]
        flat[j, 15] = np.float32(ties) / np.float32(14)
    return ch


def test_features_bitwise(L):
    shape = (5, 9, 131)
    fl = synth.peaks3d(shape, seed=61, eb_rel=1e-3)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    got = L.features(f, fh, float(fl.xi))
    torch.cuda.synchronize()
    got = got.view(torch.int16).cpu().numpy().view(np.uint16).reshape(*shape, 16)
    ch = features_reference(fl)
    ref = OL.bf16(ch).astype(np.float32).view(np.uint32) >> 16
    assert np.array_equal(got.astype(np.uint32), ref)
    # the case exercises every flag and both sides of the clamp
    for c in (4, 5, 6, 7, 8, 9, 10, 11):
        assert ch[..., c].any(), c
    assert (np.abs(ch[..., 1]) == 1).any() and ((np.abs(ch[..., 1]) < 1) & (ch[..., 1] != 0)).any()
    assert (ch[..., 15] > 0).any()


# ----------------------------------------------------- whole backward pass
def close_bf16(got, ref, bound, factor=2e-4, what=""):
    """got is the BF16 rounding (nearest even, 2^-8 relative at most) of an
    FP32 result within factor * bound of the exact value ref."""
    e = factor * bound
    err = np.abs(got - ref)
    lim = e + 2.0 ** -8 * (np.abs(ref) + e) + 1e-30
    bad = err > lim
    assert not bad.any(), f"{what}: {bad.sum()} entries off, worst {err[bad].max()} vs {lim[bad].min()}"


def test_network_forward_backward_elementwise(L):
    """The whole forward and backward pass of the network, step by step, each
    step element by element against the float64 oracle given the GPU's own
    inputs to that step (so a BF16 rounding flip upstream does not carry into
    the comparison), at the FP32-accumulation bound of the per-kernel tests;
    then the gradients net.backward accumulated equal the step-by-step ones
    bit for bit (every kernel is deterministic)."""
    shape = (4, 6, 130)
    n = int(np.prod(shape))
    fl = synth.peaks3d(shape, seed=71, eb_rel=1e-3)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    net = L.ProposalNet(seed=3)
    x0 = L.features(f, fh, float(fl.xi))
    k = np.random.default_rng(72).integers(0, 16, shape)
    tgt = torch.from_numpy(k.astype(np.float32)).cuda()
    net.build_images(mirror=True)
    net.grad.zero_()
    a, z = net.forward(x0, shape)
    scale = 1.0 / tgt.numel()
    loss = net.backward(a, z, tgt.view(-1), shape, scale)
    torch.cuda.synchronize()
    net.check()
    params = net.params_numpy()
    A = [host(t).reshape(*shape, -1) for t in a]
    # forward: each layer from the GPU's own input
    for l in range(3):
        cin_r, cout_r, _, _ = L.LAYERS[l]
        w, b = params[l]
        wb = OL.bf16(w)
        xin = A[l][..., :cin_r]
        pre = OL.conv3d(xin, wb) + b
        bound = OL.conv3d(np.abs(xin), np.abs(wb)) + np.abs(b)
        close_bf16(A[l + 1][..., :cout_r], np.maximum(pre, 0.0), bound, what=f"x{l + 1}")
    w3, b3 = params[3]
    zref = OL.conv3d(A[3], OL.bf16(w3)) + b3
    close(host(z).reshape(*shape, 16), zref, OL.conv3d(np.abs(A[3]), np.abs(OL.bf16(w3))) + np.abs(b3), what="z")
    zg = host(z).reshape(*shape, 16)
    assert float(loss.item()) == pytest.approx(float(OL.cross_entropy(zg, k).sum()), rel=1e-5)
    # backward, one step at a time on the GPU, each checked on its own inputs
    err = err_word()
    dz = torch.empty(n, 16, dtype=torch.bfloat16, device="cuda")
    L.head_grad(z, tgt.view(-1), scale, dz, torch.zeros(1, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    ref = scale * (OL.softmax(zg) - np.eye(16)[k])
    D = host(dz).reshape(*shape, 16)
    assert np.all(np.abs(D - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6 * scale)
    steps = {}

    def wgrad_step(l, x_t, cin_pad, dz_t, cout_pad):
        cin_r, cout_r, _, _ = L.LAYERS[l]
        dw = torch.zeros(27, cout_r, cin_r, dtype=torch.float32, device="cuda")
        db = torch.zeros(cout_pad, dtype=torch.float32, device="cuda")
        L.wgrad(x_t, cin_pad, dz_t, cout_pad, shape, dw, db)
        torch.cuda.synchronize()
        xh = host(x_t).reshape(*shape, cin_pad)[..., :cin_r]
        dzh = host(dz_t).reshape(*shape, cout_pad)[..., :cout_r]
        close(host(dw), OL.conv3d_wgrad(xh, dzh), OL.conv3d_wgrad(np.abs(xh), np.abs(dzh)), factor=1e-4,
              what=f"dw{l}")
        close(host(db)[:cout_r], dzh.sum(axis=(0, 1, 2)), np.abs(dzh).sum(axis=(0, 1, 2)), factor=1e-4,
              what=f"db{l}")
        steps[l] = (dw, db[:cout_r])

    wgrad_step(3, a[3], 32, dz, 16)
    cur, cin_cur = dz, 16
    for l in (3, 2, 1):
        cin_r, cout_r, _, _ = L.LAYERS[l]
        nxt = torch.empty(n, 32, dtype=torch.bfloat16, device="cuda")
        L.conv(cur, cin_cur, 32, L.MODE_DGRAD, shape, net._mimg[l], err, out_bf16=nxt, mask=a[l])
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        dyh = host(cur).reshape(*shape, cin_cur)[..., :cout_r]
        wb = OL.bf16(params[l][0])
        ref = np.where(A[l][..., :cin_r] > 0, OL.conv3d_transpose(dyh, wb), 0.0)
        bound = OL.conv3d_transpose(np.abs(dyh), np.abs(wb))
        close_bf16(host(nxt).reshape(*shape, 32)[..., :cin_r], ref, bound, what=f"dgrad through layer {l}")
        wgrad_step(l - 1, a[l - 1], L.LAYERS[l - 1][2], nxt, 32)
        cur, cin_cur = nxt, 32
    for l in range(4):
        assert torch.equal(net.dw[l], steps[l][0]), l
        assert torch.equal(net.db[l][:L.LAYERS[l][1]], steps[l][1]), l


def test_training_is_deterministic(L):
    """Two trainings from the same seed and data give the same weights bit for
    bit (the weight gradients add their partial sums in a fixed order)."""
    data = L.training_set(count=3, shape=(24, 24, 130), eb_rel=1e-4, seed0=9300)
    nets = []
    for _ in range(2):
        net = L.ProposalNet(seed=8)
        L.train(net, data, epochs=2, lr=3e-3)
        nets.append(net)
    torch.cuda.synchronize()
    assert torch.equal(nets[0].flat, nets[1].flat)


LAYER_COUT = (32, 32, 32, 16)


# --------------------------------------------------------------- training
def test_training_reduces_loss_and_keeps_invariants(L):
    from paper_2601_01787_gb300 import api
    data = L.training_set(count=8, shape=(48, 48, 64), eb_rel=1e-4, seed0=9100)
    net = L.ProposalNet(seed=5)
    log = L.train(net, data, epochs=6, lr=3e-3)
    losses = [e[1] for e in log.epochs]
    assert losses[-1] < 0.85 * losses[0], losses
    # the exact loop finishes from the proposal: every invariant of the plain method holds
    fl = synth.peaks3d((48, 48, 64), seed=9200, eb_rel=1e-4)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    lr = L.correct_learned(f, fh, float(fl.xi), net)
    assert lr.result.status == api.OK
    v = api.verify(f, lr.result.out)
    assert v["codes_equal"] and v["wrong_labels"] == 0
    g = lr.result.out.cpu().numpy()
    lo = np.array([oracle.floor_bound(x, fl.xi) for x in fl.f.ravel()], np.float32).reshape(fl.f.shape)
    hi = np.array([oracle.ceil_bound(x, fl.xi) for x in fl.f.ravel()], np.float32).reshape(fl.f.shape)
    assert np.all(g >= lo) and np.all(g <= hi)


def test_trained_proposal_cuts_sweeps(L):
    """What the trained network gains: trained by its recipe (200 seeded 128^3
    Gaussian-peak triples, 12 epochs; about 45 s, cached with the build), its
    start takes the exact loop to a correct field in clearly fewer sweeps than
    the plain start on an unseen 256^3 field, and the result passes every check
    the plain result passes."""
    from paper_2601_01787_gb300 import api
    net, _ = L.default_net()
    fl = synth.peaks3d((256, 256, 256), seed=9002, eb_rel=1e-4)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    plain = api.correct(f, fh, float(fl.xi), edit_capacity=0)
    lr = L.correct_learned(f, fh, float(fl.xi), net, edit_capacity=0)
    assert plain.status == api.ERR_CAPACITY and lr.result.status == api.ERR_CAPACITY  # converged; no list asked
    assert not lr.fallback
    sp, sl = plain.stats["sweeps"], lr.from_g0.stats["sweeps"]
    assert sl <= 0.85 * sp, (sl, sp)
    assert lr.from_g0.stats["first_distorted"] < plain.stats["first_distorted"]
    v = api.verify(f, lr.result.out)
    assert v["codes_equal"] and v["wrong_labels"] == 0
    g = lr.result.out
    xi = float(fl.xi)
    assert bool(((g.double() - f.double()).abs() <= xi).all())


def test_learned_fallback_runs_the_plain_loop(L):
    """When the loop from the proposal ends without a correct field (here: at
    a one-sweep cap), the plain loop from fhat runs and its result is
    returned, with the fallback recorded."""
    from paper_2601_01787_gb300 import api
    fl = synth.peaks3d((24, 40, 130), seed=81, eb_rel=1e-4)
    f, fh = torch.from_numpy(fl.f).cuda(), torch.from_numpy(fl.fhat).cuda()
    net = L.ProposalNet(seed=2)
    lr = L.correct_learned(f, fh, float(fl.xi), net, max_sweeps=1)
    assert lr.from_g0.status == api.ERR_MAX_SWEEPS
    assert lr.fallback
    plain = api.correct(f, fh, float(fl.xi), max_sweeps=1)
    assert lr.result.status == plain.status
    assert torch.equal(lr.result.out.view(torch.int32), plain.out.view(torch.int32))
