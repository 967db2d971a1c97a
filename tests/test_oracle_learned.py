"""Pins of the learned-proposal oracle (oracle/learned.py) on the CPU.

The conv is pinned to a brute-force loop and to scipy's correlate; its
backward operators to the adjoint identities that define them; the whole
backward pass to central finite differences of the forward loss; the BF16
rounding to torch's own conversion.
"""
import numpy as np
import pytest
import torch

from oracle import learned as OL


def _rand(shape, seed, scale=1.0):
    return np.random.default_rng(seed).standard_normal(shape) * scale


def test_bf16_matches_torch_conversion():
    a = np.concatenate([_rand(5000, 1, 3.0), np.array([0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e-38, 1e30])])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(OL.bf16(a), ref)


def test_conv3d_brute_force():
    nz, ny, nx, ci, co = 3, 4, 5, 3, 2
    x = _rand((nz, ny, nx, ci), 2)
    w = _rand((27, co, ci), 3)
    y = OL.conv3d(x, w)
    ref = np.zeros((nz, ny, nx, co))
    for z in range(nz):
        for yy in range(ny):
            for xx in range(nx):
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            a, b, c = z + dz, yy + dy, xx + dx
                            if 0 <= a < nz and 0 <= b < ny and 0 <= c < nx:
                                o = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
                                ref[z, yy, xx] += w[o] @ x[a, b, c]
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_conv3d_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    x = _rand((6, 7, 9, 2), 4)
    w = _rand((27, 3, 2), 5)
    y = OL.conv3d(x, w)
    for co in range(3):
        acc = np.zeros(x.shape[:3])
        for ci in range(2):
            k = w[:, co, ci].reshape(3, 3, 3)  # [dz][dy][dx]
            acc += signal.correlate(x[..., ci], k, mode="same", method="direct")
        np.testing.assert_allclose(y[..., co], acc, rtol=1e-12, atol=1e-12)


def test_transpose_is_adjoint():
    x = _rand((4, 5, 6, 3), 6)
    dy = _rand((4, 5, 6, 2), 7)
    w = _rand((27, 2, 3), 8)
    lhs = np.sum(OL.conv3d(x, w) * dy)
    rhs = np.sum(x * OL.conv3d_transpose(dy, w))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_wgrad_is_gradient_of_bilinear_form():
    x = _rand((4, 5, 6, 3), 9)
    dy = _rand((4, 5, 6, 2), 10)
    w = _rand((27, 2, 3), 11)
    lhs = np.sum(OL.conv3d(x, w) * dy)
    rhs = np.sum(OL.conv3d_wgrad(x, dy) * w)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def _tiny_params(seed, chans=(3, 4, 4, 4, 1)):
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((27, chans[l + 1], chans[l])) * 0.3, rng.standard_normal(chans[l + 1]) * 0.1)
            for l in range(4)]


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(12)
    feat = rng.standard_normal((3, 4, 5, 3))
    k = rng.integers(0, 5, (3, 4, 5))
    params = _tiny_params(13, chans=(3, 4, 4, 4, 5))
    scale = 0.37

    def loss(ps):
        # -log softmax(z)_k written through scipy's logsumexp
        from scipy.special import logsumexp
        z = OL.forward(feat, ps, bf16_points=False)["z"]
        return scale * np.sum(logsumexp(z, axis=-1) - np.take_along_axis(z, k[..., None], -1)[..., 0])

    grads, _ = OL.backward(OL.forward(feat, params, bf16_points=False), k, params, scale, bf16_points=False)
    h = 1e-6
    for l in range(4):
        w, b = params[l]
        for idx in [tuple(rng.integers(0, s) for s in w.shape) for _ in range(6)]:
            wp = [(pw.copy(), pb.copy()) for pw, pb in params]
            wm = [(pw.copy(), pb.copy()) for pw, pb in params]
            wp[l][0][idx] += h
            wm[l][0][idx] -= h
            fd = (loss(wp) - loss(wm)) / (2 * h)
            assert abs(fd - grads[l][0][idx]) <= 1e-6 + 1e-5 * abs(fd), (l, idx, fd, grads[l][0][idx])
        for j in range(len(b)):
            bp = [(pw.copy(), pb.copy()) for pw, pb in params]
            bm = [(pw.copy(), pb.copy()) for pw, pb in params]
            bp[l][1][j] += h
            bm[l][1][j] -= h
            fd = (loss(bp) - loss(bm)) / (2 * h)
            assert abs(fd - grads[l][1][j]) <= 1e-6 + 1e-5 * abs(fd), (l, j, fd, grads[l][1][j])


def test_cross_entropy_special_cases():
    z = np.array([[0.0, 0.0, 0.0, 0.0], [1000.0, 0.0, -5.0, 2.0], [3.0, 3.0, -1e4, 0.0]])
    k = np.array([2, 0, 1])
    ce = OL.cross_entropy(z, k)
    assert ce[0] == pytest.approx(np.log(4.0))          # uniform logits
    assert ce[1] == pytest.approx(0.0, abs=1e-12)        # a dominant right logit
    assert ce[2] == pytest.approx(np.log(2.0 + np.exp(-3.0)))
    assert np.allclose(OL.softmax(z).sum(axis=-1), 1.0)


def test_edit_count_counts_the_halving_chain():
    import oracle
    f, xi = np.float32(0.3), np.float32(1e-4)
    L = oracle.floor_bound(f, xi)
    fhat = np.float32(f + np.float32(0.7e-4))
    g = fhat
    for k in range(0, 12):
        assert OL.edit_count(fhat, g, L, oracle.edit) == k
        g, _ = oracle.edit(g, L)
    # near 0.3 (ulp 3e-8) the chain reaches L after 13 halvings of 1.7e-4
    assert OL.edit_count(fhat, L, L, oracle.edit) == 13
    # near 1e-3 (ulp 1.2e-10) L is about 20 halvings away: the count is capped
    f2 = np.float32(1e-3)
    L2 = oracle.floor_bound(f2, xi)
    assert OL.edit_count(np.float32(f2 + np.float32(0.7e-4)), L2, L2, oracle.edit) == OL.CLASSES - 1


def test_forward_single_voxel_closed_form():
    # one voxel, 1 channel everywhere: the conv keeps only the centre tap
    params = []
    for l in range(4):
        w = np.zeros((27, 1, 1))
        w[13, 0, 0] = [2.0, 0.5, 3.0, -1.0][l]
        params.append((w, np.array([0.25 * (l + 1)])))
    acts = OL.forward(np.array([[[[0.75]]]]), params, bf16_points=False)
    x = 0.75
    for l in range(3):
        x = max(params[l][0][13, 0, 0] * x + params[l][1][0], 0.0)
    zz = -1.0 * x + 1.0
    assert acts["z"][0, 0, 0, 0] == pytest.approx(zz)
    assert acts["p"][0, 0, 0, 0] == pytest.approx(1.0)  # one class
