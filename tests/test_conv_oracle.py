"""Pins for the conv3d oracle of the learned warm start (CPU only): delta kernels, brute force
on a tiny grid, the adjoint identities of the transpose and weight-gradient operators,
central finite differences of the whole network's loss, and BF16 rounding against torch."""
import numpy as np
import pytest

from oracle import conv3d as C


def rng(seed=0):
    return np.random.default_rng(seed)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    v = rng(1).standard_normal(10_000) * 10.0 ** rng(2).integers(-20, 20, 10_000)
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(C.bf16(v), ref)
    assert C.bf16(1.0 + 2.0 ** -8) == 1.0                      # tie -> even
    assert C.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6      # tie -> even


def test_delta_kernels():
    x = rng(3).standard_normal((4, 5, 6, 16))
    w = np.zeros((27, 16, 16))
    w[13] = np.eye(16)  # centre tap
    np.testing.assert_array_equal(C.conv3d(x, w), x)
    w = np.zeros((27, 16, 16))
    w[C.TAPS.index((0, 0, 1))] = np.eye(16)
    out = C.conv3d(x, w)
    np.testing.assert_array_equal(out[:, :, :-1], x[:, :, 1:])
    assert not out[:, :, -1].any()


def test_conv_brute_force():
    r = rng(4)
    x = r.standard_normal((3, 4, 5, 2))
    w = r.standard_normal((27, 3, 2))
    b = r.standard_normal(3)
    D, H, W, _ = x.shape
    ref = np.zeros((D, H, W, 3))
    for z in range(D):
        for y in range(H):
            for xx in range(W):
                for co in range(3):
                    s = b[co]
                    for t, (dz, dy, dx) in enumerate(C.TAPS):
                        zz, yy, x2 = z + dz, y + dy, xx + dx
                        if 0 <= zz < D and 0 <= yy < H and 0 <= x2 < W:
                            for ci in range(2):
                                s += w[t, co, ci] * x[zz, yy, x2, ci]
                    ref[z, y, xx, co] = s
    np.testing.assert_allclose(C.conv3d(x, w, b), ref, rtol=1e-13, atol=1e-13)


def test_adjoint_identities():
    r = rng(5)
    x = r.standard_normal((5, 4, 6, 16))
    g = r.standard_normal((5, 4, 6, 16))
    w = r.standard_normal((27, 16, 16))
    w2 = r.standard_normal((27, 16, 16))
    lhs = np.sum(C.conv3d(x, w) * g)
    assert abs(lhs - np.sum(x * C.conv3d_transpose(g, w))) < 1e-10 * abs(lhs)
    # <conv(x, w2), g> is linear in w2 with gradient wgrad(x, g)
    lhs = np.sum(C.conv3d(x, w2) * g)
    assert abs(lhs - np.sum(w2 * C.conv3d_wgrad(x, g))) < 1e-10 * abs(lhs)


def small_params(seed=7, chans=(3, 16, 16, 16, 1)):
    r = rng(seed)
    params = []
    for cin, cout in zip(chans[:-1], chans[1:]):
        w = np.zeros((27, 16, 16))
        w[:, :cout, :cin] = r.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin))
        b = np.zeros(16)
        b[:cout] = 0.05 * r.standard_normal(cout)
        params.append((w, b))
    return params


def test_network_gradients_match_finite_differences():
    r = rng(8)
    params = small_params()
    x = np.zeros((5, 6, 4, 16))
    x[..., :3] = r.standard_normal((5, 6, 4, 3))
    target = r.standard_normal((5, 6, 4))
    loss, _, grads = C.loss_and_grads(params, x, target, rounding=False)
    h = 1e-6
    for layer, idx in [(0, (13, 2, 1)), (1, (4, 7, 9)), (2, (20, 0, 15)), (3, (13, 0, 5))]:
        pw = [(w.copy(), b.copy()) for w, b in params]
        pw[layer][0][idx] += h
        lp, _, _ = C.loss_and_grads(pw, x, target, rounding=False)
        pw[layer][0][idx] -= 2 * h
        lm, _, _ = C.loss_and_grads(pw, x, target, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[layer][0][idx]) <= 1e-6 * max(abs(fd), 1e-3), (layer, fd, grads[layer][0][idx])
        pb = [(w.copy(), b.copy()) for w, b in params]
        co = idx[1]
        pb[layer][1][co] += h
        lp, _, _ = C.loss_and_grads(pb, x, target, rounding=False)
        pb[layer][1][co] -= 2 * h
        lm, _, _ = C.loss_and_grads(pb, x, target, rounding=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grads[layer][1][co]) <= 1e-6 * max(abs(fd), 1e-3)


def test_adam_first_step_is_lr_times_sign():
    """With m = v = 0, the first Adam step moves every parameter by lr * g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = C.adam_step(np.ones(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p, 1.0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # a constant gradient keeps the bias-corrected step at lr * sign(g)
    for step in range(2, 6):
        p2, m, v = C.adam_step(p, g, m, v, step, lr=0.01)
        np.testing.assert_allclose(p - p2, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
        p = p2
