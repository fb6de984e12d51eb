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


def _csr(dense):
    rp, ci, va = [0], [], []
    for row in dense:
        nz = np.nonzero(row)[0]
        ci.extend(nz.tolist())
        va.extend(row[nz].tolist())
        rp.append(len(ci))
    return np.array(rp), np.array(ci), np.array(va)


def test_warmstart_input_diagonal_matrix_gives_exact_correction():
    """For a diagonal A one Jacobi step is exact: e + s0 X[:,0] = A^{-1} b, and the target
    equals X[:,0]."""
    r = rng(9)
    d = 1.0 + r.random(40)
    xm1, xm2, b = r.standard_normal((3, 40))
    X, (s0, s1, s2) = C.warmstart_input(*_csr(np.diag(d)), xm1, xm2, b)
    e = 2.0 * xm1 - xm2
    np.testing.assert_allclose(e + s0 * X[:, 0], b / d, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(C.warmstart_target(b / d, xm1, xm2, s0), X[:, 0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(s2 * X[:, 2], d, rtol=1e-15)
    assert abs(np.sqrt(np.mean(X[:, 0] ** 2)) - 1.0) < 1e-14
    assert not X[:, 3:].any()


def test_warmstart_input_brute_force():
    r = rng(10)
    n = 7
    dense = r.standard_normal((n, n)) * (r.random((n, n)) < 0.5)
    dense[3, 3] = 0.0                       # no diagonal entry: d = 1
    np.fill_diagonal(dense[:3, :3], 2.0 + r.random(3))
    xm1, xm2, b = r.standard_normal((3, n))
    X, (s0, s1, s2) = C.warmstart_input(*_csr(dense), xm1, xm2, b)
    for i in range(n):
        res = b[i] - sum(dense[i, j] * (2 * xm1[j] - xm2[j]) for j in range(n))
        di = dense[i, i] if dense[i, i] != 0 else 1.0
        assert abs(X[i, 1] * s1 - res) <= 1e-13 * max(1.0, abs(res))
        assert abs(X[i, 0] * s0 - res / di) <= 1e-13 * max(1.0, abs(res / di))
        assert X[i, 2] * s2 == pytest.approx(di, rel=1e-15)


def test_warmstart_input_exact_extrapolation_is_zero_residual():
    """If x_t lies on the line through x_{t-2}, x_{t-1} the residual is zero (integer data, so
    exactly), the residual channels are zero and their scales fall back to 1."""
    r = rng(11)
    dense = np.diag(r.integers(2, 5, 6).astype(float)) + np.eye(6, k=1)
    xm2, dx = r.integers(-4, 5, (2, 6)).astype(float)
    xm1 = xm2 + dx
    b = dense @ (xm1 + dx)
    X, (s0, s1, s2) = C.warmstart_input(*_csr(dense), xm1, xm2, b)
    assert (s0, s1) == (1.0, 1.0)
    assert not X[:, :2].any()
    np.testing.assert_allclose(X[:, 2] * s2, np.diag(dense), rtol=1e-15)


def test_warmstart_energy_step_minimises_the_energy_error():
    """On a random SPD system: the oracle's gamma is the minimiser of the A-norm error
    E(g) = (x* - e - g d)^T A (x* - e - g d), found here from three samples of the parabola
    (dense products, no residual formula); E(gamma) <= E(0) and <= E(1); the exact correction
    direction gives gamma = 1 and x_hat = x*; a zero correction gives gamma = 0."""
    r = rng(12)
    n = 9
    m = r.standard_normal((n, n))
    dense = m @ m.T + n * np.eye(n)
    dense[np.abs(dense) < 0.3] = 0.0
    dense = (dense + dense.T) / 2 + n * np.eye(n)
    xs, xm1, xm2 = r.standard_normal((3, n))
    b = dense @ xs
    out = r.standard_normal(n).astype(np.float32)
    s0 = 0.7
    xh, gamma = C.warmstart_energy_step(*_csr(dense), xm1, xm2, b, out, s0)
    e, d = 2 * xm1 - xm2, s0 * out.astype(np.float64)

    def E(g):
        err = xs - e - g * d
        return float(err @ dense @ err)

    e0, e1, e2 = E(0.0), E(1.0), E(2.0)
    g_star = (e0 - e1) / (e0 - 2 * e1 + e2) + 0.5   # vertex of the parabola through g = 0, 1, 2
    assert gamma == pytest.approx(g_star, rel=1e-9)
    assert E(gamma) <= min(e0, e1) + 1e-12 * e0
    np.testing.assert_allclose(xh, e + gamma * d, rtol=0, atol=1e-14)
    # the exact correction (as FP32 output of a unit scale) is taken whole
    exact = (xs - e).astype(np.float32)
    xh2, g2 = C.warmstart_energy_step(*_csr(dense), xm1, xm2, dense @ (e + exact.astype(np.float64)), exact, 1.0)
    assert g2 == pytest.approx(1.0, rel=1e-12)
    _, g3 = C.warmstart_energy_step(*_csr(dense), xm1, xm2, b, np.zeros(n, np.float32), s0)
    assert g3 == 0.0


def _relax_pins(relax):
    """The pins of one damped Jacobi sweep, applied to an implementation `relax(row_ptr, col,
    val, b, x, omega)`: on a diagonal matrix one sweep with omega = 1 is the exact solution
    b / diag(A); the solution of a dense LU solve is a fixed point; the error after one sweep
    equals (I - omega D^-1 A) times the error before it, with D^-1 A formed from the dense
    matrix; repeated sweeps on a diagonally dominant matrix converge to the LU solution; a row
    without a diagonal entry divides by 1."""
    r = rng(21)
    n = 11
    diag = r.uniform(1.0, 3.0, n)
    b = r.standard_normal(n)
    x0 = r.standard_normal(n)
    np.testing.assert_allclose(relax(*_csr(np.diag(diag)), b, x0, 1.0), b / diag, rtol=1e-15, atol=0)
    m = r.standard_normal((n, n))
    m[np.abs(m) < 0.8] = 0.0
    dense = m + np.diag(np.abs(m).sum(axis=1) * 1.5 + 1.0)   # strictly diagonally dominant
    xs = np.linalg.solve(dense, b)
    np.testing.assert_allclose(relax(*_csr(dense), b, xs, 0.8), xs, rtol=0, atol=1e-13)
    prop = np.eye(n) - 0.8 * (dense / np.diag(dense)[:, None])
    np.testing.assert_allclose(relax(*_csr(dense), b, x0, 0.8) - xs, prop @ (x0 - xs), rtol=0, atol=1e-13)
    x = x0.copy()
    for _ in range(200):
        x = relax(*_csr(dense), b, x, 0.8)
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-12)
    # rows 0 and 1 without a diagonal entry: d = 1
    nodiag = dense.copy()
    nodiag[0, 0] = nodiag[1, 1] = 0.0
    got = relax(*_csr(nodiag), b, x0, 0.5)
    assert got[0] == pytest.approx(x0[0] + 0.5 * (b[0] - nodiag[0] @ x0), rel=1e-13)


def test_warmstart_relax_pins():
    _relax_pins(C.warmstart_relax)


def _relax_mutant(kind):
    """A copy of the oracle's sweep with one plausible mistake planted."""
    def relax(row_ptr, col, val, b, x, omega):
        n = len(row_ptr) - 1
        x = np.asarray(x, dtype=np.float64)
        out = np.empty(n)
        for i in range(n):
            s, d, rowsum = 0.0, 0.0, 0.0
            for j in range(row_ptr[i], row_ptr[i + 1]):
                s += val[j] * x[col[j]]
                rowsum += abs(val[j])
                if col[j] == i:
                    d = val[j]
            if d == 0.0:
                d = 1.0
            if kind == "sign":              # the residual with the wrong sign
                out[i] = x[i] + omega * ((s - b[i]) / d)
            elif kind == "omega_on_x":      # the damping applied to the old iterate
                out[i] = omega * x[i] + (b[i] - s) / d
            elif kind == "row_sum":         # the row's absolute sum instead of its diagonal
                out[i] = x[i] + omega * ((b[i] - s) / rowsum)
            elif kind == "no_division":     # the residual not scaled by the diagonal
                out[i] = x[i] + omega * (b[i] - s)
            elif kind == "updated_gather":  # Gauss-Seidel: rows read values already updated
                x = x.copy()
                x[i] = x[i] + omega * ((b[i] - s) / d)
                out[i] = x[i]
        return out
    return relax


@pytest.mark.parametrize("kind", ["sign", "omega_on_x", "row_sum", "no_division", "updated_gather"])
def test_warmstart_relax_pins_catch_mutants(kind):
    """Each planted mistake in the sweep fails at least one of its pins."""
    with pytest.raises(AssertionError):
        _relax_pins(_relax_mutant(kind))


def _sym_system(seed, n=10):
    r = rng(seed)
    m = r.standard_normal((n, n))
    m[np.abs(m) < 0.9] = 0.0
    m = (m + m.T) / 2
    dense = m + np.diag(np.abs(m).sum(axis=1) * 1.5 + 1.0)   # symmetric, diagonally dominant
    return dense, r


def test_warmstart_swept_loss_pins():
    _swept_pins(C.warmstart_swept_loss)


def _swept_pins(swept_loss):
    """The loss after Jacobi sweeps: with no sweep it is the plain MSE of the output against
    the target and its gradient 2 (out - y) / n; with sweeps it equals mean((P^s delta)^2) for
    P = I - omega D^-1 A formed as a dense matrix, and its gradient equals the dense
    (2/n) (P^s)^T P^s delta (which pins the transposition); central finite differences of the
    loss agree with the gradient."""
    dense, r = _sym_system(31)
    n = dense.shape[0]
    rp, ci, va = _csr(dense)
    out = r.standard_normal(n)
    xt, xm1, xm2 = r.standard_normal((3, n))
    s0, omega = 0.7, 0.8
    y = (xt - 2 * xm1 + xm2) / s0
    loss0, g0 = swept_loss(rp, ci, va, out, xt, xm1, xm2, s0, omega, 0)
    assert loss0 == pytest.approx(float(np.mean((out - y) ** 2)), rel=1e-14)
    np.testing.assert_allclose(g0, 2 * (out - y) / n, rtol=1e-14, atol=0)
    P = np.eye(n) - omega * (dense / np.diag(dense)[:, None])
    for sweeps in (1, 3):
        Ps = np.linalg.matrix_power(P, sweeps)
        loss, g = swept_loss(rp, ci, va, out, xt, xm1, xm2, s0, omega, sweeps)
        e = Ps @ (out - y)
        assert loss == pytest.approx(float(np.mean(e * e)), rel=1e-12)
        np.testing.assert_allclose(g, 2.0 / n * (Ps.T @ e), rtol=0, atol=1e-13 * np.abs(g).max())
        h = 1e-6
        for k in (0, 4, n - 1):
            up, dn = out.copy(), out.copy()
            up[k] += h
            dn[k] -= h
            lu, _ = swept_loss(rp, ci, va, up, xt, xm1, xm2, s0, omega, sweeps)
            ld, _ = swept_loss(rp, ci, va, dn, xt, xm1, xm2, s0, omega, sweeps)
            assert (lu - ld) / (2 * h) == pytest.approx(g[k], rel=1e-6, abs=1e-10)


def _swept_mutant(kind):
    """A copy of the oracle's swept loss with one plausible mistake planted."""
    def swept(row_ptr, col, val, out, xt, xm1, xm2, s0, omega, sweeps):
        n = len(row_ptr) - 1
        d = np.ones(n)
        for i in range(n):
            for j in range(row_ptr[i], row_ptr[i + 1]):
                if col[j] == i and val[j] != 0.0:
                    d[i] = val[j]
        e = np.asarray(out, dtype=np.float64) - (np.asarray(xt) - 2.0 * np.asarray(xm1) + np.asarray(xm2)) / s0

        def prop(v):
            return np.array([v[i] - omega * sum(val[j] * v[col[j]] for j in range(row_ptr[i], row_ptr[i + 1])) / d[i]
                             for i in range(n)])

        def prop_t(g):
            return np.array([g[i] - omega * sum(val[j] * g[col[j]] / d[col[j]]
                                                for j in range(row_ptr[i], row_ptr[i + 1])) for i in range(n)])

        for _ in range(sweeps):
            e = prop(e)
        loss = float(np.mean(e * e))
        g = e
        for _ in range(sweeps):
            g = prop(g) if kind == "no_transpose" else prop_t(g)
        if kind == "scale":        # the 2/n factor dropped
            return loss, g
        if kind == "one_fewer":    # one transposed sweep short in the backward pass
            g = e
            for _ in range(max(sweeps - 1, 0)):
                g = prop_t(g)
        if kind == "sign_target":  # the target's extrapolation sign flipped
            e2 = np.asarray(out, dtype=np.float64) - (np.asarray(xt) + 2.0 * np.asarray(xm1) - np.asarray(xm2)) / s0
            return float(np.mean(e2 * e2)), 2.0 * e2 / n
        return loss, 2.0 * g / n
    return swept


@pytest.mark.parametrize("kind", ["no_transpose", "scale", "one_fewer", "sign_target"])
def test_warmstart_swept_loss_pins_catch_mutants(kind):
    """Each planted mistake in the swept loss fails at least one of its pins."""
    with pytest.raises(AssertionError):
        _swept_pins(_swept_mutant(kind))
