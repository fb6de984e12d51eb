"""CPU oracle of the learned warm start's 3D convolutional network (numpy FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring): imported by the tests and nowhere on
the product path; it shares no code with the CUDA kernels.

Network: four 3x3x3 convolutions with zero padding 1 on a channels-last grid (D, H, W, C),
channels padded to 16 (3 -> 16 -> 16 -> 16 -> 1), ReLU after the first three.  Weights are
indexed w[tap][co][ci] with tap = 9 (dz+1) + 3 (dy+1) + (dx+1).  Every operand the GPU stores
in BF16 (input, weights, activations, output gradient, hidden-layer gradients) is rounded to
BF16 here at the same point; all arithmetic is FP64, so the oracle differs from the GPU only
by the GPU's FP32 accumulation order (and, rarely, a BF16 rounding that flips because of it).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16(a) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (rounded.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def conv3d(x: np.ndarray, w: np.ndarray, bias=None) -> np.ndarray:
    """out[z,y,x,co] = bias[co] + sum_tap sum_ci w[tap,co,ci] x[z+dz, y+dy, x+dx, ci] (zero outside)."""
    D, H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((D, H, W, w.shape[1]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        sl = xp[1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :]
        out += np.tensordot(sl, w[t], axes=([3], [1]))
    if bias is not None:
        out += bias
    return out


def conv3d_transpose(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3d in its input: dx[z,y,x,ci] = sum_tap sum_co w[tap,co,ci] g[z-dz, y-dy, x-dx, co]."""
    D, H, W, _ = g.shape
    gp = np.pad(g, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((D, H, W, w.shape[2]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        sl = gp[1 - dz:1 - dz + D, 1 - dy:1 - dy + H, 1 - dx:1 - dx + W, :]
        out += np.tensordot(sl, w[t], axes=([3], [0]))
    return out


def conv3d_wgrad(a: np.ndarray, g: np.ndarray) -> np.ndarray:
    """dW[tap,co,ci] = sum_v g[v,co] a[v + offset(tap), ci] (zero outside)."""
    D, H, W, _ = a.shape
    ap = np.pad(a, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dw = np.zeros((27, g.shape[3], a.shape[3]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        sl = ap[1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :]
        dw[t] = np.tensordot(g, sl, axes=([0, 1, 2], [0, 1, 2]))
    return dw


def forward(params, x16: np.ndarray, rounding: bool = True):
    """Activations a0..a3 (BF16-rounded after ReLU) and the FP64 output channel 0."""
    rnd = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    acts = [rnd(x16)]
    for layer, (w, b) in enumerate(params):
        z = conv3d(acts[-1], rnd(w), b)
        if layer < len(params) - 1:
            acts.append(rnd(np.maximum(z, 0.0)))
        else:
            out = z[..., 0]
    return acts, out


def loss_and_grads(params, x16: np.ndarray, target: np.ndarray, rounding: bool = True):
    """MSE loss mean((out - target)^2) and its gradients dW, db for every layer (chain rule,
    with the GPU's BF16 rounding of the propagated gradients)."""
    rnd = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    acts, out = forward(params, x16, rounding)
    nvox = out.size
    diff = out - target
    loss = float(np.mean(diff * diff))
    g = np.zeros(out.shape + (params[-1][0].shape[1],))
    g[..., 0] = 2.0 * diff / nvox
    g = rnd(g)
    grads = [None] * len(params)
    for layer in range(len(params) - 1, -1, -1):
        w, _ = params[layer]
        a_in = acts[layer]
        dw = conv3d_wgrad(a_in, g)
        db = g.sum(axis=(0, 1, 2))
        grads[layer] = (dw, db)
        if layer > 0:
            ga = conv3d_transpose(g, rnd(w))
            g = rnd(ga * (a_in > 0))
    return loss, out, grads


def warmstart_input(row_ptr, col, val, xm1, xm2, b):
    """Network input of the learned initial guess before BF16 rounding, and its scales.

    The linear extrapolation e = 2 x_{t-1} - x_{t-2} of the time step A x_t = b leaves the
    residual r = b - A e; with d = diag(A) (1 where a row has no nonzero diagonal entry) the
    channels are (r/d)/s0, r/s1, d/s2, zero elsewhere, s0..s2 the rms of r/d, r, d (1 where
    zero).  Returns (X[n][16], (s0, s1, s2))."""
    n = len(row_ptr) - 1
    e = 2.0 * np.asarray(xm1, dtype=np.float64) - np.asarray(xm2, dtype=np.float64)
    r = np.array(b, dtype=np.float64)
    d = np.zeros(n)
    for i in range(n):
        for j in range(row_ptr[i], row_ptr[i + 1]):
            r[i] -= val[j] * e[col[j]]
            if col[j] == i:
                d[i] = val[j]
    d[d == 0.0] = 1.0
    z = r / d
    scales = []
    for v in (z, r, d):
        s = float(np.sqrt(np.mean(v * v)))
        scales.append(s if s > 0 else 1.0)
    X = np.zeros((n, 16))
    X[:, 0] = z / scales[0]
    X[:, 1] = r / scales[1]
    X[:, 2] = d / scales[2]
    return X, tuple(scales)


def warmstart_target(xt, xm1, xm2, s0):
    """What the network is trained to output: (x_t - (2 x_{t-1} - x_{t-2})) / s0."""
    return (np.asarray(xt) - (2.0 * np.asarray(xm1) - np.asarray(xm2))) / s0


def warmstart_energy_step(row_ptr, col, val, xm1, xm2, b, out, s0):
    """The energy step along the network's correction: e = 2 x_{t-1} - x_{t-2}, r = b - A e,
    d = s0 out, gamma = <r, d> / <d, A d> (0 if <d, A d> <= 0), x_hat = e + gamma d.  For SPD A,
    gamma minimises ||x_t - e - gamma d||_A over gamma, since A (x_t - e) = r.  Returns
    (x_hat, gamma); rows summed left to right in FP64."""
    n = len(row_ptr) - 1
    e = 2.0 * np.asarray(xm1, dtype=np.float64) - np.asarray(xm2, dtype=np.float64)
    d = float(s0) * np.asarray(out, dtype=np.float64)
    r = np.array(b, dtype=np.float64)
    ad = np.zeros(n)
    for i in range(n):
        for j in range(row_ptr[i], row_ptr[i + 1]):
            r[i] -= val[j] * e[col[j]]
            ad[i] += val[j] * d[col[j]]
    num, den = float(np.dot(r, d)), float(np.dot(d, ad))
    gamma = num / den if den > 0 and np.isfinite(num / den) else 0.0
    return e + gamma * d, gamma


def warmstart_relax(row_ptr, col, val, b, x, omega):
    """One damped Jacobi sweep on A x = b from the guess x: for every row i,
    x'_i = x_i + omega (b_i - sum_j a_ij x_j) / d_i with d_i = a_ii (1 where the row has no
    nonzero diagonal entry); each row's products summed left to right in FP64.  The error
    x' - x* is (I - omega D^-1 A)(x - x*), which damps error at the large eigenvalues of D^-1 A
    (rough error on a diagonally dominant operator)."""
    n = len(row_ptr) - 1
    x = np.asarray(x, dtype=np.float64)
    out = np.empty(n)
    for i in range(n):
        s, d = 0.0, 0.0
        for j in range(row_ptr[i], row_ptr[i + 1]):
            s += val[j] * x[col[j]]
            if col[j] == i:
                d = val[j]
        if d == 0.0:
            d = 1.0
        out[i] = x[i] + omega * ((b[i] - s) / d)
    return out


def warmstart_swept_loss(row_ptr, col, val, out, xt, xm1, xm2, s0, omega, sweeps):
    """Loss of the learned guess in the form CG receives it -- after `sweeps` damped Jacobi
    sweeps -- and its gradient with respect to the network output, for a symmetric A.

    The guess x_hat = e + s0 out (e = 2 x_{t-1} - x_{t-2}) has the error s0 delta with
    delta = out - (x_t - e) / s0.  A sweep x <- x + omega D^-1 (b - A x) with b = A x_t maps an
    error e to P e = e - omega D^-1 A e (b drops out).  loss = mean((P^s delta)^2); its
    gradient is (2/n) (P^T)^s P^s delta, where P^T g = g - omega A (D^-1 g) because A is
    symmetric.  d_i = a_ii (1 where the row has no nonzero diagonal entry); rows summed left
    to right in FP64.  Returns (loss, gradient)."""
    n = len(row_ptr) - 1
    d = np.ones(n)
    for i in range(n):
        for j in range(row_ptr[i], row_ptr[i + 1]):
            if col[j] == i and val[j] != 0.0:
                d[i] = val[j]
    e = np.asarray(out, dtype=np.float64) - (np.asarray(xt) - 2.0 * np.asarray(xm1) + np.asarray(xm2)) / s0
    for _ in range(sweeps):
        nxt = np.empty(n)
        for i in range(n):
            acc = 0.0
            for j in range(row_ptr[i], row_ptr[i + 1]):
                acc += val[j] * e[col[j]]
            nxt[i] = e[i] + omega * ((0.0 - acc) / d[i])
        e = nxt
    loss = float(np.mean(e * e))
    g = e
    for _ in range(sweeps):
        nxt = np.empty(n)
        for i in range(n):
            acc = 0.0
            for j in range(row_ptr[i], row_ptr[i + 1]):
                acc += val[j] * (g[col[j]] / d[col[j]])
            nxt[i] = g[i] - omega * acc
        g = nxt
    return loss, 2.0 * g / n


def adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, ICLR 2015, Algorithm 1) in FP64; returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
