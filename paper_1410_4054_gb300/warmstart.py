"""Learned initial guess for a sequence of implicit time steps (a BF16 convolutional network).

A 4-layer 3x3x3 convolutional network (3 -> 16 -> 16 -> 16 -> 1 channels, ReLU between
layers, channel counts padded to 16) corrects the linear extrapolation of the solution
sequence.  Every numerical step runs in the library's CUDA kernels through the C ABI (BF16
tensor-core implicit-GEMM convolutions with FP32 accumulation, FP32 Adam); this module only
owns the buffers and sequences the calls.

Input: the residual r = b_t - A e of the extrapolation e = 2 x_{t-1} - x_{t-2}, as r/d (one
Jacobi step, d = diag(A)), r and d, each divided by its own rms s0, s1, s2 so that every BF16
channel is of order one.  The exact correction x_t - e = A^{-1} r is a function of r and of
the coefficients, which the translation-invariant network sees only through d and r, so the
network is told nothing it would have to memorise position by position.  Prediction
x_hat = e + s0 net(input), loss = mean((net - (x_t - e)/s0)^2).  The weights start at the
identity on channel 0 (relu(z) - relu(-z) = z through two hidden channels), i.e. at the Jacobi
step, and training moves them from there.
The network's error is rough (its BF16 operands round every voxel independently), and CG
removes rough error slowly on this operator while it removes the smooth error of the
extrapolation in a few iterations; so the learned start takes x_hat through RELAX_SWEEPS damped
Jacobi sweeps (pk_warmstart_relax), which damp error at the large eigenvalues of D^-1 A and
leave the smooth part to CG.  The same sweeps applied to the extrapolation are reported as the
ablation (they do not help it: its error is already smooth).
The solver is always run to the same tolerance: of the guess and x_{t-1}, the one with the
smaller residual ||b - A x0|| is the initial guess, so the plain warm start is both fallback and
yardstick.
The experiment also reports the extrapolation alone (network output taken as zero), so the
network's own contribution is visible, and the energy step: the network's correction d taken as
a search direction from e, x0 = e + gamma d with the gamma that minimises the A-norm of the
error along d (one more pass over A), so that the start is never worse than e in that norm.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import pk

CH = 16
LAYERS = ((3, 16), (16, 16), (16, 16), (16, 1))
# damped Jacobi sweeps applied to the learned guess before the residual check (see relax)
RELAX_OMEGA = 0.8
RELAX_SWEEPS = 3
# train on the error of the guess after those sweeps (pk_warmstart_loss_swept)
TRAIN_SWEPT = False


def initial_weights(seed=0, noise_std=1e-3):
    """FP32 weights [27][16][16] and biases [16] of the four layers at initialisation: an exact
    identity on channel 0 through hidden channels 0 (relu(z)) and 1 (relu(-z)) at the centre
    tap, He-scaled random weights into hidden channels 2..15, and output weights from channels
    2..15 of standard deviation noise_std."""
    rng = np.random.default_rng(seed)
    c = 13  # centre tap (dz, dy, dx) = (0, 0, 0)
    params = []
    for li, (cin, cout) in enumerate(LAYERS):
        w = np.zeros((27, CH, CH), dtype=np.float32)
        if li < len(LAYERS) - 1:
            w[:, 2:cout, :cin] = rng.standard_normal((27, cout - 2, cin)) * math.sqrt(2.0 / (27 * cin))
            if li == 0:
                w[c, 0, 0], w[c, 1, 0] = 1.0, -1.0
            else:
                w[c, 0, 0], w[c, 1, 1] = 1.0, 1.0
        else:
            w[:, 0, 2:cin] = rng.standard_normal((27, cin - 2)) * noise_std
            w[c, 0, 0], w[c, 0, 1] = 1.0, -1.0
        params.append((w, np.zeros(CH, dtype=np.float32)))
    return params


class ConvNet:
    """Parameters (FP32 master, BF16 copies, flipped BF16 copies, Adam moments) and buffers."""

    def __init__(self, dims, device="cuda", seed=0):
        import torch

        self.torch = torch
        self.dims = tuple(int(d) for d in dims)
        self.n = int(np.prod(self.dims))
        self.device = device
        self.W32, self.b32, self.W16, self.Wf16 = [], [], [], []
        self.mW, self.vW, self.mb, self.vb, self.dW, self.db = [], [], [], [], [], []
        for w, bias in initial_weights(seed):
            W32 = torch.from_numpy(w).to(device)
            self.W32.append(W32)
            self.b32.append(torch.from_numpy(bias).to(device))
            self.W16.append(W32.to(torch.bfloat16).contiguous())
            self.Wf16.append(torch.empty_like(self.W16[-1]))
            for lst, shape in ((self.mW, W32.shape), (self.vW, W32.shape), (self.dW, W32.shape),
                               (self.mb, (CH,)), (self.vb, (CH,)), (self.db, (CH,))):
                lst.append(torch.zeros(shape, dtype=torch.float32, device=device))
        vox = self.dims + (CH,)
        self.acts = [torch.zeros(vox, dtype=torch.bfloat16, device=device) for _ in range(len(LAYERS))]
        self.grads = [torch.zeros(vox, dtype=torch.bfloat16, device=device) for _ in range(len(LAYERS))]
        self.out = torch.zeros(self.dims, dtype=torch.float32, device=device)
        self.scales = torch.zeros(3, dtype=torch.float64, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.scratch = torch.zeros(pk.warmstart_scratch_doubles(), dtype=torch.float64, device=device)
        self.wscratch = torch.zeros(pk.conv3d_wgrad_scratch_floats(self.dims), dtype=torch.float32,
                                    device=device)
        self.work = None  # 3 n doubles for the swept loss, allocated on first use
        self.step = 0
        self.refresh_flipped()

    def refresh_flipped(self):
        for w16, wf in zip(self.W16, self.Wf16):
            pk.conv3d_flip(w16, wf)

    # -------------------------------------------------------------- checkpoints
    def state_dict(self) -> dict:
        """FP32 master weights and biases, Adam moments and step (host tensors); the BF16
        copies are derived from the masters on load."""
        cpu = lambda lst: [t.detach().cpu().clone() for t in lst]  # noqa: E731
        return {"dims": self.dims, "step": self.step, "W32": cpu(self.W32), "b32": cpu(self.b32),
                "mW": cpu(self.mW), "vW": cpu(self.vW), "mb": cpu(self.mb), "vb": cpu(self.vb)}

    def load_state_dict(self, d: dict):
        if tuple(d["dims"]) != self.dims:
            raise ValueError(f"checkpoint for grid {tuple(d['dims'])}, network built for {self.dims}")
        for key in ("W32", "b32", "mW", "vW", "mb", "vb"):
            for dst, src in zip(getattr(self, key), d[key]):
                dst.copy_(src.to(dst.device))
        for w32, w16 in zip(self.W32, self.W16):
            w16.copy_(w32.to(self.torch.bfloat16))
        self.step = int(d["step"])
        self.refresh_flipped()

    def save(self, path):
        self.torch.save(self.state_dict(), path)

    def load(self, path):
        self.load_state_dict(self.torch.load(path, map_location="cpu"))

    def pack(self, A, xm1, xm2, b):
        """acts[0] = packed network input; scales = (s0, s1, s2)."""
        pk.warmstart_input(A, xm1, xm2, b, self.acts[0], self.scales, self.scratch)

    def forward(self):
        """out = net(acts[0]) (FP32 channel 0); hidden activations kept for backward."""
        for li in range(len(LAYERS)):
            last = li == len(LAYERS) - 1
            pk.conv3d_fwd(self.acts[li], self.W16[li], self.b32[li],
                          self.out if last else self.acts[li + 1], self.dims,
                          relu=not last, out_f32=last)
        return self.out

    def backward(self):
        """grads[3] holds dL/d(out) (BF16, channel 0): weight/bias gradients into dW, db."""
        for li in range(len(LAYERS) - 1, -1, -1):
            pk.conv3d_wgrad(self.acts[li], self.grads[li], self.wscratch, self.dW[li], self.db[li],
                            self.dims)
            if li > 0:
                # dL/dz_{li-1} = conv(g, flipped W) masked by the ReLU derivative
                pk.conv3d_fwd(self.grads[li], self.Wf16[li], None, self.grads[li - 1], self.dims,
                              relu=False, out_f32=False, mask=self.acts[li])

    def adam(self, lr=1e-3):
        self.step += 1
        for li in range(len(LAYERS)):
            pk.adam_step(self.W32[li], self.dW[li], self.mW[li], self.vW[li], lr, self.step,
                         p_bf16=self.W16[li])
            pk.adam_step(self.b32[li], self.db[li], self.mb[li], self.vb[li], lr, self.step)
        self.refresh_flipped()

    def train_sample(self, A, xm1, xm2, b, xt, lr=1e-3, swept=None):
        """One Adam step on one sample.  swept = (omega, sweeps): the loss is taken on the guess
        after that many damped Jacobi sweeps (the form the solver receives), else on the guess
        itself."""
        self.pack(A, xm1, xm2, b)
        self.forward()
        if swept:
            if self.work is None:
                self.work = self.torch.zeros(3 * self.n, dtype=self.torch.float64, device=self.device)
            pk.warmstart_loss_swept(A, self.out, xt, xm1, xm2, self.scales, swept[0], swept[1],
                                    self.grads[-1], self.loss, self.work, self.scratch)
        else:
            pk.warmstart_loss(self.n, self.out, xt, xm1, xm2, self.scales, self.grads[-1], self.loss,
                              self.scratch)
        self.backward()
        self.adam(lr)

    def predict(self, A, xm1, xm2, b, xhat):
        self.pack(A, xm1, xm2, b)
        self.forward()
        pk.warmstart_apply(self.n, self.out, xm1, xm2, self.scales, xhat)

    def predict_energy(self, A, xm1, xm2, b, xhat, gamma):
        """x_hat = e + gamma s0 net with gamma minimising the A-norm error along the network's
        correction: never farther from x_t (A-norm) than the extrapolation e."""
        self.pack(A, xm1, xm2, b)
        self.forward()
        pk.warmstart_apply_energy(A, self.out, xm1, xm2, b, self.scales, xhat, gamma, self.scratch)


def relax(A, b, x, tmp, omega=RELAX_OMEGA, sweeps=RELAX_SWEEPS):
    """`sweeps` damped Jacobi sweeps on A x = b from x, alternating between x and tmp (a vector
    of the same size); returns the one that holds the result.  Each sweep damps the guess's
    error at the large eigenvalues of D^-1 A by |1 - omega lambda|: the rough error a BF16
    network leaves, which CG reduces slowly, while the smooth error that CG removes in a few
    iterations is left to CG."""
    src, dst = x, tmp
    for _ in range(sweeps):
        pk.warmstart_relax(A, b, src, omega, dst)
        src, dst = dst, src
    return src


def run_transient(k=64, steps=300, train_last=150, epochs=30, lr=1e-3, tol=1e-8, seed=0,
                  device="cuda", log=None, checkpoint=None, resume=False,
                  relax_omega=None, relax_sweeps=None, train_swept=None):
    """The transient experiment: solve the whole sequence with the x_{t-1} warm start, train on
    steps 2..train_last, then re-solve steps train_last+1..steps from (a) the linear
    extrapolation 2 x_{t-1} - x_{t-2} and (b) the learned guess, each measured against x_{t-1} by
    its residual.  Returns per-step iteration counts and times of all three, plus training
    statistics.

    checkpoint: a file for the solved sequence (x_t, b_t, plain warm-start iterations and
    times) and the network (weights, Adam state), written after training.  resume=True loads
    it, skips solving the sequence and continues training for `epochs` more epochs (0:
    evaluate the saved network as it is)."""
    import os

    import torch

    from . import workloads as W

    relax_omega = RELAX_OMEGA if relax_omega is None else float(relax_omega)
    relax_sweeps = RELAX_SWEEPS if relax_sweeps is None else int(relax_sweeps)
    train_swept = TRAIN_SWEPT if train_swept is None else bool(train_swept)
    swept = (relax_omega, relax_sweeps) if train_swept else None

    T = W.transient_heat(k, steps=steps, seed=seed)
    A = pk.CSRMatrix.from_workload(T.M)
    n = T.M.n
    dt = T.dt
    zeros = torch.zeros(n, dtype=torch.float64, device=device)
    net = ConvNet((k, k, k), device=device, seed=seed)
    if resume and checkpoint and os.path.exists(checkpoint):
        ck = torch.load(checkpoint, map_location="cpu")
        if (ck["k"], ck["steps"], ck["seed"]) != (k, steps, seed):
            raise ValueError("checkpoint of a different transient sequence")
        xs = [v.to(device) for v in ck["xs"]]
        bs = [None, None] + [v.to(device) for v in ck["bs"][2:]]
        base_iters, base_ms = list(ck["base_iters"]), list(ck["base_ms"])
        net.load_state_dict(ck["net"])
    else:
        xs = [zeros.clone(), zeros.clone()]  # x_{-1}, x_0
        bs = [None, None]
        base_iters, base_ms = [], []
        for t in range(1, steps + 1):
            f = torch.from_numpy(T.source(t)).to(device)
            b = xs[-1] + dt * f
            x = xs[-1].clone()
            info = pk.cg_solve(A, b, x, tol=tol, maxit=10_000)
            assert info["status"] == pk.PK_OK, info
            base_iters.append(info["iters"])
            base_ms.append(info["solve_ms"])
            xs.append(x)
            bs.append(b)
    # sample t: x_{t-1} = xs[t], x_{t-2} = xs[t-1], b_t = bs[t+1], target x_t = xs[t+1]
    train = list(range(2, train_last + 1))
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    first_loss = final_loss = None
    for ep in range(epochs):
        order = rng.permutation(train)
        acc = 0.0
        for t in order:
            net.train_sample(A, xs[t], xs[t - 1], bs[t + 1], xs[t + 1], lr=lr, swept=swept)
            if ep in (0, epochs - 1):
                acc += float(net.loss.item())
        if ep == 0:
            first_loss = acc / len(train)
        if ep == epochs - 1:
            final_loss = acc / len(train)
        if log:
            log(f"epoch {ep}")
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    if checkpoint:
        torch.save({"k": k, "steps": steps, "seed": seed, "xs": [v.cpu() for v in xs],
                    "bs": [None, None] + [v.cpu() for v in bs[2:]], "base_iters": base_iters,
                    "base_ms": base_ms, "net": net.state_dict()}, checkpoint)

    xhat = zeros.clone()
    xtmp = zeros.clone()
    r2 = torch.zeros(2, dtype=torch.float64, device=device)

    gamma = torch.zeros(1, dtype=torch.float64, device=device)
    gammas = []

    def evaluate(mode):
        iters, ms, chosen, ratio, kept = [], [], 0, [], []
        for t in range(train_last + 1, steps + 1):
            b = bs[t + 1]
            st = torch.cuda.Event(enable_timing=True)
            en = torch.cuda.Event(enable_timing=True)
            st.record()
            if mode.startswith("learned"):
                net.predict(A, xs[t], xs[t - 1], b, xhat)
            elif mode == "energy":
                net.predict_energy(A, xs[t], xs[t - 1], b, xhat, gamma)
            else:
                pk.warmstart_apply(n, None, xs[t], xs[t - 1], net.scales, xhat)
            guess = xhat
            if mode.endswith("relaxed"):
                guess = relax(A, b, xhat, xtmp, relax_omega, relax_sweeps)
            pk.residual_norm2(A, b, guess, r2[0:1])
            pk.residual_norm2(A, b, xs[t], r2[1:2])
            en.record()
            torch.cuda.synchronize()
            ra, rb = float(r2[0]), float(r2[1])
            ratio.append(np.sqrt(ra / rb) if rb > 0 else 1.0)
            pick = ra < rb
            chosen += int(pick)
            kept.append(np.sqrt(min(ra, rb) / rb) if rb > 0 else 1.0)
            x = (guess if pick else xs[t]).clone()
            info = pk.cg_solve(A, b, x, tol=tol, maxit=10_000)
            assert info["status"] == pk.PK_OK, info
            iters.append(info["iters"])
            ms.append(info["solve_ms"] + st.elapsed_time(en))
            if mode == "energy":
                gammas.append(float(gamma.item()))
        return iters, ms, chosen, float(np.mean(ratio)), float(max(kept))

    ex_iters, ex_ms, ex_chosen, ex_ratio, ex_kept = evaluate("extrap")
    ln_iters, ln_ms, ln_chosen, ln_ratio, ln_kept = evaluate("learned")
    en_iters, en_ms, en_chosen, en_ratio, en_kept = evaluate("energy")
    lr_iters, lr_ms, lr_chosen, lr_ratio, lr_kept = evaluate("learned_relaxed")
    er_iters, er_ms, er_chosen, er_ratio, er_kept = evaluate("extrap_relaxed")
    ev = slice(train_last, steps)
    return {
        "k": k, "n": n, "steps": steps, "train_samples": len(train), "epochs": epochs,
        "train_s": train_s, "first_epoch_loss": first_loss, "final_epoch_loss": final_loss,
        "baseline_iters_eval": base_iters[ev], "extrap_iters_eval": ex_iters,
        "learned_iters_eval": ln_iters,
        "baseline_mean_iters": float(np.mean(base_iters[ev])),
        "extrap_mean_iters": float(np.mean(ex_iters)),
        "learned_mean_iters": float(np.mean(ln_iters)),
        "baseline_mean_ms": float(np.mean(base_ms[ev])),
        "extrap_mean_ms": float(np.mean(ex_ms)),
        "learned_mean_ms": float(np.mean(ln_ms)),
        "extrap_residual_ratio": ex_ratio, "learned_residual_ratio": ln_ratio,
        "extrap_chosen_steps": ex_chosen, "learned_chosen_steps": ln_chosen,
        "extrap_max_kept_ratio": ex_kept, "learned_max_kept_ratio": ln_kept,
        "energy_iters_eval": en_iters, "energy_mean_iters": float(np.mean(en_iters)),
        "energy_mean_ms": float(np.mean(en_ms)), "energy_residual_ratio": en_ratio,
        "energy_chosen_steps": en_chosen, "energy_max_kept_ratio": en_kept,
        "energy_gamma_mean": float(np.mean(gammas)), "energy_gamma_min": float(np.min(gammas)),
        "energy_gamma_max": float(np.max(gammas)),
        "relax_omega": relax_omega, "relax_sweeps": relax_sweeps, "train_swept": train_swept,
        "learned_relaxed_iters_eval": lr_iters, "learned_relaxed_mean_iters": float(np.mean(lr_iters)),
        "learned_relaxed_mean_ms": float(np.mean(lr_ms)), "learned_relaxed_residual_ratio": lr_ratio,
        "learned_relaxed_chosen_steps": lr_chosen, "learned_relaxed_max_kept_ratio": lr_kept,
        "extrap_relaxed_iters_eval": er_iters, "extrap_relaxed_mean_iters": float(np.mean(er_iters)),
        "extrap_relaxed_mean_ms": float(np.mean(er_ms)), "extrap_relaxed_residual_ratio": er_ratio,
        "extrap_relaxed_chosen_steps": er_chosen, "extrap_relaxed_max_kept_ratio": er_kept,
    }
