"""GPU parity of the learned warm start's kernels against the conv3d oracle (FP64 on the same
BF16-rounded operands), and the transient experiment with its fallback."""
import numpy as np
import pytest

from oracle import conv3d as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1410_4054_gb300 import pk  # noqa: E402
from paper_1410_4054_gb300 import warmstart as WS  # noqa: E402

DEV = "cuda:0"


def bf16_dev(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(DEV).to(torch.bfloat16).contiguous()


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SHAPES = [(8, 8, 8), (5, 6, 70), (3, 4, 129), (64, 64, 64)]


@pytest.mark.parametrize("dims", SHAPES)
def test_conv_forward_matches_oracle(dims):
    r = np.random.default_rng(1)
    x = C.bf16(r.standard_normal(dims + (16,)))
    w = C.bf16(r.standard_normal((27, 16, 16)) * 0.1)
    b = r.standard_normal(16).astype(np.float32).astype(np.float64)
    ref = C.conv3d(x, w, b)
    X, Wt = bf16_dev(x), bf16_dev(w)
    bias = torch.from_numpy(b.astype(np.float32)).to(DEV)
    Y = torch.zeros(dims + (16,), dtype=torch.bfloat16, device=DEV)
    pk.conv3d_fwd(X, Wt, bias, Y, dims, relu=True)
    Yf = torch.zeros(dims, dtype=torch.float32, device=DEV)
    pk.conv3d_fwd(X, Wt, bias, Yf, dims, relu=False, out_f32=True)
    pk.conv3d_check()
    torch.cuda.synchronize()
    # FP32 output: only the accumulation order differs from the FP64 oracle
    assert rel_l2(host(Yf), ref[..., 0]) <= 1e-6
    # BF16 output after ReLU: equal up to one BF16 rounding step where FP32 accumulation flips it
    y, yr = host(Y), C.bf16(np.maximum(ref, 0.0))
    # (near zero, FP32 accumulation may move a value across 0 before the ReLU: absolute term)
    assert np.all(np.abs(y - yr) <= 2.0 ** -7 * np.abs(yr) + 1e-5 * np.abs(yr).max())
    assert rel_l2(y, yr) <= 1e-3


@pytest.mark.parametrize("dims", [(8, 8, 8), (5, 6, 70), (16, 16, 16)])
def test_conv_backward_data_and_weights_match_oracle(dims):
    r = np.random.default_rng(2)
    a = C.bf16(np.maximum(r.standard_normal(dims + (16,)), 0.0))  # a ReLU output: many zeros
    g = C.bf16(r.standard_normal(dims + (16,)))
    w = C.bf16(r.standard_normal((27, 16, 16)) * 0.1)
    A, G, Wt = bf16_dev(a), bf16_dev(g), bf16_dev(w)
    Wf = torch.empty_like(Wt)
    pk.conv3d_flip(Wt, Wf)
    dX = torch.zeros(dims + (16,), dtype=torch.bfloat16, device=DEV)
    pk.conv3d_fwd(G, Wf, None, dX, dims, relu=False, mask=A)
    scratch = torch.zeros(pk.conv3d_wgrad_scratch_floats(dims), dtype=torch.float32, device=DEV)
    dW = torch.zeros((27, 16, 16), dtype=torch.float32, device=DEV)
    db = torch.zeros(16, dtype=torch.float32, device=DEV)
    pk.conv3d_wgrad(A, G, scratch, dW, db, dims)
    pk.conv3d_check()
    torch.cuda.synchronize()
    ref_dx = C.bf16(C.conv3d_transpose(g, w) * (a > 0))
    dx = host(dX)
    assert np.all(np.abs(dx - ref_dx) <= 2.0 ** -7 * np.abs(ref_dx) + 1e-5 * np.abs(ref_dx).max())
    assert rel_l2(dx, ref_dx) <= 1e-3
    ref_dw = C.conv3d_wgrad(a, g)
    assert rel_l2(host(dW), ref_dw) <= 1e-5
    assert rel_l2(host(db), g.sum(axis=(0, 1, 2))) <= 1e-5


def test_warmstart_input_matches_oracle():
    from paper_1410_4054_gb300 import workloads as W

    T = W.transient_heat(16, steps=3, seed=2)
    A = pk.CSRMatrix.from_workload(T.M)
    r = np.random.default_rng(6)
    xm1, xm2, b = r.standard_normal((3, T.M.n))
    net = WS.ConvNet((16, 16, 16), device=DEV, seed=1)
    net.pack(A, *(torch.from_numpy(v).to(DEV) for v in (xm1, xm2, b)))
    torch.cuda.synchronize()
    X, scales = C.warmstart_input(T.M.row_ptr, T.M.col, T.M.val, xm1, xm2, b)
    np.testing.assert_allclose(net.scales.cpu().numpy(), scales, rtol=1e-12)
    got, ref = host(net.acts[0]).reshape(-1, 16), C.bf16(X)
    # FP64 rows summed in another order can move a value across a BF16 rounding boundary
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref))
    assert np.mean(got != ref) < 1e-3


def test_warmstart_energy_step_matches_oracle():
    """pk_warmstart_apply_energy against the oracle on the transient operator: gamma to 1e-12
    relative, x_hat to 1e-13 relative (same FP32 correction, FP64 sums in another order)."""
    from paper_1410_4054_gb300 import workloads as W

    T = W.transient_heat(16, steps=3, seed=2)
    A = pk.CSRMatrix.from_workload(T.M)
    r = np.random.default_rng(7)
    xm1, xm2 = r.standard_normal((2, T.M.n))
    b = T.M.matvec(xm1 + 0.01 * r.standard_normal(T.M.n))
    out = (0.01 * r.standard_normal(T.M.n)).astype(np.float32)
    scales = torch.tensor([0.3, 1.0, 1.0], dtype=torch.float64, device=DEV)
    xh = torch.zeros(T.M.n, dtype=torch.float64, device=DEV)
    gamma = torch.zeros(1, dtype=torch.float64, device=DEV)
    scratch = torch.zeros(pk.warmstart_scratch_doubles(), dtype=torch.float64, device=DEV)
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(DEV)  # noqa: E731
    for _ in range(2):  # twice in a row: the scratch counter is reset by each call
        pk.warmstart_apply_energy(A, dv(out), dv(xm1), dv(xm2), dv(b), scales, xh, gamma, scratch)
        torch.cuda.synchronize()
        ref, g = C.warmstart_energy_step(T.M.row_ptr, T.M.col, T.M.val, xm1, xm2, b, out, 0.3)
        assert gamma.item() == pytest.approx(g, rel=1e-12)
        assert rel_l2(xh.cpu().numpy(), ref) <= 1e-13


def test_warmstart_relax_matches_oracle():
    """pk_warmstart_relax (one damped Jacobi sweep) against the oracle, element by element: on
    the transient operator and on a random matrix whose rows mostly lack a diagonal entry
    (divisor 1 there), two sweeps in a row alternating the buffers as the learned start does;
    xout == x and omega outside (0, 2) are rejected."""
    from paper_1410_4054_gb300 import workloads as W

    r = np.random.default_rng(5)
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(DEV)  # noqa: E731
    for M in (W.transient_heat(16, steps=3, seed=2).M, W.random_uniform(3001, 28, seed=1)):
        A = pk.CSRMatrix.from_workload(M)
        absA = W.CSR(M.n, M.row_ptr, M.col, np.abs(M.val))
        diag = np.ones(M.n)
        for i in range(M.n):
            for j in range(M.row_ptr[i], M.row_ptr[i + 1]):
                if M.col[j] == i and M.val[j] != 0.0:
                    diag[i] = M.val[j]
        b = r.standard_normal(M.n)
        x = r.standard_normal(M.n)
        xd, yd, bd = dv(x), torch.zeros(M.n, dtype=torch.float64, device=DEV), dv(b)
        for omega in (0.8, 0.5):
            pk.warmstart_relax(A, bd, xd, omega, yd)
            torch.cuda.synchronize()
            ref = C.warmstart_relax(M.row_ptr, M.col, M.val, b, x, omega)
            bound = 1e-13 * (np.abs(x) + omega * (np.abs(b) + absA.matvec(np.abs(x))) / np.abs(diag))
            assert np.all(np.abs(yd.cpu().numpy() - ref) <= bound)
            xd, yd, x = yd, xd, ref   # the next sweep starts from this one's result
        with pytest.raises(RuntimeError, match="xout must not be x"):
            pk.warmstart_relax(A, bd, xd, 0.8, xd)
        with pytest.raises(RuntimeError, match="omega"):
            pk.warmstart_relax(A, bd, xd, 2.0, yd)
        A.close()


def test_warmstart_swept_loss_matches_oracle():
    """pk_warmstart_loss_swept (the loss after Jacobi sweeps and its output gradient) against
    the oracle on the transient operator (symmetric): the loss to 1e-12 relative and the BF16
    gradient within one BF16 step of the oracle's rounded gradient, zeros in the other
    channels; 0 and 3 sweeps, two calls in a row; bad omega and sweeps rejected."""
    from paper_1410_4054_gb300 import workloads as W

    T = W.transient_heat(16, steps=3, seed=2)
    M = T.M
    A = pk.CSRMatrix.from_workload(M)
    r = np.random.default_rng(11)
    n = M.n
    dv = lambda v: torch.from_numpy(np.ascontiguousarray(v)).to(DEV)  # noqa: E731
    xt, xm1, xm2 = r.standard_normal((3, n))
    out = (0.3 * r.standard_normal(n)).astype(np.float32)
    scales = torch.tensor([0.4, 1.0, 1.0], dtype=torch.float64, device=DEV)
    G = torch.zeros((n, 16), dtype=torch.bfloat16, device=DEV)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    work = torch.zeros(3 * n, dtype=torch.float64, device=DEV)
    scratch = torch.zeros(pk.warmstart_scratch_doubles(), dtype=torch.float64, device=DEV)
    for sweeps in (3, 0, 3):
        pk.warmstart_loss_swept(A, dv(out), dv(xt), dv(xm1), dv(xm2), scales, 0.8, sweeps, G, loss,
                                work, scratch)
        torch.cuda.synchronize()
        ref_loss, ref_g = C.warmstart_swept_loss(M.row_ptr, M.col, M.val, out, xt, xm1, xm2, 0.4, 0.8,
                                                 sweeps)
        assert loss.item() == pytest.approx(ref_loss, rel=1e-12)
        got = host(G)
        ref = C.bf16(ref_g.astype(np.float32))
        step = np.abs(ref) * 2.0 ** -7 + 1e-30
        assert np.all(np.abs(got[:, 0] - ref) <= step)
        assert np.all(got[:, 1:] == 0.0)
    with pytest.raises(RuntimeError, match="omega"):
        pk.warmstart_loss_swept(A, dv(out), dv(xt), dv(xm1), dv(xm2), scales, 0.0, 3, G, loss, work, scratch)
    with pytest.raises(RuntimeError, match="sweeps"):
        pk.warmstart_loss_swept(A, dv(out), dv(xt), dv(xm1), dv(xm2), scales, 0.8, 9, G, loss, work, scratch)
    A.close()


def _grid_operator(dims, r):
    """A symmetric 7-point operator on the grid: 1D second differences summed over the three
    axes with random positive weights, plus 1 on the diagonal (an implicit time step)."""
    import scipy.sparse as sp

    from paper_1410_4054_gb300 import workloads as W

    eyes = [sp.identity(d, format="csr") for d in dims]
    M = sp.identity(int(np.prod(dims)), format="csr")
    for ax, d in enumerate(dims):
        T = sp.diags([-np.ones(d - 1), 2 * np.ones(d), -np.ones(d - 1)], [-1, 0, 1], format="csr")
        mats = [T if k == ax else eyes[k] for k in range(3)]
        M = M + (0.5 + r.random()) * sp.kron(sp.kron(mats[0], mats[1]), mats[2], format="csr")
    M = M.tocsr()
    M.sort_indices()
    return W.CSR(M.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32),
                 M.data.astype(np.float64), "grid7")


def test_network_loss_and_gradients_match_oracle():
    dims = (12, 10, 16)
    r = np.random.default_rng(3)
    net = WS.ConvNet(dims, device=DEV, seed=4)
    n = int(np.prod(dims))
    M = _grid_operator(dims, r)
    A = pk.CSRMatrix.from_workload(M)
    xm1 = torch.from_numpy(r.standard_normal(n)).to(DEV)
    xm2 = torch.from_numpy(r.standard_normal(n)).to(DEV)
    b = torch.from_numpy(r.standard_normal(n)).to(DEV)
    xt = xm1 + 0.1 * torch.from_numpy(r.standard_normal(n)).to(DEV)
    net.pack(A, xm1, xm2, b)
    net.forward()
    pk.warmstart_loss(n, net.out, xt, xm1, xm2, net.scales, net.grads[-1], net.loss, net.scratch)
    net.backward()
    pk.conv3d_check()
    torch.cuda.synchronize()
    params = [(host(w), host(bb)) for w, bb in zip(net.W16, net.b32)]
    x16 = host(net.acts[0])
    s = float(net.scales[0])
    target = C.warmstart_target(*(v.cpu().numpy() for v in (xt, xm1, xm2)), s).reshape(dims)
    loss, out, grads = C.loss_and_grads(params, x16, target)
    assert abs(float(net.loss.item()) - loss) <= 1e-5 * loss
    # whole network: hidden BF16 activations can round differently (FP32 vs FP64 sums)
    assert rel_l2(host(net.out), out) <= 1e-3
    # layer by layer on the GPU's own BF16 operands: accumulation order only
    for li, (w, bb) in enumerate(params):
        z = C.conv3d(host(net.acts[li]), w, bb)
        if li < 3:
            ref = C.bf16(np.maximum(z, 0.0))
            got = host(net.acts[li + 1])
            assert np.all(np.abs(got - ref) <= 2.0 ** -7 * np.abs(ref) + 1e-5 * np.abs(ref).max())
        else:
            assert rel_l2(host(net.out), z[..., 0]) <= 1e-6
    # whole chain: each of the three BF16 gradient stages can round differently (<= 1e-3 each)
    for li, (dw, db) in enumerate(grads):
        assert rel_l2(host(net.dW[li]), dw) <= 3e-3, li
        assert rel_l2(host(net.db[li]), db) <= 3e-3, li
    # stage by stage on the GPU's own BF16 operands: accumulation order only
    for li in range(4):
        a_in, g = host(net.acts[li]), host(net.grads[li])
        assert rel_l2(host(net.dW[li]), C.conv3d_wgrad(a_in, g)) <= 1e-5, li
        assert rel_l2(host(net.db[li]), g.sum(axis=(0, 1, 2))) <= 1e-5, li
        if li > 0:
            ref = C.bf16(C.conv3d_transpose(g, params[li][0]) * (a_in > 0))
            got = host(net.grads[li - 1])
            assert np.all(np.abs(got - ref) <= 2.0 ** -7 * np.abs(ref) + 1e-5 * np.abs(ref).max())


def test_adam_matches_oracle():
    r = np.random.default_rng(5)
    p0 = r.standard_normal(1000).astype(np.float32)
    p = torch.from_numpy(p0.copy()).to(DEV)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    p16 = torch.zeros(1000, dtype=torch.bfloat16, device=DEV)
    pr, mr, vr = p0.astype(np.float64), np.zeros(1000), np.zeros(1000)
    for step in range(1, 4):
        g = r.standard_normal(1000).astype(np.float32)
        pk.adam_step(p, torch.from_numpy(g).to(DEV), m, v, 1e-3, step, p_bf16=p16)
        pr, mr, vr = C.adam_step(pr, g.astype(np.float64), mr, vr, step)
    torch.cuda.synchronize()
    np.testing.assert_allclose(p.cpu().numpy(), pr, rtol=0, atol=2e-6)
    np.testing.assert_array_equal(host(p16), C.bf16(p.cpu().numpy()))


def test_transient_learned_warm_start():
    """Steps 1-150 train the network on the solver's own solutions; steps 151-300 are solved
    again from the learned guess, kept only where its residual is not larger than that of
    x_{t-1}.  Every solve reaches the same tolerance.  The test asserts that training lowers
    the loss, that no solve starts from a guess with a larger residual than x_{t-1}, that no
    learned form costs iterations on average, and that the learned start with its Jacobi
    sweeps needs at least one iteration fewer than the linear extrapolation, the network's own
    input, whether or not the extrapolation gets the same sweeps (measured on GB300: 3.39
    against 5.99 and 6.00)."""
    res = WS.run_transient(k=64, steps=300, train_last=150, epochs=30)
    print({k: v for k, v in res.items() if not isinstance(v, list)})
    assert len(res["learned_iters_eval"]) == 150
    assert res["final_epoch_loss"] < 0.5 * res["first_epoch_loss"]
    assert res["learned_max_kept_ratio"] <= 1.0 and res["extrap_max_kept_ratio"] <= 1.0
    assert res["learned_mean_iters"] <= res["baseline_mean_iters"]
    assert res["extrap_mean_iters"] <= res["baseline_mean_iters"]
    assert res["energy_max_kept_ratio"] <= 1.0
    assert res["energy_mean_iters"] <= res["baseline_mean_iters"]
    assert res["learned_relaxed_max_kept_ratio"] <= 1.0 and res["extrap_relaxed_max_kept_ratio"] <= 1.0
    assert res["learned_relaxed_mean_iters"] <= res["baseline_mean_iters"]
    # the learned start (network + Jacobi sweeps) needs fewer iterations than the extrapolation
    # that is the network's input, with or without the same sweeps
    assert res["learned_relaxed_mean_iters"] < res["extrap_mean_iters"] - 1.0
    assert res["learned_relaxed_mean_iters"] < res["extrap_relaxed_mean_iters"] - 1.0


def test_checkpoint_round_trip_and_resume(tmp_path):
    """A network restored from a checkpoint predicts bitwise like the saved one and takes the
    same Adam steps (moments and step count restored); run_transient resumes from its
    checkpoint without re-solving the sequence."""
    from paper_1410_4054_gb300 import workloads as W

    T = W.transient_heat(16, steps=4, seed=3)
    A = pk.CSRMatrix.from_workload(T.M)
    r = np.random.default_rng(8)
    xm1, xm2, b, xt = (torch.from_numpy(v).to(DEV) for v in r.standard_normal((4, T.M.n)))
    net = WS.ConvNet((16, 16, 16), device=DEV, seed=2)
    for _ in range(3):
        net.train_sample(A, xm1, xm2, b, xt)
    path = tmp_path / "net.pt"
    net.save(path)
    other = WS.ConvNet((16, 16, 16), device=DEV, seed=9)
    other.load(path)
    y1, y2 = torch.empty_like(xt), torch.empty_like(xt)
    net.predict(A, xm1, xm2, b, y1)
    other.predict(A, xm1, xm2, b, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    net.train_sample(A, xm1, xm2, b, xt)
    other.train_sample(A, xm1, xm2, b, xt)
    torch.cuda.synchronize()
    assert other.step == net.step
    assert all(torch.equal(a, c) for a, c in zip(net.W32, other.W32))
    with pytest.raises(ValueError, match="grid"):
        WS.ConvNet((8, 8, 8), device=DEV).load(path)
    ck = tmp_path / "transient.pt"
    first = WS.run_transient(k=16, steps=12, train_last=6, epochs=2, checkpoint=str(ck))
    again = WS.run_transient(k=16, steps=12, train_last=6, epochs=0, checkpoint=str(ck), resume=True)
    assert again["baseline_iters_eval"] == first["baseline_iters_eval"]
    assert again["learned_iters_eval"] == first["learned_iters_eval"]
