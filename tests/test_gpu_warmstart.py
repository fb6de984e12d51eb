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
    torch.cuda.synchronize()
    ref_dx = C.bf16(C.conv3d_transpose(g, w) * (a > 0))
    dx = host(dX)
    assert np.all(np.abs(dx - ref_dx) <= 2.0 ** -7 * np.abs(ref_dx) + 1e-5 * np.abs(ref_dx).max())
    assert rel_l2(dx, ref_dx) <= 1e-3
    ref_dw = C.conv3d_wgrad(a, g)
    assert rel_l2(host(dW), ref_dw) <= 1e-5
    assert rel_l2(host(db), g.sum(axis=(0, 1, 2))) <= 1e-5


def test_network_loss_and_gradients_match_oracle():
    dims = (12, 10, 16)
    r = np.random.default_rng(3)
    net = WS.ConvNet(dims, device=DEV, seed=4)
    n = int(np.prod(dims))
    xm1 = torch.from_numpy(r.standard_normal(n)).to(DEV)
    xm2 = torch.from_numpy(r.standard_normal(n)).to(DEV)
    b = torch.from_numpy(r.standard_normal(n)).to(DEV)
    xt = xm1 + 0.1 * torch.from_numpy(r.standard_normal(n)).to(DEV)
    net.pack(xm1, xm2, b)
    net.forward()
    pk.warmstart_loss(n, net.out, xt, xm1, xm2, net.scales, net.grads[-1], net.loss, net.scratch)
    net.backward()
    torch.cuda.synchronize()
    params = [(host(w), host(bb)) for w, bb in zip(net.W16, net.b32)]
    x16 = host(net.acts[0])
    s = float(net.scales[1])
    target = ((xt - 2 * xm1 + xm2) / s).cpu().numpy().reshape(dims)
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
    again from the learned guess (with the residual judge).  Every solve reaches the same
    tolerance; the learned guess may not cost iterations on average."""
    res = WS.run_transient(k=64, steps=300, train_last=150, epochs=30)
    print({k: v for k, v in res.items() if not isinstance(v, list)})
    assert len(res["learned_iters_eval"]) == 150
    # the judge never lets a guess be worse than x_{t-1} by its residual
    assert res["learned_residual_ratio"] > 0 and res["extrap_residual_ratio"] > 0
    assert res["learned_mean_iters"] <= res["baseline_mean_iters"] + 0.5
    assert res["extrap_mean_iters"] <= res["baseline_mean_iters"] + 0.5
