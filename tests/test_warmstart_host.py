"""Host-side logic of the learned warm start (CPU only): the network's initial weights."""
import numpy as np

from oracle import conv3d as C
from paper_1410_4054_gb300 import warmstart as WS


def test_identity_initialisation_is_one_jacobi_step():
    """With the output noise switched off, the initial network maps channel 0 to itself exactly
    (relu(z) - relu(-z)), so the first prediction is one Jacobi step from the extrapolation."""
    dims = (6, 5, 9)
    params = [(w.astype(np.float64), b.astype(np.float64))
              for w, b in WS.initial_weights(seed=3, noise_std=0.0)]
    x = np.zeros(dims + (16,))
    x[..., :3] = C.bf16(np.random.default_rng(7).standard_normal(dims + (3,)))
    _, out = C.forward(params, x)
    np.testing.assert_array_equal(out, x[..., 0])


def test_initial_weights_respect_channel_padding():
    """Padded channels carry no weight: layer 0 reads 3 inputs, the last layer writes 1 output."""
    params = WS.initial_weights(seed=1)
    assert not params[0][0][:, :, 3:].any()
    assert not params[-1][0][:, 1:, :].any()
    for w, b in params:
        assert w.dtype == np.float32 and w.shape == (27, 16, 16) and not b.any()
