"""Pins of the FP64 U-Net reference (oracle/unet_ref.py) to things other than itself:
scipy's correlation, closed forms of pooling and up-sampling, the layer table, and
central finite differences of the loss."""
import numpy as np
import pytest
import scipy.ndimage

from oracle import unet_ref as U


def test_param_count_matches_layer_table():
    # sum Cin*Cout = 13,200 over the 11 layers, sum Cout = 323
    assert U.num_params() == 27 * 13200 + 323 == 356723


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(5, 6, 7, 3))
    w = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=2)
    y = U.conv(x, w, b)
    for co in range(2):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            k = w[:, ci, co].reshape(3, 3, 3)  # [dz+1, dy+1, dx+1]
            ref += scipy.ndimage.correlate(x[..., ci], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(y[..., co], ref, rtol=1e-12, atol=1e-12)


def test_pool_and_up_closed_forms():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 6, 8, 2))
    p = U.pool(x)
    assert p.shape == (2, 3, 4, 2)
    assert np.isclose(p[1, 2, 3, 1], x[2:4, 4:6, 6:8, 1].mean())
    # pooling undoes up-sampling; the up-sampled copy is constant on each block
    np.testing.assert_allclose(U.pool(U.up(p)), p, rtol=0, atol=1e-15)
    assert np.all(U.up(p)[2:4, 4:6, 6:8, 0] == p[1, 2, 3, 0])
    # adjoints: <pool x, y> = <x, pool^T y>, <up x, y> = <x, up^T y>
    y = rng.normal(size=p.shape)
    assert np.isclose((p * y).sum(), (x * U.pool_backward(y)).sum())
    z = rng.normal(size=x.shape)
    assert np.isclose((U.up(p) * z).sum(), (p * U.up_backward(z)).sum())


@pytest.fixture(scope="module")
def tiny():
    rng = np.random.default_rng(3)
    flat = U.he_params(5)
    x = rng.normal(size=(4, 4, 4, 6))
    x[rng.random((4, 4, 4)) < 0.5, 3:] = 0.0  # nodes without data gradient
    t = rng.normal(size=(4, 4, 4, 3)) * 0.3
    return flat, x, t


def test_node_weights():
    x = np.zeros((1, 1, 3, 6))
    x[0, 0, 1, 4] = 2.0
    x[0, 0, 2, :3] = 1.0
    np.testing.assert_array_equal(U.node_weights(x, 4.0)[0, 0, :, 0], [1.0, 5.0, 1.0])


def _loss(flat, x, t, w=1.0):
    out, _ = U.forward(U.unpack(flat), x)
    return U.loss(out, t, w)


@pytest.mark.parametrize("lam", [0.0, 4.0])
def test_gradients_match_finite_differences(tiny, lam):
    flat, x, t = tiny
    w = U.node_weights(x, lam)
    p = U.unpack(flat)
    out, acts = U.forward(p, x)
    g = U.pack(U.backward(p, acts, t, w))
    rng = np.random.default_rng(4)
    # a few entries of every layer's weights and biases
    idx, k = [], 0
    for _, ci, co in U.LAYERS:
        nw = 27 * ci * co
        idx += list(k + rng.choice(nw, 6, replace=False)) + list(k + nw + rng.choice(co, 2, replace=False))
        k += nw + co
    eps = 1e-6
    for i in idx:
        fp = flat.copy()
        fp[i] += eps
        fm = flat.copy()
        fm[i] -= eps
        fd = (_loss(fp, x, t, w) - _loss(fm, x, t, w)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_every_layer_receives_gradient(tiny):
    flat, x, t = tiny
    p = U.unpack(flat)
    out, acts = U.forward(p, x)
    g = U.backward(p, acts, t)
    for name, _, _ in U.LAYERS:
        assert np.abs(g[name][0]).sum() > 0, name
