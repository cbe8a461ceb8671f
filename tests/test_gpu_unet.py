"""The warm-start U-Net's CUDA kernels (through the C ABI) against the FP64 reference.

The library computes in BF16 (weights, activations and stored gradients rounded to
8 significant bits, relative step 2^-8) with FP32 accumulation and an FP32 output
layer; the reference computes
the same network in FP64 from the same BF16-rounded weights and input.  Eleven
layers of rounding give relative errors near 1e-2 in the output and a few 1e-2 in the
gradients; the checks allow 3e-2 (output, loss) and 6e-2 (each layer's gradient), far
below what a wrong tap, a swapped operand or a missing skip path produces (O(1)).
"""
import os

import numpy as np
import pytest

from oracle import unet_ref as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1603_08161_b300 import vd
    return vd, torch


def bf16(a):
    """Round float32 values to the nearest BF16 (ties to even), as float64."""
    a = np.ascontiguousarray(a, np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(dims, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    flat = U.he_params(seed + 100).astype(np.float32)
    x = rng.normal(size=(nx * ny * nz, 6)).astype(np.float32)
    t = (0.3 * rng.normal(size=(nx * ny * nz, 3))).astype(np.float32)
    return flat, x, t


# (12, 8, 20) has ragged 16-voxel row tiles; (96, 8, 8) has 96-, 48- and 24-voxel rows
# (the shared-memory staged convolution with 6, 3 and 2 tiles per row)
DIMS = [(16, 16, 16), (12, 8, 20), (96, 8, 8)]


@pytest.mark.parametrize("dims", DIMS)
def test_forward_matches_reference(env, dims):
    vd, torch = env
    nx, ny, nz = dims
    flat, x, _ = _case(dims, 1)
    net = vd.UNet(dims, seed=0)
    assert net.n_params == U.num_params()
    net.set_params(flat)
    np.testing.assert_array_equal(net.get_params(), flat)
    xin = torch.from_numpy(x).cuda()
    out = torch.zeros((nx * ny * nz, 3), device="cuda")
    net.forward(xin, out)
    ref, _ = U.forward(U.unpack(bf16(flat)), bf16(x).reshape(nz, ny, nx, 6))
    assert _rel(out.cpu().numpy().astype(np.float64), ref.reshape(-1, 3)) < 3e-2


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("lam", [0.0, 4.0])
def test_gradients_match_reference(env, dims, lam):
    vd, torch = env
    nx, ny, nz = dims
    flat, x, t = _case(dims, 2)
    x[np.random.default_rng(8).random(x.shape[0]) < 0.6, 3:] = 0.0  # nodes without data gradient
    net = vd.UNet(dims, seed=0)
    net.set_params(flat)
    loss = net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), 0.0, surface_weight=lam)
    g = net.get_grads()
    p = U.unpack(bf16(flat))
    xv = bf16(x).reshape(nz, ny, nx, 6)
    w = U.node_weights(xv, lam)
    out, acts = U.forward(p, xv)
    tt = t.reshape(nz, ny, nx, 3).astype(np.float64)
    assert abs(loss - U.loss(out, tt, w)) / U.loss(out, tt, w) < 3e-2
    gref = U.backward(p, acts, tt, w)
    gg = U.unpack(g)
    for name, _, _ in U.LAYERS:
        assert _rel(gg[name][0], gref[name][0]) < 6e-2, name
        assert _rel(gg[name][1], gref[name][1]) < 6e-2, name
    # lr = 0 leaves the parameters alone
    np.testing.assert_array_equal(net.get_params(), flat)


def test_adam_first_step(env):
    """Adam's first step from zero moments is p - lr g / (|g| + eps) (bias-corrected)."""
    vd, torch = env
    dims = (8, 8, 8)
    flat, x, t = _case(dims, 3)
    net = vd.UNet(dims, seed=0)
    net.set_params(flat)
    xin, tin = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    net.train_step(xin, tin, 0.0)
    g = net.get_grads().astype(np.float64)
    lr = 1e-3
    net.train_step(xin, tin, lr)
    dp = net.get_params().astype(np.float64) - flat
    exp = -lr * g / (np.abs(g) + 1e-8)
    m = np.abs(g) > 1e-5  # where the step is sign(g) to within the atomics' rounding
    assert m.sum() > 1000
    assert np.abs(dp[m] - exp[m]).max() < 2e-2 * lr


def test_training_lowers_the_loss(env):
    vd, torch = env
    dims = (8, 8, 8)
    _, x, t = _case(dims, 4)
    net = vd.UNet(dims, seed=7)
    xin, tin = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0 = net.train_step(xin, tin, 0.0)
    for _ in range(30):
        net.train_step(xin, tin, 3e-3)
    assert net.train_step(xin, tin, 0.0) < 0.7 * l0


def test_save_load_roundtrip(env, tmp_path):
    vd, _ = env
    a = vd.UNet((8, 8, 8), seed=11)
    b = vd.UNet((8, 8, 8), seed=12)
    assert not np.array_equal(a.get_params(), b.get_params())
    path = str(tmp_path / "w.bin")
    a.save(path)
    assert os.path.getsize(path) == 8 + 4 + 2 * 4 * 11 + 4 + 4 * U.num_params()
    b.load(path)
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    with open(path, "r+b") as f:  # a file for another layer table is refused
        f.seek(12)
        f.write(np.int32(7).tobytes())
    with pytest.raises(vd.VDError):
        b.load(path)


def test_bad_dims_rejected(env):
    vd, _ = env
    with pytest.raises(vd.VDError):
        vd.UNet((10, 8, 8))
