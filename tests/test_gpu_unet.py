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


# ------------------------------------------------------------------ layer by layer, element by element
#
# Each kernel of the forward and backward pass is checked on its own: the FP64
# reference is applied to the GPU's own BF16 input tensors of that step (read back with
# vd_unet_get_tensor), so no rounding error propagates from earlier layers, and every
# element must lie in the interval that the arithmetic allows:
#   * products of two BF16 values are exact in FP32; a sum of n of them accumulated in
#     FP32 in any order, rounding or truncating, is within n 2^-23 sum|terms| of the
#     exact sum (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 4.2,
#     with the unit roundoff doubled for truncation);
#   * ReLU and rounding to BF16 (round to nearest even) are both non-decreasing, so a
#     stored value computed from an FP32 sum within [y - e, y + e] of the exact y lies
#     in [rne(relu(y - e)), rne(relu(y + e))];
#   * a ReLU mask multiplies by exactly 0 or 1, taken from the stored activation;
#   * the weights enter as BF16, the biases as the FP32 master values (added in the
#     FP32 epilogue).
# A wrong tap, a dropped edge voxel, a swapped operand or a missing skip path moves an
# element by a whole term, far outside these intervals; the intervals are a few 1e-4
# of sum|terms| wide (one BF16 step, 2^-8 relative, where rounding decides).

U_ACC = 2.0 ** -23


def rne_bf16(v):
    """FP64 values rounded to BF16 (8 significant bits), ties to even, exactly."""
    m, e = np.frexp(np.asarray(v, np.float64))
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def _rounded_interval(y, T, n, relu=False):
    e = n * U_ACC * T
    lo, hi = y - e, y + e
    if relu:
        lo, hi = np.maximum(lo, 0.0), np.maximum(hi, 0.0)
    return rne_bf16(lo), rne_bf16(hi)


def _assert_within(what, g, lo, hi):
    bad = (g < lo) | (g > hi)
    if bad.any():
        k = np.argmax(np.where(bad, np.maximum(lo - g, g - hi), -1))
        raise AssertionError(f"{what}: {int(bad.sum())} of {g.size} elements outside their rounding interval; "
                             f"worst: gpu {g.flat[k]:.6e} not in [{lo.flat[k]:.6e}, {hi.flat[k]:.6e}]")


def _conv_fwd_check(what, x, w, b, y_gpu, relu):
    y = U.conv(x, w, b)
    T = U.conv(np.abs(x), np.abs(w), np.abs(b))
    lo, hi = _rounded_interval(y, T, 27 * x.shape[-1] + 2, relu)
    _assert_within(what, y_gpu, lo, hi)


def _dgrad_interval(x_shape, w, gy):
    """Interval of the stored BF16 input gradient of a convolution (before any mask)."""
    zeros = np.zeros(x_shape)
    gx, _, _ = U.conv_backward(zeros, w, gy)
    T, _, _ = U.conv_backward(zeros, np.abs(w), np.abs(gy))
    return _rounded_interval(gx, T, 27 * gy.shape[-1] + 2)


def _wgrad_check(what, x, gy, gw_gpu, gb_gpu):
    _, gw, gb = U.conv_backward(x, np.zeros((27, x.shape[-1], gy.shape[-1])), gy)
    _, Tw, Tb = U.conv_backward(np.abs(x), np.zeros((27, x.shape[-1], gy.shape[-1])), np.abs(gy))
    n = int(np.prod(gy.shape[:3])) + 64
    assert np.all(np.abs(gw_gpu - gw) <= n * U_ACC * Tw), f"{what} weight gradient"
    assert np.all(np.abs(gb_gpu - gb) <= n * U_ACC * Tb), f"{what} bias gradient"


@pytest.mark.parametrize("dims", DIMS)
def test_every_kernel_element_by_element(env, dims):
    vd, torch = env
    nx, ny, nz = dims
    n = nx * ny * nz
    flat, x, t = _case(dims, 5)
    x[np.random.default_rng(9).random(n) < 0.5, 3:] = 0.0
    lam = 4.0
    net = vd.UNet(dims, seed=0)
    net.set_params(flat)
    # the parameters as the kernels use them: BF16 weights, FP32 (master) biases
    p = {name: (bf16(w), b) for name, (w, b) in U.unpack(flat.astype(np.float64)).items()}
    xin, tin = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    outf = torch.zeros((n, 3), device="cuda")
    net.forward(xin, outf)
    outf = outf.cpu().numpy().astype(np.float64).reshape(nz, ny, nx, 3)
    net.train_step(xin, tin, 0.0, surface_weight=lam)
    T = {k: net.tensor(k).astype(np.float64) for k in vd.UNET_TENSORS}
    G = U.unpack(net.get_grads().astype(np.float64))

    # ---- forward pass
    np.testing.assert_array_equal(T["x"][..., :6], bf16(x).reshape(nz, ny, nx, 6))
    assert not T["x"][..., 6:].any()
    chain = [("a1", T["x"][..., :6], "e1a"), ("b1", T["e1a"], "e1"), ("a2", T["p1"], "e2a"), ("b2", T["e2a"], "e2"),
             ("a3", T["p2"], "e3a"), ("b3", T["e3a"], "e3"), ("c2", T["cat2"], "d2a"), ("d2", T["d2a"], "d2"),
             ("c1", T["cat1"], "d1a"), ("d1", T["d1a"], "d1")]
    for name, xin_l, out in chain:
        _conv_fwd_check(f"forward {name}", xin_l, *p[name], T[out][..., :p[name][0].shape[2]], relu=True)
    y = U.conv(T["d1"], *p["head"])
    Th = U.conv(np.abs(T["d1"]), np.abs(p["head"][0]), np.abs(p["head"][1]))
    assert np.all(np.abs(outf - y) <= (27 * 16 + 2) * U_ACC * Th), "forward head (FP32 output)"
    for src, dst in (("e1", "p1"), ("e2", "p2")):
        s8 = U.pool(T[src])
        lo, hi = _rounded_interval(s8, U.pool(np.abs(T[src])), 9)
        _assert_within(f"pool {src}", T[dst], lo, hi)
    np.testing.assert_array_equal(T["cat2"][..., :64], U.up(T["e3"]))
    np.testing.assert_array_equal(T["cat2"][..., 64:], T["e2"])
    np.testing.assert_array_equal(T["cat1"][..., :32], U.up(T["d2"]))
    np.testing.assert_array_equal(T["cat1"][..., 32:], T["e1"])

    # ---- loss gradient: 2 w (out - t) / (3 n) from the FP32 output, four FP32 roundings
    w = U.node_weights(bf16(x).reshape(nz, ny, nx, 6), lam)
    g64 = 2.0 * w * (outf - t.reshape(nz, ny, nx, 3).astype(np.float64)) / (3.0 * n)
    lo, hi = rne_bf16(g64 - 8 * 2.0 ** -24 * np.abs(g64)), rne_bf16(g64 + 8 * 2.0 ** -24 * np.abs(g64))
    _assert_within("loss gradient", T["gout"][..., :3], lo, hi)
    assert not T["gout"][..., 3:].any()

    # ---- backward pass: input gradients (masked by the stored activations' ReLU)
    def dgrad(name, gy, x_shape, got, mask=None, what=None):
        lo, hi = _dgrad_interval(x_shape, p[name][0], gy)
        if got is not None:
            m = 1.0 if mask is None else (mask > 0)
            _assert_within(what or f"dgrad {name}", got, lo * m, hi * m)
        return lo, hi

    dgrad("head", T["gout"][..., :3], T["d1"].shape, T["gd1"], T["d1"])
    dgrad("d1", T["gd1"], T["d1a"].shape, T["gd1a"], T["d1a"])
    lo_c1, hi_c1 = dgrad("c1", T["gd1a"], T["cat1"].shape, None)
    _assert_within("dgrad c1 (up-sampled part)", T["gcat1"][..., :32], lo_c1[..., :32], hi_c1[..., :32])
    ub = U.up_backward(T["gcat1"][..., :32])
    lo, hi = _rounded_interval(ub, U.up_backward(np.abs(T["gcat1"][..., :32])), 9)
    _assert_within("up-sampling gradient d2", T["gd2"], lo * (T["d2"] > 0), hi * (T["d2"] > 0))
    dgrad("d2", T["gd2"], T["d2a"].shape, T["gd2a"], T["d2a"])
    lo_c2, hi_c2 = dgrad("c2", T["gd2a"], T["cat2"].shape, None)
    _assert_within("dgrad c2 (up-sampled part)", T["gcat2"][..., :64], lo_c2[..., :64], hi_c2[..., :64])
    ub = U.up_backward(T["gcat2"][..., :64])
    lo, hi = _rounded_interval(ub, U.up_backward(np.abs(T["gcat2"][..., :64])), 9)
    _assert_within("up-sampling gradient e3", T["ge3"], lo * (T["e3"] > 0), hi * (T["e3"] > 0))
    dgrad("b3", T["ge3"], T["e3a"].shape, T["ge3a"], T["e3a"])
    dgrad("a3", T["ge3a"], T["p2"].shape, T["gp2"])
    for skip, gp, act, lo_s, hi_s in (("ge2", "gp2", "e2", lo_c2[..., 64:], hi_c2[..., 64:]),
                                      ("ge1", "gp1", "e1", lo_c1[..., 32:], hi_c1[..., 32:])):
        if skip == "ge1":
            dgrad("b2", T["ge2"], T["e2a"].shape, T["ge2a"], T["e2a"])
            dgrad("a2", T["ge2a"], T["p1"].shape, T["gp1"])
        pb = U.up(T[gp]) * 0.125
        e = U_ACC * (np.abs(pb) + np.maximum(np.abs(lo_s), np.abs(hi_s)))
        m = T[act] > 0
        _assert_within(f"skip + pooling gradient {act}", T[skip], rne_bf16(pb + lo_s - e) * m,
                       rne_bf16(pb + hi_s + e) * m)
    dgrad("b1", T["ge1"], T["e1a"].shape, T["ge1a"], T["e1a"])

    # ---- weight and bias gradients (FP32 sums over all voxels)
    for name, xl, gy in (("head", T["d1"], T["gout"][..., :3]), ("d1", T["d1a"], T["gd1"]),
                         ("c1", T["cat1"], T["gd1a"]), ("d2", T["d2a"], T["gd2"]), ("c2", T["cat2"], T["gd2a"]),
                         ("b3", T["e3a"], T["ge3"]), ("a3", T["p2"], T["ge3a"]), ("b2", T["e2a"], T["ge2"]),
                         ("a2", T["p1"], T["ge2a"]), ("b1", T["e1a"], T["ge1"]), ("a1", T["x"][..., :6], T["ge1a"])):
        _wgrad_check(name, xl, gy, *G[name])
