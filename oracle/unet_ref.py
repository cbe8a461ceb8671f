"""FP64 CPU reference of the warm-start U-Net -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import this
module; the CUDA library never loads it and shares no code with it.  It is the plain
definition of the network that the library documents (include/vd.h, learned warm
start), written with numpy in double precision, and the hand-derived backward pass:

  volumes are (D, H, W, C) arrays (z, y, x, channel), node i = x + W (y + H z);
  conv(x; w, b)[v, co] = b[co] + sum_tap sum_ci x[v + off(tap), ci] w[tap, ci, co], with
      off(tap) = (tap // 9 - 1, tap // 3 % 3 - 1, tap % 3 - 1) and zeros outside;
  pool = mean over 2x2x2 blocks, up = nearest-neighbour copy to 2x2x2 blocks;
  e1 = relu(b1(relu(a1(x))))          cat1 = [up(d2), e1]
  e2 = relu(b2(relu(a2(pool(e1)))))   cat2 = [up(e3), e2]
  e3 = relu(b3(relu(a3(pool(e2)))))   d2 = relu(d2c(relu(c2(cat2))))
  out = head(relu(d1c(relu(c1(cat1)))))
  loss = sum over nodes i of w_i |out_i - target_i|^2 / (3 n), with w_i = 1 + lambda at
      nodes whose gradient input (channels 3-5) is not all zero, else 1.

Parity status: pinned.  tests/test_unet_ref.py checks the convolution against
scipy.ndimage.correlate, pooling and up-sampling against closed forms, the parameter
count against the layer table, and every gradient against central finite differences
of the loss.  (No part of the network comes from the paper; the method's own warm start
is the previous frame's warp, Sec. 7.1.)
"""
from __future__ import annotations

import numpy as np

# (name, Cin, Cout) in parameter order
LAYERS = [("a1", 6, 16), ("b1", 16, 16), ("a2", 16, 32), ("b2", 32, 32), ("a3", 32, 64), ("b3", 64, 64),
          ("c2", 96, 32), ("d2", 32, 32), ("c1", 48, 16), ("d1", 16, 16), ("head", 16, 3)]


def num_params():
    return sum(27 * ci * co + co for _, ci, co in LAYERS)


def unpack(flat):
    """Flat parameter vector -> {name: (w (27, Cin, Cout), b (Cout,))}."""
    flat = np.asarray(flat, np.float64)
    out, k = {}, 0
    for name, ci, co in LAYERS:
        w = flat[k:k + 27 * ci * co].reshape(27, ci, co)
        k += 27 * ci * co
        b = flat[k:k + co]
        k += co
        out[name] = (w, b)
    assert k == flat.size
    return out


def pack(grads):
    return np.concatenate([np.concatenate([grads[n][0].ravel(), grads[n][1].ravel()]) for n, _, _ in LAYERS])


def _offsets():
    return [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def _shifted(xp, dz, dy, dx, D, H, W):
    """x[v + off] for every v, from the zero-padded volume xp."""
    return xp[1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W]


def conv(x, w, b):
    D, H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (D, H, W, b.size)).copy()
    for t, (dz, dy, dx) in enumerate(_offsets()):
        y += _shifted(xp, dz, dy, dx, D, H, W) @ w[t]
    return y


def conv_backward(x, w, gy):
    """Gradients of sum(gy * conv(x; w, b)) with respect to x, w and b."""
    D, H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    g2 = gy.reshape(-1, gy.shape[-1])
    for t, (dz, dy, dx) in enumerate(_offsets()):
        xs = _shifted(xp, dz, dy, dx, D, H, W)
        gw[t] = xs.reshape(-1, xs.shape[-1]).T @ g2
        gxp[1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + W] += gy @ w[t].T
    return gxp[1:-1, 1:-1, 1:-1], gw, gy.sum(axis=(0, 1, 2))


def pool(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def pool_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_backward(gy):
    D, H, W, C = gy.shape
    return gy.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def forward(p, x):
    """Network output and every intermediate (for the backward pass)."""
    a = {}
    a["x"] = x
    a["e1a"] = relu(conv(x, *p["a1"]))
    a["e1"] = relu(conv(a["e1a"], *p["b1"]))
    a["p1"] = pool(a["e1"])
    a["e2a"] = relu(conv(a["p1"], *p["a2"]))
    a["e2"] = relu(conv(a["e2a"], *p["b2"]))
    a["p2"] = pool(a["e2"])
    a["e3a"] = relu(conv(a["p2"], *p["a3"]))
    a["e3"] = relu(conv(a["e3a"], *p["b3"]))
    a["cat2"] = np.concatenate([up(a["e3"]), a["e2"]], axis=-1)
    a["d2a"] = relu(conv(a["cat2"], *p["c2"]))
    a["d2"] = relu(conv(a["d2a"], *p["d2"]))
    a["cat1"] = np.concatenate([up(a["d2"]), a["e1"]], axis=-1)
    a["d1a"] = relu(conv(a["cat1"], *p["c1"]))
    a["d1"] = relu(conv(a["d1a"], *p["d1"]))
    a["out"] = conv(a["d1"], *p["head"])
    return a["out"], a


def node_weights(x, surface_weight):
    """w_i = 1 + surface_weight where the gradient input (channels 3-5) is not all zero."""
    return 1.0 + surface_weight * np.any(x[..., 3:6] != 0, axis=-1, keepdims=True)


def loss(out, target, w=1.0):
    """sum_i w_i |out_i - target_i|^2 / (3 n)."""
    return float(np.mean(w * (out - target) ** 2))


def backward(p, a, target, w=1.0):
    """Gradients of the loss with respect to every parameter: {name: (gw, gb)}."""
    g = {}
    gout = 2.0 * w * (a["out"] - target) / a["out"].size

    def layer(name, x_in, gy, y_relu=None):
        if y_relu is not None:
            gy = gy * (y_relu > 0)
        gx, gw, gb = conv_backward(x_in, p[name][0], gy)
        g[name] = (gw, gb)
        return gx

    gd1 = layer("head", a["d1"], gout)
    gd1a = layer("d1", a["d1a"], gd1, a["d1"])
    gcat1 = layer("c1", a["cat1"], gd1a, a["d1a"])
    c = a["d2"].shape[-1]
    gd2 = up_backward(gcat1[..., :c])
    ge1 = gcat1[..., c:]
    gd2a = layer("d2", a["d2a"], gd2, a["d2"])
    gcat2 = layer("c2", a["cat2"], gd2a, a["d2a"])
    c = a["e3"].shape[-1]
    ge3 = up_backward(gcat2[..., :c])
    ge2 = gcat2[..., c:]
    ge3a = layer("b3", a["e3a"], ge3, a["e3"])
    gp2 = layer("a3", a["p2"], ge3a, a["e3a"])
    ge2 = ge2 + pool_backward(gp2)
    ge2a = layer("b2", a["e2a"], ge2, a["e2"])
    gp1 = layer("a2", a["p1"], ge2a, a["e2a"])
    ge1 = ge1 + pool_backward(gp1)
    ge1a = layer("b1", a["e1a"], ge1, a["e1"])
    layer("a1", a["x"], ge1a, a["e1a"])
    return g


def he_params(seed, head_scale=1.0):
    """Seeded He-normal weights and small random biases (a test input, not the
    library's initialisation)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, ci, co in LAYERS:
        s = np.sqrt(2.0 / (27.0 * ci)) * (head_scale if name == "head" else 1.0)
        parts.append(rng.normal(0.0, s, 27 * ci * co))
        parts.append(rng.normal(0.0, 0.05, co))
    return np.concatenate(parts)
