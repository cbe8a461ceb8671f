"""Learned warm start and the Gauss-Newton energy target, through the C ABI.

* The network input (u / h and the data-term gradient scaled by one Jacobi step of the
  full system) against the FP64 oracle's right-hand side with w_r = 0 (Eq. 2-3 only)
  and its diagonal; tolerance as for the other single stages (2e-5 of the scale).
* vd_warm_start keeps a prediction only when it lowers E_total (Eq. 1): a zero network
  leaves u as it was; a wild network is rejected and u, R are restored bit for bit.
* An energy target ends the flip-flop loop after the first iteration that reaches it.
"""
import numpy as np
import pytest

import oracle
from oracle import unet_ref as U
from paper_1603_08161_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1603_08161_b300 import vd as mod
    return mod


def _frame():
    # 16^3 lattice (a multiple of 4 per axis, as the network needs)
    return synth.sphere_frame(W=64, H=48, f=60.0, n=16, seed=5, n_sparse=20, name="sphere16")


def _warp(nn, seed):
    rng = np.random.default_rng(seed)
    u = rng.normal(0, 0.003, (nn, 3)).astype(np.float32)
    w = rng.normal(0, 0.03, (nn, 3))
    R = np.zeros((nn, 3, 3))
    for i in range(nn):
        th = np.linalg.norm(w[i])
        k = w[i] / th
        Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R[i] = np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx
    return u, R.astype(np.float32)


def _degrees(mask, dims):
    nx, ny, nz = dims
    m = mask.reshape(nz, ny, nx)
    deg = np.zeros_like(m, dtype=np.int64)
    for ax in range(3):
        for s in (1, -1):
            sh = np.zeros_like(m)
            src = [slice(None)] * 3
            dst = [slice(None)] * 3
            if s == 1:
                src[ax], dst[ax] = slice(1, None), slice(None, -1)
            else:
                src[ax], dst[ax] = slice(None, -1), slice(1, None)
            sh[tuple(dst)] = m[tuple(src)]
            deg += sh & m
    return deg.reshape(-1)


@pytest.mark.parametrize("mode", ["all", "surface"])
def test_features_match_oracle(vd, mode):
    fr = _frame()
    am = vd.VD_ACTIVE_ALL if mode == "all" else vd.VD_ACTIVE_SURFACE
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, am)
    lat.set_frame_from(fr)
    u, R = _warp(lat.nn, 1)
    lat.set_warp(u, R)
    prm = vd.params()
    x = lat.warm_features(prm)
    ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE,
                                   params=dict(w_reg=0.0))
    ref.set_warp(u.astype(np.float64), R.astype(np.float64))
    ref.associate()
    b, d = ref.rhs()
    m = ref.active_mask()
    h = float(fr.spacing)
    dd = d + 2.0 * 1.0 * _degrees(m, fr.dims)[:, None]
    g = np.where(dd > 0, b / (h * np.where(dd > 0, dd, 1.0)), 0.0)
    g[~m] = 0.0
    uu = np.where(m[:, None], u.astype(np.float64) / h, 0.0)
    assert np.abs(x[:, :3] - uu).max() < 1e-6 * max(np.abs(uu).max(), 1.0)
    assert np.abs(x[:, 3:] - g).max() < 2e-5 * np.abs(g).max()
    assert np.abs(g).max() > 0


@pytest.mark.parametrize("mode", ["all", "surface"])
def test_zero_network_keeps_u(vd, mode):
    fr = _frame()
    am = vd.VD_ACTIVE_ALL if mode == "all" else vd.VD_ACTIVE_SURFACE
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, am)
    lat.set_frame_from(fr)
    u, R = _warp(lat.nn, 2)
    lat.set_warp(u, R)
    net = vd.UNet(fr.dims)
    net.set_params(np.zeros(net.n_params, np.float32))
    prm = vd.params()
    rep = lat.warm_start(net, prm)
    u1, R1 = lat.get_warp()
    np.testing.assert_array_equal(u1, u)
    ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
    ref.set_warp(u.astype(np.float64), R.astype(np.float64))
    ref.associate()
    e0 = ref.energy()[0]
    assert abs(rep["e_start"] - e0) / e0 < 1e-5
    ref.fit_rotations()
    ref.associate()
    e1 = ref.energy()[0]
    assert abs(rep["e_predicted"] - e1) / e1 < 1e-5
    # refitting the rotations of a random warp lowers E_reg: the candidate is kept
    assert rep["used_prediction"] == 1 and e1 < e0
    m = ref.active_mask()
    _, R0 = ref.get_warp()
    assert np.abs(R1[m] - R0[m]).max() < 1e-5


def test_wild_network_is_rejected(vd):
    fr = _frame()
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL)
    lat.set_frame_from(fr)
    u, R = _warp(lat.nn, 3)
    lat.set_warp(u, R)
    net = vd.UNet(fr.dims)
    net.set_params((U.he_params(9) * 30.0).astype(np.float32))
    rep = lat.warm_start(net, vd.params())
    assert rep["used_prediction"] == 0 and not (rep["e_predicted"] < rep["e_start"])
    u1, R1 = lat.get_warp()
    np.testing.assert_array_equal(u1, u)
    np.testing.assert_array_equal(R1.reshape(-1, 9), R.reshape(-1, 9))


def test_network_grid_must_match(vd):
    fr = _frame()
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL)
    lat.set_frame_from(fr)
    net = vd.UNet((8, 8, 8))
    with pytest.raises(vd.VDError):
        lat.warm_start(net, vd.params())


@pytest.mark.parametrize("mode", ["all", "surface"])
@pytest.mark.parametrize("persistent", [True, False])
def test_energy_target_stops_early(vd, mode, persistent, monkeypatch):
    monkeypatch.setenv("VD_PERSISTENT", "1" if persistent else "0")
    fr = synth.config1()
    am = vd.VD_ACTIVE_ALL if mode == "all" else vd.VD_ACTIVE_SURFACE
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, am)
    lat.set_frame_from(fr)
    r3 = lat.solve(vd.params(gn_iters=3, cg_iters=10, init=vd.VD_INIT_ZERO))
    u3, _ = lat.get_warp()
    lat.set_energy_target(r3["e_total"] * (1 + 1e-7))
    r = lat.solve(vd.params(gn_iters=10, cg_iters=10, init=vd.VD_INIT_ZERO))
    assert r["gn_done"] == 3
    assert r["e_total"] <= r3["e_total"] * (1 + 1e-7)
    u, _ = lat.get_warp()
    assert np.abs(u - u3).max() < 1e-5 * fr.spacing
    # a target that is never met runs every iteration; removing it does too
    lat.set_energy_target(0.0)
    assert lat.solve(vd.params(gn_iters=10, cg_iters=10, init=vd.VD_INIT_ZERO))["gn_done"] == 10
    lat.set_energy_target(-1.0)
    r10 = lat.solve(vd.params(gn_iters=10, cg_iters=10, init=vd.VD_INIT_ZERO))
    assert r10["gn_done"] == 10 and r10["e_total"] < r3["e_total"]
