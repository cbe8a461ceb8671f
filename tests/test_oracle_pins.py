"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a hand computation, a brute-force search or a library routine, chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails one of them.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from paper_1603_08161_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_rot(rng, scale=1.0):
    """Rotation from an axis-angle vector (Rodrigues), angle ~ scale * |N(0, 1)|."""
    w = rng.normal(size=3) * scale
    th = np.linalg.norm(w)
    if th == 0:
        return np.eye(3)
    k = w / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx


def _node_pos(fr):
    nx, ny, nz = fr.dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.float64)
    return fr.origin.astype(np.float64) + float(np.float32(fr.spacing)) * idx


def _with_sparse(fr, canon, target):
    return dataclasses.replace(fr, sp_canon=np.asarray(canon, np.float32).reshape(-1, 3),
                               sp_target=np.asarray(target, np.float32).reshape(-1, 3))


def _no_dense(fr):
    return dataclasses.replace(fr, src_pts=np.zeros((0, 3), np.float32),
                               src_nrm=np.zeros((0, 3), np.float32))


def _small_frame(n=4, tilt=20.0, shift=(0.0, 0.0, 0.01), n_sparse=6, seed=0):
    rng = np.random.default_rng(seed)
    fr = synth.plane_frame(W=32, H=24, f=30.0, n=n, tilt_deg=tilt, shift=shift)
    lo = fr.origin.astype(np.float64) + 0.1
    hi = lo + (np.array(fr.dims) - 1) * fr.spacing - 0.2
    canon = rng.uniform(lo, hi, size=(n_sparse, 3))
    target = canon + rng.normal(0, 0.01, size=canon.shape)
    return _with_sparse(fr, canon, target)


# ---------------------------------------------------------------- golden single cell

def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, *v = line.split()
                out[k] = np.array([float(x) for x in v])
    return out


def test_single_cell_golden():
    g = _golden("single_cell.txt")
    dims = tuple(int(v) for v in g["dims"])
    fr = synth.Frame(depth=np.zeros((4, 4), np.float32), K=np.array([4, 4, 1.5, 1.5], np.float32),
                     pose=np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float32),
                     src_pts=np.zeros((0, 3), np.float32), src_nrm=np.zeros((0, 3), np.float32),
                     sp_canon=g["f_hat"].reshape(1, 3).astype(np.float32),
                     sp_target=(g["f_hat"] + g["d"]).reshape(1, 3).astype(np.float32),
                     dims=dims, origin=g["origin"].astype(np.float32), spacing=float(g["spacing"][0]))
    w = g["weights"]
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL,
                                 params=dict(w_sparse=w[0], w_dense=w[1], w_reg=w[2]))
    o.associate()
    # float32 inputs: the pair's offset is d only up to float32 rounding of f
    d32 = (np.float32(g["f_hat"] + g["d"]).astype(np.float64) - np.float32(g["f_hat"]).astype(np.float64))
    e = o.energy()
    assert e[2] == pytest.approx(float(d32 @ d32), rel=1e-12)
    assert e[3] == 0.0 and e[1] == 0.0
    assert e[0] == pytest.approx(w[0] * float(d32 @ d32), rel=1e-12)
    assert g["E_total"][0] == pytest.approx(w[0] * float(g["d"] @ g["d"]), rel=1e-12)
    b, diag = o.rhs()
    np.testing.assert_allclose(b, np.tile(1.25 * d32, (8, 1)), rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(b, np.tile(g["b"], (8, 1)), rtol=2e-5)
    np.testing.assert_allclose(diag, np.full((8, 3), g["diag"][0]), rtol=1e-6)
    p = np.zeros((8, 3))
    p[0, 0] = 1.0
    q = o.apply(p)
    assert q[0, 0] == pytest.approx(g["Ap_node0_x"][0], rel=1e-6)
    for j in (1, 2, 4):
        assert q[j, 0] == pytest.approx(g["Ap_nbr_x"][0], rel=1e-6)
    for j in (3, 5, 6, 7):
        assert q[j, 0] == pytest.approx(g["Ap_far_x"][0], rel=1e-6)
    assert np.abs(q[:, 1:]).max() < 1e-12
    delta = o.cholesky()
    np.testing.assert_allclose(delta, np.tile(d32, (8, 1)), atol=1e-12)
    o.add_increment(delta)
    assert o.fit_rotations() == 0
    _, R = o.get_warp()
    np.testing.assert_allclose(R, np.tile(np.eye(3), (8, 1, 1)), atol=1e-12)
    assert o.energy()[0] < 1e-24


# ---------------------------------------------------------------- S(x), Sec. 4

@pytest.mark.parametrize("with_pose", [False, True])
def test_affine_warp_reproduced_exactly(with_pose):
    """Trilinear interpolation reproduces affine maps: with u_i = (Q - I) t^_i + c,
    S(x) = R_g (Q x + c) + t_g for every interior x, so targets placed there give
    E_sparse = 0, and moving one target by e gives E_sparse = |e|^2."""
    rng = np.random.default_rng(3)
    fr = _no_dense(synth.plane_frame(n=5))
    Q = _rand_rot(rng, 0.3) + 0.05 * rng.normal(size=(3, 3))      # a general affine map
    c = rng.normal(0, 0.02, 3)
    Rg, tg = (_rand_rot(rng, 0.2), rng.normal(0, 0.05, 3)) if with_pose else (np.eye(3), np.zeros(3))
    fr = dataclasses.replace(fr, pose=np.concatenate([Rg.ravel(), tg]).astype(np.float32))
    Rg = fr.pose[:9].astype(np.float64).reshape(3, 3)
    tg = fr.pose[9:].astype(np.float64)
    lo = fr.origin.astype(np.float64)
    hi = lo + (np.array(fr.dims) - 1) * fr.spacing
    x = rng.uniform(lo + 1e-3, hi - 1e-3, size=(50, 3)).astype(np.float32).astype(np.float64)
    tgt = (Rg @ (Q @ x.T + c[:, None])).T + tg
    e = np.zeros_like(tgt)
    e[7] = [1e-3, -2e-3, 5e-4]
    fr = _with_sparse(fr, x, (tgt + e))
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    P = _node_pos(fr)
    o.set_warp(u=(P @ (Q - np.eye(3)).T) + c)
    tgt32 = (tgt + e).astype(np.float32).astype(np.float64)
    expect = np.sum(((Rg @ (Q @ x.T + c[:, None])).T + tg - tgt32) ** 2)
    assert o.energy()[2] == pytest.approx(expect, rel=1e-9, abs=1e-20)
    assert expect == pytest.approx(e[7] @ e[7], rel=1e-3)


# ---------------------------------------------------------------- E_reg, Eq. 4

def test_arap_zero_under_rigid_motion_and_rotation_step_recovers_it():
    rng = np.random.default_rng(5)
    fr = _no_dense(synth.plane_frame(n=5))
    Q = _rand_rot(rng, 0.7)
    c = rng.normal(0, 0.05, 3)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    P = _node_pos(fr)
    u = P @ (Q - np.eye(3)).T + c
    o.set_warp(u=u, R=np.tile(Q, (o.nn, 1, 1)))
    e = o.energy()
    assert e[3] < 1e-26 * o.nn
    o.set_warp(u=u)                         # R = I: the rotation step must find Q
    assert o.energy()[3] > 1e-4
    assert o.fit_rotations() == 0
    _, R = o.get_warp()
    assert np.abs(R - Q).max() < 1e-12
    assert o.energy()[3] < 1e-26 * o.nn


def test_arap_single_displaced_node_closed_form():
    """Moving one interior node by delta (R = I) touches 6 undirected edges, each
    counted in both directions: E_reg = 12 |delta|^2.  A boundary corner: 6 |delta|^2."""
    fr = _no_dense(synth.plane_frame(n=5))
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    delta = np.array([0.003, -0.001, 0.002])
    for node, deg in ((2 + 5 * (2 + 5 * 2), 6), (0, 3), (2, 4)):
        u = np.zeros((o.nn, 3))
        u[node] = delta
        o.set_warp(u=u)
        assert o.energy()[3] == pytest.approx(2 * deg * delta @ delta, rel=1e-12)


# ---------------------------------------------------------------- target maps + association

def test_target_maps_plane_by_hand():
    fr = synth.plane_frame(W=12, H=9, f=10.0, n=4, tilt_deg=25.0)
    o = oracle.Oracle.from_frame(fr)
    V, N, valid = o.target_maps()
    fx, fy, cx, cy = fr.K.astype(np.float64)
    vv, uu = np.mgrid[0:9, 0:12]
    D = fr.depth.astype(np.float64)
    np.testing.assert_allclose(V[..., 2], D, rtol=0, atol=0)
    np.testing.assert_allclose(V[..., 0], D * (uu - cx) / fx, rtol=1e-15, atol=1e-15)
    interior = np.zeros_like(valid)
    interior[1:-1, 1:-1] = True
    assert (valid == interior).all()
    th = math.radians(25.0)
    nrm = np.array([math.sin(th), 0.0, -math.cos(th)])            # plane normal facing camera
    np.testing.assert_allclose(N[valid], np.tile(nrm, (valid.sum(), 1)), atol=2e-6)
    # a hole invalidates the centre and its 4-neighbours
    d2 = fr.depth.copy()
    d2[4, 5] = 0
    o2 = oracle.Oracle.from_frame(dataclasses.replace(fr, depth=d2))
    _, _, v2 = o2.target_maps()
    for (r, q) in ((4, 5), (3, 5), (5, 5), (4, 4), (4, 6)):
        assert not v2[r, q]
    assert v2[3, 4] and v2[5, 6]


@pytest.mark.parametrize("tilt,dz,rot", [(0.0, 0.0, 0.0), (0.0, 0.01, 0.0), (30.0, 0.004, 0.0),
                                         (0.0, 0.0, 25.0), (30.0, 0.004, -20.0)])
def test_association_weights_by_hand(tilt, dz, rot):
    """Plane seen through its own pixels: each sample projects to its own pixel, and
    w_c = ((Phi_d + Phi_n + Phi_v)/3)^2 with Phi_r(x) = 1 - x/eps_r (Sec. 5.1).  With
    every R_i = Q (u = 0) the model normal is Q n^_c."""
    eps_d, eps_n, eps_v = 0.05, 0.5, 0.8
    fr = synth.plane_frame(W=16, H=12, f=12.0, n=8, tilt_deg=tilt, shift=(0, 0, dz))
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    Q = synth._rotation([0.0, 1.0, 0.0], math.radians(rot))
    o.set_warp(None, np.tile(Q, (o.nn, 1, 1)))
    o.associate()
    pix, w, r = o.association()
    cell, _ = o.sample_cells()
    fx, fy, cx, cy = fr.K.astype(np.float64)
    th = math.radians(tilt)
    nrm = np.array([math.sin(th), 0.0, -math.cos(th)])
    checked = 0
    for s in range(fr.C):
        v, u = divmod(s, fr.W)
        if cell[s] < 0 or not (1 <= u < fr.W - 1 and 1 <= v < fr.H - 1):
            assert w[s] == 0
            continue
        assert pix[s] == s
        p = fr.src_pts[s].astype(np.float64)
        pa = fr.depth[v, u] * np.array([(u - cx) / fx, (v - cy) / fy, 1.0])
        nc = Q @ fr.src_nrm[s].astype(np.float64)
        phi_d = 1 - np.linalg.norm(p - pa) / eps_d
        phi_n = 1.0 - (1.0 - nc @ nrm) / eps_n
        phi_v = 1 - (1 - nc @ (-p / np.linalg.norm(p))) / eps_v
        if min(phi_d, phi_n, phi_v) < 0:
            assert w[s] == 0
            continue
        assert w[s] == pytest.approx(((phi_d + phi_n + phi_v) / 3) ** 2, rel=2e-5)
        assert r[s] == pytest.approx(math.sqrt(w[s]) * (p - pa) @ nrm, abs=2e-7)
        checked += 1
    assert checked > 20


def test_association_pruning_thresholds():
    """A sample farther than eps_d from its target, or whose normal deviates by more
    than eps_n, or seen at a grazing angle beyond eps_v, gets w_c = 0."""
    fr = synth.plane_frame(W=16, H=12, f=12.0, n=8, shift=(0, 0, 0.06))       # 6 cm > eps_d
    o = oracle.Oracle.from_frame(fr)
    assert o.associate() == 0
    o.set_params(eps_d=0.07)
    assert o.associate() > 0
    fr2 = synth.plane_frame(W=16, H=12, f=12.0, n=8, tilt_deg=78.0)           # grazing view
    o2 = oracle.Oracle.from_frame(fr2)
    o2.associate()
    pix, w, _ = o2.association()
    th = math.radians(78.0)
    nrm = np.array([math.sin(th), 0.0, -math.cos(th)])
    p = fr2.src_pts.astype(np.float64)
    ndotv = -(p @ nrm) / np.linalg.norm(p, axis=1)
    ok = pix >= 0
    graze = ok & (1 - ndotv > 0.8)
    assert graze.sum() >= 3 and (ok & ~graze).sum() >= 3
    assert np.all(w[graze] == 0) and np.all(w[ok & ~graze] > 0)
    bent = dataclasses.replace(fr, src_nrm=np.tile(np.float32([0.8, 0, -0.6]), (fr.C, 1)))
    o3 = oracle.Oracle.from_frame(dataclasses.replace(bent, depth=synth.plane_frame(
        W=16, H=12, f=12.0, n=8).depth))                                      # 1 - 0.6 = 0.4 < 0.5
    assert o3.associate() > 0
    o3.set_params(eps_n=0.35)
    assert o3.associate() == 0


def test_active_set_one_ring():
    """One sample in cell (1,1,1) of a 5^3 lattice: M = its 8 corners plus their
    6-neighbours = 8 + 6 * 4 = 32 nodes (Sec. 6)."""
    fr = _no_dense(synth.plane_frame(n=5))
    h = fr.spacing
    x = fr.origin.astype(np.float64) + 1.5 * h
    fr = dataclasses.replace(fr, src_pts=np.float32([x]), src_nrm=np.float32([[0, 0, -1]]))
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_SURFACE)
    m = o.active_mask().reshape(5, 5, 5)                     # [z, y, x]
    assert m.sum() == 32
    assert m[1:3, 1:3, 1:3].all()
    assert not m[0, 0, 0] and m[0, 1, 1] and m[1, 1, 3] and not m[3, 3, 3]


# ---------------------------------------------------------------- Jacobian vs E

@pytest.mark.parametrize("mode,posed", [(oracle.ACTIVE_ALL, False), (oracle.ACTIVE_SURFACE, False),
                                         (oracle.ACTIVE_ALL, True)])
def test_jacobian_matches_finite_differences(mode, posed):
    """-2 b = grad E (b = -J^T r) against central differences of E (Eq. 1) with the
    association held fixed, on a 4^3 lattice with random warp and rotations (and a
    non-identity global pose R_g, t_g)."""
    rng = np.random.default_rng(11)
    fr = _small_frame(n=4)
    if posed:
        Rg = _rand_rot(np.random.default_rng(99), 0.05)
        fr = dataclasses.replace(fr, pose=np.concatenate([Rg.ravel(), [0.004, -0.003, 0.002]]).astype(np.float32))
    o = oracle.Oracle.from_frame(fr, mode, params=dict(w_sparse=3.0, w_dense=2.0, w_reg=0.7))
    u0 = rng.normal(0, 0.004, (o.nn, 3))
    R0 = np.stack([_rand_rot(rng, 0.1) for _ in range(o.nn)])
    o.set_warp(u0, R0)
    assert o.associate() > 10
    b, _ = o.rhs()
    act = o.active_mask()
    eps = 1e-6
    worst = 0.0
    for i in np.nonzero(act)[0]:
        for a in range(3):
            up = u0.copy()
            up[i, a] += eps
            o.set_warp(up, R0)
            ep = o.energy()[0]
            up[i, a] -= 2 * eps
            o.set_warp(up, R0)
            em = o.energy()[0]
            fd = (ep - em) / (2 * eps)
            worst = max(worst, abs(fd - (-2 * b[i, a])) / (abs(fd) + 1e-3))
    assert worst < 1e-6
    assert np.all(b[~act] == 0)


# ---------------------------------------------------------------- position step

@pytest.mark.parametrize("n", [4, 5, 6])
def test_pcg_reaches_cholesky(n):
    rng = np.random.default_rng(n)
    fr = _small_frame(n=n, seed=n)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    o.set_warp(rng.normal(0, 0.003, (o.nn, 3)), np.stack([_rand_rot(rng, 0.05) for _ in range(o.nn)]))
    o.associate()
    exact = o.cholesky()
    x, it, _ = o.pcg(3 * o.num_active() + 50, tol=1e-15)
    assert np.abs(x - exact).max() < 1e-10
    # the Cholesky solve itself against numpy on the dense normal matrix built column by column
    N3 = 3 * o.nn
    A = np.zeros((N3, N3))
    for k in range(N3):
        e = np.zeros(N3)
        e[k] = 1.0
        A[:, k] = o.apply(e).ravel()
    b, _ = o.rhs()
    np.testing.assert_allclose(A, A.T, atol=1e-12)
    ref = np.linalg.solve(A, b.ravel())
    assert np.abs(ref - exact.ravel()).max() < 1e-10


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_pcg_iterates_match_textbook_pcg(k):
    """The first k iterates of the Jacobi-preconditioned CG equal those of a textbook
    PCG (scipy.sparse.linalg.cg, x0 = 0, M = diag(J^T J)^-1) on the same system."""
    from scipy.sparse.linalg import cg
    rng = np.random.default_rng(21)
    fr = _small_frame(n=4, seed=3)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL, params=dict(w_sparse=30.0, w_reg=0.3))
    o.set_warp(rng.normal(0, 0.003, (o.nn, 3)))
    o.associate()
    N3 = 3 * o.nn
    A = np.zeros((N3, N3))
    for j in range(N3):
        e = np.zeros(N3)
        e[j] = 1.0
        A[:, j] = o.apply(e).ravel()
    b, _ = o.rhs()
    b = b.ravel()
    dg = np.diag(A).copy()
    assert np.ptp(dg) > 1.0                               # a non-trivial preconditioner
    x_ref, _ = cg(A, b, x0=np.zeros(N3), M=np.diag(1.0 / dg), maxiter=k, rtol=0.0, atol=0.0)
    x, it, _ = o.pcg(k)
    assert it == k
    assert np.abs(x.ravel() - x_ref).max() <= 1e-10 * np.abs(x_ref).max()


def test_translation_closed_form():
    """Sparse-only data with every target f = f^ + d (w_d = 0): the exact position step
    gives u_i = d on every node of the connected lattice and E = 0."""
    rng = np.random.default_rng(2)
    fr = _small_frame(n=5, n_sparse=9)
    d = np.array([0.012, -0.007, 0.02])
    fr = _with_sparse(fr, fr.sp_canon, fr.sp_canon.astype(np.float64) + d)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL, params=dict(w_dense=0.0))
    o.associate()
    delta = o.cholesky()
    d32 = (fr.sp_target.astype(np.float64) - fr.sp_canon.astype(np.float64)).mean(0)
    assert np.abs(delta - d).max() < 5e-8          # float32 rounding of the targets
    o.add_increment(delta)
    o.fit_rotations()
    assert o.energy()[0] < 1e-13
    x, it, _ = o.pcg(10)
    assert np.abs(x).max() < 1e-7
    del d32, rng


def test_arap_only_keeps_zero():
    fr = _small_frame(n=4)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL, params=dict(w_sparse=0.0, w_dense=0.0))
    res = o.solve(3, 10)
    u, R = o.get_warp()
    assert np.all(u == 0) and list(res["cg_done"]) == [0, 0, 0]
    assert np.abs(R - np.eye(3)).max() == 0


def test_rigid_sparse_targets_converge():
    """Sparse targets under a rigid motion (Q, c): flip-flop drives E to 0 and every
    R_i to Q (ARAP is minimised exactly by the rigid warp)."""
    rng = np.random.default_rng(8)
    fr = _no_dense(synth.plane_frame(n=4))
    lo = fr.origin.astype(np.float64)
    hi = lo + 3 * fr.spacing
    canon = rng.uniform(lo, hi, (12, 3))
    Q = _rand_rot(rng, 0.15)
    c = rng.normal(0, 0.01, 3)
    fr = _with_sparse(fr, canon, (canon @ Q.T) + c)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    o.associate()
    e0 = o.energy()[0]
    res = o.solve(60, 3 * 64 + 20, cg_tol=1e-14)
    e = res["energy"][:, 0]
    assert e[-1] < 1e-8 * e0
    _, R = o.get_warp()
    assert np.abs(R - Q).max() < 1e-3


def test_descent_with_fixed_association():
    """Block-coordinate descent: with the association frozen, E does not increase
    after any CG iteration (CG minimises the exactly quadratic position energy over
    growing Krylov spaces) nor after a rotation step (exact minimiser in R)."""
    rng = np.random.default_rng(4)
    fr = _small_frame(n=5)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    o.set_warp(rng.normal(0, 0.003, (o.nn, 3)))
    o.associate()
    for g in range(3):
        u0, R0 = o.get_warp()
        e_prev = o.energy()[0]
        for k in range(1, 25):
            o.set_warp(u0, R0)
            x, it, _ = o.pcg(k)
            o.add_increment(x)
            e = o.energy()[0]
            assert e <= e_prev * (1 + 1e-12)
            e_prev = e
        o.set_warp(u0, R0)
        x, _, _ = o.pcg(24)
        o.add_increment(x)
        e_before = o.energy()[0]
        o.fit_rotations()
        assert o.energy()[0] <= e_before * (1 + 1e-12)


# ---------------------------------------------------------------- rotation step, Sec. 7.1

def _objective(R, D, E):
    return np.sum((D - E @ R.T) ** 2)


def _rotvec(w):
    th = np.linalg.norm(w)
    if th < 1e-300:
        return np.eye(3)
    k = w / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_procrustes_matches_brute_force(seed):
    """Per-node rotation = argmin_R sum_j |(t_i - t_j) - R (t^_i - t^_j)|^2.  Compare
    with a dense search over SO(3) (random unit quaternions) refined by a local
    search in axis-angle coordinates, with no SVD involved."""
    rng = np.random.default_rng(seed)
    h = 0.1
    E = np.array([[h, 0, 0], [-h, 0, 0], [0, h, 0], [0, -h, 0], [0, 0, h], [0, 0, -h]])
    Qt = _rand_rot(rng, 1.5)
    D = E @ Qt.T + rng.normal(0, 0.03, E.shape)
    if seed == 3:
        D = D * np.array([1, 1, -1])                          # det(A) < 0 case
    A = D.T @ E                                               # sum_j d_j e_j^T
    R = oracle.procrustes(A)
    assert R is not None
    assert abs(np.linalg.det(R) - 1) < 1e-12 and np.abs(R.T @ R - np.eye(3)).max() < 1e-12
    q = rng.normal(size=(100000, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    a, b, c, d = q.T
    Rs = np.stack([np.stack([a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)], -1),
                   np.stack([2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)], -1),
                   np.stack([2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d], -1)], 1)
    objs = np.sum((D[None] - np.einsum("jb,nab->nja", E, Rs)) ** 2, axis=(1, 2))
    best = Rs[np.argmin(objs)]
    f_R = _objective(R, D, E)
    assert f_R <= objs.min() + 1e-12
    # local refinement: coordinate search on a left perturbation exp(w) best
    step = 0.05
    cur = best
    fcur = _objective(cur, D, E)
    while step > 1e-11:
        improved = False
        for k in range(3):
            for sgn in (1.0, -1.0):
                w = np.zeros(3)
                w[k] = sgn * step
                cand = _rotvec(w) @ cur
                fc = _objective(cand, D, E)
                if fc < fcur:
                    cur, fcur, improved = cand, fc, True
        if not improved:
            step *= 0.5
    # a derivative-free search resolves the minimiser only to ~sqrt(eps) ~ 1e-8
    assert np.abs(cur - R).max() < 1e-7
    assert f_R <= fcur + 1e-14
    # first-order optimality in closed form: R^T A is symmetric at the minimiser
    M = R.T @ A
    assert np.abs(M - M.T).max() < 1e-12 * np.abs(A).max()


def test_svd3_against_library():
    rng = np.random.default_rng(0)
    for _ in range(50):
        A = rng.normal(size=(3, 3))
        U, s, V = oracle.svd3(A)
        np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-12)
        np.testing.assert_allclose(U @ np.diag(s) @ V.T, A, atol=1e-12)
        np.testing.assert_allclose(U.T @ U, np.eye(3), atol=1e-12)
        np.testing.assert_allclose(V.T @ V, np.eye(3), atol=1e-12)
    A = np.outer([1.0, 2, 3], [0.5, -1, 2])                   # rank 1: not unique
    assert oracle.procrustes(A) is None
    A2 = np.array([[1.0, 0, 0], [0, 2, 0], [0, 0, 0]])        # rank 2: unique
    np.testing.assert_allclose(oracle.procrustes(A2), np.eye(3), atol=1e-15)


def test_rotation_degenerate_nodes_keep_previous():
    """When the deformed one-ring collapses onto a line, the best rotation is not
    unique (rank A_i <= 1): every node keeps its previous R_i and is counted.  A
    collapse onto a plane (rank 2) still has a unique best rotation."""
    fr = _no_dense(synth.plane_frame(n=4))
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    P = _node_pos(fr)
    rng = np.random.default_rng(1)
    Rr = np.stack([_rand_rot(rng, 0.2) for _ in range(o.nn)])
    line = np.zeros_like(P)
    line[:, 0] = P[:, 0]
    o.set_warp(line - P, Rr)
    assert o.fit_rotations() == o.nn
    _, R = o.get_warp()
    np.testing.assert_array_equal(R, Rr)
    plane = P.copy()
    plane[:, 2] = 1.0
    o.set_warp(plane - P, Rr)
    assert o.fit_rotations() == 0
    _, R = o.get_warp()
    np.testing.assert_allclose(R, np.tile(np.eye(3), (o.nn, 1, 1)), atol=1e-12)


def test_flip_flop_order_positions_before_rotations():
    """Sec. 7.1 fixes the order inside an iteration: positions with the rotations fixed,
    then rotations with the positions fixed.  From u = 0 and every R_i = Q != I, with one
    sparse pair whose target is its own canonical point f^ (w_d = 0), the exact position
    step with R = Q minimises w_s |S(f^) - f^|^2 + w_r E_reg(R = Q), which is zero only for
    the rigid rotation of the lattice about f^: u_i = (Q - I)(t^_i - f^); the rotation step
    then keeps R_i = Q.  Rotations first would refit R = I at u = 0 and leave u = 0."""
    rng = np.random.default_rng(11)
    fr = _no_dense(synth.plane_frame(n=4))
    f_hat = fr.origin.astype(np.float64) + np.array([1.3, 1.7, 0.6]) * fr.spacing
    fr = _with_sparse(fr, f_hat, f_hat)
    f32 = fr.sp_canon.astype(np.float64)[0]
    Q = _rand_rot(rng, 0.4)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL, params=dict(w_dense=0.0))
    o.set_warp(None, np.tile(Q, (o.nn, 1, 1)))
    res = o.solve(1, 0, cholesky=True)
    u, R = o.get_warp()
    u_closed = (_node_pos(fr) - f32) @ (Q - np.eye(3)).T
    assert np.abs(u - u_closed).max() < 1e-12
    assert np.abs(R - Q).max() < 1e-12
    assert res["energy"][-1, 0] < 1e-24


def test_solve_is_the_stages_in_the_papers_order():
    """vdo_solve with re-association equals driving the stages one by one in the order
    of Sec. 7.1 (associate, position step by PCG, add the increment, rotation step),
    which the per-iteration association checks of the GPU tests rely on."""
    fr = synth.config1()
    a = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    res = a.solve(3, 10, fixed_association=False)
    b = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    for g in range(3):
        b.associate()
        x, it, _ = b.pcg(10)
        b.add_increment(x)
        b.fit_rotations()
        assert np.array_equal(b.energy(), res["energy"][g])
    ua, Ra = a.get_warp()
    ub, Rb = b.get_warp()
    assert np.array_equal(ua, ub) and np.array_equal(Ra, Rb)


def test_non_finite_inputs_are_invalid():
    """A depth that is not a positive finite number is an invalid pixel (like 0), and a
    sample with a non-finite position or normal is ignored (like one outside the
    lattice): the frame then gives exactly the association and energy of the frame with
    those pixels set to 0 and those samples removed."""
    fr = synth.config1()
    rng = np.random.default_rng(5)
    on = np.argwhere(fr.depth > 0)
    pick = on[rng.choice(len(on), 12, replace=False)]
    depth = fr.depth.copy()
    depth[pick[:6, 0], pick[:6, 1]] = np.nan
    depth[pick[6:9, 0], pick[6:9, 1]] = np.inf
    depth[pick[9:, 0], pick[9:, 1]] = -np.inf
    bad = [5, 17, 23, 31, 40]
    pts, nrm = fr.src_pts.copy(), fr.src_nrm.copy()
    pts[5] = np.nan
    pts[17, 1] = np.inf
    nrm[23] = np.nan
    nrm[31, 2] = -np.inf
    nrm[40, 0] = np.inf
    noisy = dataclasses.replace(fr, depth=depth, src_pts=pts, src_nrm=nrm)
    keep = np.setdiff1d(np.arange(fr.C), bad)
    clean = dataclasses.replace(fr, depth=np.where(np.isfinite(depth) & (depth > 0), depth, 0).astype(np.float32),
                                src_pts=fr.src_pts[keep], src_nrm=fr.src_nrm[keep])
    a = oracle.Oracle.from_frame(noisy, oracle.ACTIVE_SURFACE)
    b = oracle.Oracle.from_frame(clean, oracle.ACTIVE_SURFACE)
    assert np.array_equal(a.active_mask(), b.active_mask())
    _, Na, va = a.target_maps()
    _, Nb, vb = b.target_maps()
    assert np.array_equal(va, vb) and np.array_equal(Na, Nb)
    ra = a.solve(2, 10, fixed_association=False)
    rb = b.solve(2, 10, fixed_association=False)
    pa, wa, _ = a.association()
    pb, wb, _ = b.association()
    assert (pa[bad] == -1).all() and (wa[bad] == 0).all()
    assert np.array_equal(pa[keep], pb) and np.array_equal(wa[keep], wb)
    assert np.array_equal(ra["energy"], rb["energy"]) and np.isfinite(ra["energy"]).all()
    # an observed feature position that is not finite makes the energy non-finite
    ft = fr.sp_target.copy()
    ft[2, 0] = np.nan
    c = oracle.Oracle.from_frame(dataclasses.replace(fr, sp_target=ft), oracle.ACTIVE_ALL)
    assert not np.isfinite(c.solve(1, 5)["energy"][-1, 0])


# ---------------------------------------------------------------- hierarchy (Sec. 7.2)

def test_coarse_levels_are_nested_parents():
    """n nodes per axis -> n // 2 + 1: coarse node X sits on finer node 2X, and the
    coarse lattice covers the finer one (its last cell is the parent of the last one)."""
    for n in (2, 3, 4, 9, 16, 17, 48, 49, 96):
        c = oracle.coarse_dims((n, n, n))[0]
        assert 2 * (c - 2) <= n - 2 <= 2 * (c - 1) - 1 or n == 2
        assert 2 * (c - 1) >= n - 1 and 2 * (c - 2) < n - 1 or n == 2
    assert oracle.coarse_dims((96, 96, 96)) == (49, 49, 49)
    assert oracle.coarse_dims((49, 49, 49)) == (25, 25, 25)


def _affine(pos, A, c):
    return pos @ A.T + c


def test_prolongation_and_injection_reproduce_affine_fields():
    """Trilinear prolongation reproduces an affine displacement field exactly at every
    finer node, and injection followed by prolongation onto a zero field gives it back."""
    rng = np.random.default_rng(12)
    fr = synth.config1()
    H = oracle.Hierarchy(fr, 3)
    A = rng.normal(0, 0.05, (3, 3))
    c = rng.normal(0, 0.01, 3)
    fine, coarse = H.levels[0], H.levels[1]
    pos_f = _node_pos(fr)
    crs = dataclasses.replace(fr, dims=coarse.dims, spacing=float(np.float32(2 * fr.spacing)))
    pos_c = _node_pos(crs)
    # prolongation of an affine coarse increment onto a zero fine field
    coarse.set_warp(_affine(pos_c, A, c))
    fine.set_warp(None)
    H.prolongate(1, np.zeros((coarse.nn, 3)))
    u, _ = fine.get_warp()
    assert np.abs(u - _affine(pos_f, A, c)).max() < 1e-13
    # injection of the fine field: coarse node X takes fine node 2X, and a coarse node
    # past the end of the (even) fine axis the linear extrapolation: the affine field
    starts = H.restrict()
    nx, ny, nz = fr.dims
    X, Y, Z = np.meshgrid(np.arange(coarse.dims[0]), np.arange(coarse.dims[1]), np.arange(coarse.dims[2]),
                          indexing="ij")
    inside = (2 * X < nx) & (2 * Y < ny) & (2 * Z < nz)
    src = (2 * X + nx * (2 * Y + ny * 2 * Z))[inside]
    dst = (X + coarse.dims[0] * (Y + coarse.dims[1] * Z))
    assert np.array_equal(starts[1][dst[inside]], u[src])
    assert (~inside).any()
    assert np.abs(starts[1] - _affine(pos_c, A, c)).max() < 1e-13
    # ... and prolongating the injected field onto zero reproduces the affine field
    fine.set_warp(None)
    H.prolongate(1, np.zeros((coarse.nn, 3)))
    u2, _ = fine.get_warp()
    assert np.abs(u2 - _affine(pos_f, A, c)).max() < 1e-13


def test_coarse_level_gathers_the_finest_constraints():
    """A coarse level holds exactly the constraints of the finest level, each expressed
    trilinearly in the coarse nodes: under a warp that is trilinear on the coarse grid
    (a random coarse field prolongated to the fine lattice, R = I) both levels warp every
    sample to the same point, so the association and the data energies (Eq. 2, 3)
    agree to rounding.  Samples outside the finest lattice stay out of the coarse one."""
    rng = np.random.default_rng(13)
    base = synth.config1()
    extra = base.src_pts[:40].copy()
    extra[:, 2] = 1.5                                          # beyond the fine lattice, inside the coarse
    fr = dataclasses.replace(base, src_pts=np.concatenate([base.src_pts, extra]),
                             src_nrm=np.concatenate([base.src_nrm, base.src_nrm[:40]]))
    H = oracle.Hierarchy(fr, 2)
    fine, coarse = H.levels
    cf, _ = fine.sample_cells()
    cc, _ = coarse.sample_cells()
    assert np.array_equal(cf < 0, cc < 0) and (cf[fr.C - 40:] < 0).any()
    coarse.set_warp(rng.normal(0, 0.01, (coarse.nn, 3)))
    fine.set_warp(None)
    H.prolongate(1, np.zeros((coarse.nn, 3)))
    fine.associate()
    coarse.associate()
    pf, wf, rf = fine.association()
    pc, wc, rc = coarse.association()
    assert np.array_equal(pf, pc) and (wf > 0).sum() > 100
    assert np.abs(wf - wc).max() < 1e-12 and np.abs(rf - rc).max() < 1e-12
    ef, ec = fine.energy(), coarse.energy()
    assert abs(ef[1] - ec[1]) <= 1e-10 * ef[1] and abs(ef[2] - ec[2]) <= 1e-10 * ef[2]


def test_hierarchy_recovers_rigid_targets():
    """Sparse targets under a rigid motion (Q, c): the coarse-to-fine flip-flop drives
    E to 0 and every fine R_i to Q, as the single level does."""
    rng = np.random.default_rng(14)
    fr = _no_dense(synth.plane_frame(n=9))
    lo = fr.origin.astype(np.float64)
    canon = rng.uniform(lo, lo + 8 * fr.spacing, (20, 3))
    Q = _rand_rot(rng, 0.15)
    c = rng.normal(0, 0.01, 3)
    fr = _with_sparse(fr, canon, canon @ Q.T + c)
    H = oracle.Hierarchy(fr, 2)
    res = H.solve([(30, 3 * 125), (30, 3 * 729)], fixed_association=True)
    assert res[-1]["energy"][-1, 0] < 1e-12
    _, R = H.levels[0].get_warp()
    assert np.abs(R - Q).max() < 1e-4


def test_coarse_start_resolves_the_low_frequencies():
    """The motivation of Sec. 7.2: a translation of every sparse target is a pure
    low-frequency correction that a few fine CG iterations propagate only a few nodes
    far; with the coarse levels first, the same fine iterations end far closer to the
    exact solution (u = d everywhere, E = 0)."""
    rng = np.random.default_rng(15)
    fr = _no_dense(synth.plane_frame(n=33))
    lo = fr.origin.astype(np.float64)
    canon = rng.uniform(lo, lo + 32 * fr.spacing, (30, 3))
    fr = _with_sparse(fr, canon, canon + np.array([0.02, -0.01, 0.015]))
    one = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    e1 = one.solve(2, 10)["energy"][-1, 0]
    H = oracle.Hierarchy(fr, 3)
    e3 = H.solve([(2, 10), (2, 10), (2, 10)])[-1]["energy"][-1, 0]
    assert e3 < 0.1 * e1


# ---------------------------------------------------------------- global pose (Sec. 6)

def _pose(Q, c):
    return np.concatenate([np.asarray(Q, np.float64).ravel(), np.asarray(c, np.float64)])


def test_icp_gradient_matches_finite_differences():
    """b of the pose's normal equations is half the gradient of the point-to-plane energy
    over the pose perturbation xi = (omega, tau) (R <- exp([omega]x) R, t <- t + tau),
    checked by central differences with the association held fixed."""
    rng = np.random.default_rng(21)
    Q0 = _rand_rot(rng, 0.03)
    fr = synth.corner_frame(rot=_rand_rot(rng, 0.05), shift=(0.01, -0.008, 0.012))
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    o.set_warp(rng.normal(0, 0.002, (o.nn, 3)))
    P0 = _pose(Q0, rng.normal(0, 0.005, 3))
    o.set_pose(P0)
    o.associate()
    A, b, E0, n = o.icp_system()
    assert n > 50 and E0 > 0
    eps = 1e-6
    g = np.zeros(6)
    for i in range(6):
        xi = np.zeros(6)
        for sgn in (1, -1):
            xi[:] = 0
            xi[i] = sgn * eps
            w = xi[:3]
            th = np.linalg.norm(w)
            Kx = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
            Rw = np.eye(3) + (np.sin(th) / th if th else 1.0) * Kx + ((1 - np.cos(th)) / th ** 2 if th else 0.5) * Kx @ Kx
            o.set_pose(_pose(Rw @ P0[:9].reshape(3, 3), P0[9:] + xi[3:]))
            g[i] += sgn * o.icp_system()[2] / (2 * eps)
    assert np.abs(g - 2 * b).max() <= 1e-6 * np.abs(2 * b).max()
    assert np.allclose(A, A.T) and np.all(np.linalg.eigvalsh(A) > 0)


def test_icp_recovers_a_rigid_motion():
    """The observed corner is the canonical one moved by (Q, c): from the identity pose,
    dense projective ICP converges to (Q, c), where every residual vanishes -- up to the
    float32 rounding of the depth map and the samples (about 1e-8 here)."""
    rng = np.random.default_rng(22)
    Q = _rand_rot(rng, 0.012)
    c = np.array([0.004, -0.003, 0.005])
    fr = synth.corner_frame(rot=Q, shift=c)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    it, e = o.icp(8)
    P = o.get_pose()
    assert it == 8 and e[0] > 1e-3 and e[-1] < 1e-12
    assert np.abs(P[:9].reshape(3, 3) - Q).max() < 1e-7
    assert np.abs(P[9:] - c).max() < 1e-7


def test_icp_keeps_the_true_pose():
    """At the true pose the energy is zero (to the float32 rounding of the inputs) and
    a step leaves the pose where it is."""
    fr = synth.corner_frame()
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    it, e = o.icp(2)
    P = o.get_pose()
    assert e[0] < 1e-13
    assert np.abs(P - _pose(np.eye(3), np.zeros(3))).max() < 1e-7


# ---------------------------------------------------------------- source samples (Sec. 4, 5.1)

def _smooth_field(n=24, seed=0):
    """A random smooth field whose zero set is closed and inside the grid."""
    rng = np.random.default_rng(seed)
    ax = np.linspace(-1, 1, n)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    f = x ** 2 + 1.3 * y ** 2 + 0.8 * z ** 2 - 0.45
    for _ in range(4):
        k = rng.normal(0, 3, 3)
        f = f + 0.06 * np.sin(k[0] * x + k[1] * y + k[2] * z + rng.uniform(0, 6))
    return f.astype(np.float32), np.array([-1.0, -1.0, -1.0]), 2.0 / (n - 1)


def _edges_of(tri):
    out = {}
    for t in tri:
        vs = [tuple(v) for v in t]
        for a, b in ((0, 1), (1, 2), (2, 0)):
            out.setdefault(frozenset((vs[a], vs[b])), []).append((vs[a], vs[b]))
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_marching_cubes_closed_oriented_surface(seed):
    """A closed iso-surface inside the grid comes out watertight and consistently
    oriented: every mesh edge belongs to exactly two triangles, which traverse it in
    opposite directions (the face rule resolves a shared ambiguous face the same way in
    both cells)."""
    g, o, hs = _smooth_field(seed=seed)
    tri, _ = oracle.marching_cubes(g, o, hs)
    degenerate = np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1) == 0
    assert len(tri) > 500
    for e, uses in _edges_of(tri[~degenerate] if degenerate.any() else tri).items():
        if len(e) < 2:
            continue
        assert len(uses) == 2 and uses[0] == uses[1][::-1], uses


def test_marching_cubes_sphere_volume_and_outward_normals():
    """Sphere SDF: the mesh encloses 4/3 pi r^3 (divergence theorem, O(h^2) error),
    every face normal (by vertex order) and every vertex normal points outward, and the
    vertices lie on the sphere to O(h^2)."""
    g, o, hs = synth.sdf_grid("sphere", n=64)
    tri, nrm = oracle.marching_cubes(g, o, hs)
    c = np.array([0.0, 0.0, 1.0])
    vol = np.einsum("ij,ij->i", tri[:, 0] - c, np.cross(tri[:, 1] - c, tri[:, 2] - c)).sum() / 6.0
    assert abs(vol - 4.0 / 3.0 * np.pi * 0.3 ** 3) < 0.01 * 4.0 / 3.0 * np.pi * 0.3 ** 3
    fn = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    radial = tri.mean(1) - c
    assert (np.einsum("ij,ij->i", fn, radial) > 0).all()
    assert (np.einsum("ijk,ijk->ij", nrm, tri - c) > 0).all()
    assert np.abs(np.linalg.norm(tri - c, axis=2) - 0.3).max() < 2 * hs ** 2 / 0.3


def test_marching_cubes_linear_field_exact():
    """A linear field's zero set is a plane: every vertex lies on it exactly (linear
    interpolation along the edges is exact), every triangle is parallel to it, and its
    normal is the field's gradient."""
    n = 12
    ax = np.linspace(0, 1, n)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    a = np.array([0.3, -0.5, 0.8])
    g = (a[0] * x + a[1] * y + a[2] * z - 0.2).astype(np.float32)
    tri, nrm = oracle.marching_cubes(g, [0, 0, 0], 1.0 / (n - 1))
    assert len(tri) > 50
    assert np.abs(tri @ a - 0.2).max() < 2e-7          # float32 field values
    fn = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    big = np.linalg.norm(fn, axis=1) > 1e-12        # where the plane passes through a grid node,
    fn = fn[big] / np.linalg.norm(fn[big], axis=1, keepdims=True)   # fans may hold empty triangles
    assert big.sum() > 50
    assert np.abs(fn - a / np.linalg.norm(a)).max() < 1e-5
    assert np.abs(nrm - a / np.linalg.norm(a)).max() < 1e-5


def test_marching_cubes_every_case_separates_corners():
    """For every one of the 256 cases, a cell whose inside corners are at -1 and outside
    ones at +1 gives triangles whose vertices are the midpoints of crossed edges only,
    every crossed edge is used, and each triangle's normal points up the field (toward
    the outside)."""
    corners = np.array([[k & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], np.float64)
    for cs in range(1, 255):
        ins = [(cs >> k) & 1 for k in range(8)]
        g = np.array([[[-1.0 if ins[x + 2 * y + 4 * z] else 1.0 for x in range(2)] for y in range(2)]
                      for z in range(2)], np.float32)
        tri, _ = oracle.marching_cubes(g, [0, 0, 0], 1.0)
        mids = {tuple((corners[a] + corners[b]) / 2) for a in range(8) for b in range(a + 1, 8)
                if np.abs(corners[a] - corners[b]).sum() == 1 and ins[a] != ins[b]}
        used = {tuple(v) for t in tri for v in t}
        assert used == mids, cs
        # the face normal points up the trilinear field's gradient at the centroid
        vals = np.array([-1.0 if ins[k] else 1.0 for k in range(8)])
        fn = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
        for t, n_ in zip(tri, fn):
            x, y, z = t.mean(0)
            wts = lambda k: ((x if k & 1 else 1 - x), (y if k & 2 else 1 - y), (z if k & 4 else 1 - z))
            grad = np.zeros(3)
            for k in range(8):
                wx, wy, wz = wts(k)
                sx, sy, sz = (1 if k & 1 else -1), (1 if k & 2 else -1), (1 if k & 4 else -1)
                grad += vals[k] * np.array([sx * wy * wz, wx * sy * wz, wx * wy * sz])
            assert n_ @ grad > 0, cs


def test_raster_single_triangle_by_hand():
    """One triangle facing the camera at depth 1: the covered pixels are exactly those
    whose centres have non-negative barycentric coordinates, the depth is 1, and each
    sample is the back-projected pixel centre (identity warp and pose)."""
    fr = synth.plane_frame(W=40, H=30, f=30.0, n=4)
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    tri = np.array([[[-0.3, -0.2, 1.0], [0.35, -0.1, 1.0], [0.0, 0.33, 1.0]]])
    nrm = np.tile([0.0, 0.0, -1.0], (1, 3, 1))
    K = np.array([30.0, 30.0, 19.5, 14.5])
    r = oracle.render_samples(o, tri, nrm, 40, 30, K)
    X = 30.0 * tri[0, :, 0] + 19.5
    Y = 30.0 * tri[0, :, 1] + 14.5
    v, u = np.mgrid[0:30, 0:40]
    area = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0])
    lam = [((X[(j + 2) % 3] - X[(j + 1) % 3]) * (v - Y[(j + 1) % 3]) - (Y[(j + 2) % 3] - Y[(j + 1) % 3]) *
            (u - X[(j + 1) % 3])) / area for j in range(3)]
    inside = (lam[0] >= 0) & (lam[1] >= 0) & (lam[2] >= 0)
    assert np.array_equal(r["win"] == 0, inside) and inside.sum() > 50
    assert np.abs(r["depth"][inside] - 1.0).max() < 1e-12
    ray = np.stack([(u - 19.5) / 30.0, (v - 14.5) / 30.0, np.ones_like(u, float)], -1)
    assert np.abs(r["point"][inside] - ray[inside]).max() < 1e-12


def test_raster_sphere_samples_on_rays_and_surface():
    """The sphere mesh rendered with an identity warp: every sample lies on its pixel's
    ray, on the sphere's front half to O(h^2), with an outward normal facing the camera;
    the covered pixels are those of the sphere's projected disk (up to a pixel at its
    rim).  With a translation warp u = d on every node, S(p^) = p^ + d is on the ray."""
    g, og, hs = synth.sdf_grid("sphere", n=48)
    tri, nrm = oracle.marching_cubes(g, og, hs)
    fr = synth.config1()
    o = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    K = fr.K.astype(np.float64)
    r = oracle.render_samples(o, tri, nrm, fr.W, fr.H, K)
    cov = r["win"] >= 0
    v, u = np.mgrid[0:fr.H, 0:fr.W]
    ray = np.stack([(u - K[2]) / K[0], (v - K[3]) / K[1], np.ones_like(u, float)], -1)
    p = r["point"][cov]
    assert np.abs(np.cross(p, ray[cov])).max() < 1e-12
    c = np.array([0.0, 0.0, 1.0])
    assert np.abs(np.linalg.norm(p - c, axis=1) - 0.3).max() < 2 * hs ** 2 / 0.3
    assert (p[:, 2] < 1.0 + 1e-9).all() and (np.einsum("ij,ij->i", r["normal"][cov], ray[cov]) < 0).all()
    rd = ray / np.linalg.norm(ray, axis=-1, keepdims=True)
    miss = np.linalg.norm(np.cross(rd, c), axis=-1)          # ray's distance from the centre
    assert cov[miss < 0.3 - 0.02].all() and not cov[miss > 0.3 + 0.02].any()
    d = np.array([0.01, -0.02, 0.015])
    o.set_warp(np.tile(d, (o.nn, 1)))
    r2 = oracle.render_samples(o, tri, nrm, fr.W, fr.H, K)
    cov2 = r2["win"] >= 0
    assert np.abs(np.cross(r2["point"][cov2] + d, ray[cov2])).max() < 1e-12
