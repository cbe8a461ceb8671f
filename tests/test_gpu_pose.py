"""Global rigid pose by dense projective ICP (vd_estimate_pose, Sec. 6) against the FP64
oracle's ICP on the same frames.

The pose is carried in FP64 on both sides between steps; the GPU associates and sums in
FP32 (decisions re-taken in FP64 near a threshold) with FP64 accumulation across warps,
so the poses agree to a few 1e-7 (rotation entries, metres), far below what a wrong sign
or a dropped term in the 6 x 6 system gives (the step itself, ~1e-2)."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_1603_08161_b300 import synth

pytestmark = pytest.mark.gpu

POSE_TOL = 1e-6


@pytest.fixture(scope="module")
def vd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1603_08161_b300 import vd as mod
    return mod


def _rot(axis, angle):
    k = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * Kx + (1 - math.cos(angle)) * Kx @ Kx


def _pair(vd, fr, mode="all"):
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL if mode == "all" else vd.VD_ACTIVE_SURFACE)
    lat.set_frame_from(fr)
    ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
    return lat, ref


def test_icp_recovers_rigid_motion_like_the_oracle(vd):
    Q = _rot([0.3, -0.5, 0.8], 0.012)
    c = np.array([0.004, -0.003, 0.005])
    fr = synth.corner_frame(rot=Q, shift=c)
    lat, ref = _pair(vd, fr)
    pose, steps, e = lat.estimate_pose(vd.params(), 8)
    it0, e0 = ref.icp(8)
    P0 = ref.get_pose()
    print(f"corner ICP: gpu |dR| {np.abs(pose[:9].reshape(3, 3) - Q).max():.2e} |dt| {np.abs(pose[9:] - c).max():.2e}; "
          f"vs oracle {np.abs(pose - P0).max():.2e}; E {e[:3]} vs {e0[:3]}")
    assert steps == it0 == 8
    assert np.abs(pose - P0).max() < POSE_TOL
    assert np.abs(pose[:9].reshape(3, 3) - Q).max() < POSE_TOL and np.abs(pose[9:] - c).max() < POSE_TOL
    assert abs(e[0] - e0[0]) <= 1e-4 * e0[0] and abs(e[1] - e0[1]) <= 1e-2 * e0[1]


@pytest.mark.parametrize("name", ["cfg1", "ragged", "capsules"])
def test_icp_on_deforming_surfaces_matches_oracle(vd, name):
    """No known truth (the surface deforms): from the frame's identity pose and a non-zero
    lattice warp, both sides take the same steps to the same pose, and the solve that
    follows (at the estimated pose) matches the oracle's solve at its pose."""
    fr = {"cfg1": synth.config1(),
          "ragged": synth.sphere_frame(W=53, H=37, f=50.0, n=(13, 11, 9), seed=3, n_sparse=7),
          "capsules": synth.capsule_frame(W=160, H=120, f=131.25, n=24, seed=5, n_sparse=40)}[name]
    lat, ref = _pair(vd, fr)
    rng = np.random.default_rng(4)
    u = rng.normal(0, 0.002, (lat.nn, 3)).astype(np.float32)
    lat.set_warp(u, None)
    ref.set_warp(u.astype(np.float64), None)
    pose, steps, e = lat.estimate_pose(vd.params(), 5)
    it0, e0 = ref.icp(5)
    P0 = ref.get_pose()
    print(f"{name} ICP: steps {steps}, |pose - oracle| {np.abs(pose - P0).max():.2e}, E {e[0]:.4e} -> {e[-1]:.4e}")
    assert steps == it0
    assert np.abs(pose - P0).max() < POSE_TOL
    # the solve at the estimated pose
    prm = vd.params(gn_iters=3, cg_iters=10, fixed_association=True)
    rep = lat.solve(prm)
    res = ref.solve(3, 10, fixed_association=True)
    ug, _ = lat.get_warp()
    uo, _ = ref.get_warp()
    pix, _, _ = lat.association(prm)
    pix0, _, _ = ref.association()
    assert (pix == pix0).all()
    assert np.abs(ug - uo).max() <= 1e-4 * fr.spacing
    assert abs(rep["e_total"] - res["energy"][-1, 0]) <= 1e-5 * res["energy"][-1, 0]


def test_icp_without_correspondences_keeps_the_pose(vd):
    fr = dataclasses.replace(synth.config1(), depth=np.zeros_like(synth.config1().depth))
    lat, ref = _pair(vd, fr)
    pose, steps, _ = lat.estimate_pose(vd.params(), 4)
    assert steps == 0 == ref.icp(4)[0]
    assert np.array_equal(pose, fr.pose)
