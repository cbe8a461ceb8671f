"""Cached B^T B apply (VD_APPLY_CACHED, Sec. 7.1) against the oracle's explicit J^T J.

The cached 24 x 24 blocks per occupied cell are the dense samples' part of J^T J summed
in another order, so the apply and the solves must meet the same tolerances as the
matrix-free path: J^T J p within 2e-5 of the array's scale (FP32 sums of at most a few
thousand terms), solves within 1e-4 h per node and 1e-5 relative energy."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1603_08161_b300 import synth

pytestmark = pytest.mark.gpu

STAGE_RTOL = 2e-5


@pytest.fixture(scope="module")
def vd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1603_08161_b300 import vd as mod
    return mod


def _coarse(fr, n):
    """The frame's samples on an n^3 lattice over the same cube: many samples per cell."""
    dims, origin, h = synth.lattice_for(n)
    return dataclasses.replace(fr, dims=dims, origin=origin, spacing=h)


def _frames():
    c1 = synth.config1()
    return {"cfg1": c1, "ragged": synth.sphere_frame(W=53, H=37, f=50.0, n=(13, 11, 9), seed=3, n_sparse=7),
            "cfg1_coarse6": _coarse(c1, 6),
            "caps_coarse12": _coarse(synth.capsule_frame(W=160, H=120, f=131.25, n=24, seed=5, n_sparse=40), 12)}


FRAMES = _frames()


def _lattice(vd, fr, mode, apply_mode):
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL if mode == "all" else vd.VD_ACTIVE_SURFACE)
    lat.set_apply_mode(apply_mode)
    lat.set_frame_from(fr)
    return lat


@pytest.mark.parametrize("mode", ["all", "surface"])
@pytest.mark.parametrize("name", list(FRAMES))
def test_cached_apply_matches_explicit_JtJ(vd, mode, name):
    fr = FRAMES[name]
    lat = _lattice(vd, fr, mode, vd.VD_APPLY_CACHED)
    assert lat.apply_mode() == (vd.VD_APPLY_CACHED, True)
    ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
    prm = vd.params()
    lat.associate(prm)
    ref.associate()
    p = np.random.default_rng(3).normal(0, 1e-2, (lat.nn, 3)).astype(np.float32)
    q, pq = lat.apply(prm, p)
    q0 = ref.apply(p.astype(np.float64))
    m = ref.active_mask()
    assert float(np.abs(q - q0).max() / np.abs(q0).max()) < STAGE_RTOL
    pq0 = float((p.astype(np.float64)[m] * q0[m]).sum())
    assert abs(pq - pq0) / abs(pq0) < 1e-5


@pytest.mark.parametrize("mode", ["all", "surface"])
@pytest.mark.parametrize("name,gn,cg", [("cfg1", 5, 10), ("cfg1_coarse6", 4, 20), ("caps_coarse12", 4, 20)])
@pytest.mark.parametrize("fixed", [True, False])
def test_cached_solve_matches_oracle(vd, mode, name, gn, cg, fixed):
    fr = FRAMES[name]
    lat = _lattice(vd, fr, mode, vd.VD_APPLY_CACHED)
    ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
    res = ref.solve(gn, cg, fixed_association=fixed)
    rep = lat.solve(vd.params(gn_iters=gn, cg_iters=cg, fixed_association=fixed, init=vd.VD_INIT_ZERO))
    u, _ = lat.get_warp()
    u0, _ = ref.get_warp()
    prm = vd.params()
    pix, _, _ = lat.association(prm)
    pix0, _, _ = ref.association()
    err = float(np.abs(u - u0).max())
    rel = abs(rep["e_total"] - res["energy"][-1, 0]) / res["energy"][-1, 0]
    print(f"cached {name} {mode} fixed={fixed}: |du|max {err / fr.spacing:.2e} h, dE/E {rel:.2e}, {int((pix != pix0).sum())} pixels differ")
    assert (pix == pix0).all()
    assert err <= 1e-4 * fr.spacing
    assert rel <= 1e-5


def test_auto_mode_and_tuner(vd):
    fr = FRAMES["caps_coarse12"]
    lat = _lattice(vd, fr, "all", vd.VD_APPLY_AUTO)
    assert lat.apply_mode() == (vd.VD_APPLY_AUTO, True)      # thousands of samples per cell
    fine = _lattice(vd, FRAMES["cfg1"], "all", vd.VD_APPLY_AUTO)
    assert fine.apply_mode() == (vd.VD_APPLY_AUTO, False)   # a few samples per cell
    prm = vd.params(gn_iters=3, cg_iters=10, init=vd.VD_INIT_ZERO)
    mode, (ms_mf, ms_c) = lat.tune_apply(prm)
    print(f"tune_apply 12^3 with {fr.C} samples: matrix-free {ms_mf:.3f} ms, cached {ms_c:.3f} ms -> {mode}")
    assert mode in (vd.VD_APPLY_MATRIX_FREE, vd.VD_APPLY_CACHED) and ms_mf > 0 and ms_c > 0
    assert lat.apply_mode()[0] == mode
    with pytest.raises(vd.VDError):
        lat.set_apply_mode(7)
