"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances:
  * integer decisions (target pixel of each sample, active set, validity): bit-exact;
  * per-node displacement after a solve: |u_gpu - u_oracle|_inf <= 1e-4 h, and final
    energy |E_gpu - E_oracle| / E_oracle <= 1e-5 (the stated goal for configs 1-2, in
    the fixed-association parity mode);
  * single stages (b, diag, J^T J p, rotations, energies, w_c): FP32 storage and
    accumulation over at most a few hundred terms against FP64 gives relative errors
    of a few 1e-7 of the largest term; the checks use 2e-5 of the array's scale.
"""
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


def _pair(vd, fr, mode, params=None):
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL if mode == "all" else vd.VD_ACTIVE_SURFACE)
    lat.set_frame_from(fr)
    ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE,
                                   params=params)
    return lat, ref


def _rand_warp(rng, nn, su=0.004, sr=0.05):
    u = rng.normal(0, su, (nn, 3)).astype(np.float32)
    w = rng.normal(0, sr, (nn, 3))
    R = np.zeros((nn, 3, 3))
    for i in range(nn):
        th = np.linalg.norm(w[i])
        k = w[i] / th
        Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R[i] = np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx
    return u, R.astype(np.float32)


def _scale_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30))


def _frames():
    return {"cfg1": synth.config1(),
            "ragged": synth.sphere_frame(W=53, H=37, f=50.0, n=(13, 11, 9), seed=3, n_sparse=7, name="ragged")}


FRAMES = _frames()


# ------------------------------------------------------------------ frame stage

@pytest.mark.parametrize("name", ["cfg1", "ragged"])
def test_target_normals(vd, name):
    fr = FRAMES[name]
    lat, ref = _pair(vd, fr, "all")
    _, N, valid = ref.target_maps()
    g = lat.target_normals()
    gv = np.abs(g).sum(-1) > 0
    assert (gv == valid).all()
    assert np.abs(g[valid] - N[valid]).max() < 2e-6


@pytest.mark.parametrize("name", ["cfg1", "ragged"])
def test_active_set(vd, name):
    fr = FRAMES[name]
    lat, ref = _pair(vd, fr, "surface")
    m = ref.active_mask()
    assert lat.num_active() == ref.num_active() == int(m.sum())
    assert (lat.active_mask() == m).all()


# ------------------------------------------------------------------ Gauss-Newton stages

@pytest.mark.parametrize("mode", ["all", "surface"])
@pytest.mark.parametrize("name", ["cfg1", "ragged"])
@pytest.mark.parametrize("warped", [False, True])
def test_association(vd, mode, name, warped):
    fr = FRAMES[name]
    lat, ref = _pair(vd, fr, mode)
    prm = vd.params()
    if warped:
        u, R = _rand_warp(np.random.default_rng(1), lat.nn)
        lat.set_warp(u, R)
        ref.set_warp(u.astype(np.float64), R.astype(np.float64))
    lat.associate(prm)
    ref.associate()
    pix, w, r = lat.association(prm)
    pix0, w0, r0 = ref.association()
    assert (pix == pix0).all(), f"{int((pix != pix0).sum())} target pixels differ"
    assert ((w > 0) == (w0 > 0)).all()
    assert np.abs(w - w0).max() < 1e-5
    assert np.abs(r - r0).max() < 1e-6 + STAGE_RTOL * np.abs(r0).max()


@pytest.mark.parametrize("mode", ["all", "surface"])
@pytest.mark.parametrize("name", ["cfg1", "ragged"])
def test_rhs_and_diag(vd, mode, name):
    fr = FRAMES[name]
    lat, ref = _pair(vd, fr, mode)
    prm = vd.params()
    u, R = _rand_warp(np.random.default_rng(2), lat.nn)
    lat.set_warp(u, R)
    ref.set_warp(u.astype(np.float64), R.astype(np.float64))
    lat.associate(prm)
    ref.associate()
    b, d = lat.rhs(prm)
    b0, d0 = ref.rhs()
    assert _scale_err(b, b0) < STAGE_RTOL
    assert _scale_err(d, d0) < STAGE_RTOL


@pytest.mark.parametrize("mode", ["all", "surface"])
@pytest.mark.parametrize("name", ["cfg1", "ragged"])
def test_apply_JtJ(vd, mode, name):
    fr = FRAMES[name]
    lat, ref = _pair(vd, fr, mode)
    prm = vd.params()
    lat.associate(prm)
    ref.associate()
    p = np.random.default_rng(3).normal(0, 1e-2, (lat.nn, 3)).astype(np.float32)
    q, pq = lat.apply(prm, p)
    q0 = ref.apply(p.astype(np.float64))
    m = ref.active_mask()
    assert _scale_err(q, q0) < STAGE_RTOL
    pq0 = float((p.astype(np.float64)[m] * q0[m]).sum())
    assert abs(pq - pq0) / abs(pq0) < 1e-5


@pytest.mark.parametrize("mode", ["all", "surface"])
@pytest.mark.parametrize("name", ["cfg1", "ragged"])
def test_fit_rotations_and_energy(vd, mode, name):
    fr = FRAMES[name]
    lat, ref = _pair(vd, fr, mode)
    prm = vd.params()
    u, R = _rand_warp(np.random.default_rng(4), lat.nn, su=0.01)
    lat.set_warp(u, R)
    ref.set_warp(u.astype(np.float64), R.astype(np.float64))
    lat.associate(prm)
    ref.associate()
    e = lat.energy(prm)
    e0 = ref.energy()
    np.testing.assert_allclose(e, e0, rtol=1e-5)
    nd = lat.fit_rotations()
    nd0 = ref.fit_rotations()
    assert nd == nd0
    _, Rg = lat.get_warp()
    _, R0 = ref.get_warp()
    m = ref.active_mask()
    assert np.abs(Rg[m] - R0[m]).max() < 1e-5
    assert np.abs(np.einsum("nij,nkj->nik", Rg[m], Rg[m]) - np.eye(3)).max() < 1e-5
    np.testing.assert_allclose(lat.energy(prm), ref.energy(), rtol=1e-5)


def _rand_warp_fast(rng, nn, su, sr):
    """_rand_warp without the per-node loop (Rodrigues' formula on all nodes at once)."""
    u = rng.normal(0, su, (nn, 3)).astype(np.float32)
    w = rng.normal(0, sr, (nn, 3))
    th = np.linalg.norm(w, axis=1)
    k = w / th[:, None]
    K = np.zeros((nn, 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -k[:, 2], k[:, 1], -k[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = k[:, 2], -k[:, 1], k[:, 0]
    R = np.eye(3) + np.sin(th)[:, None, None] * K + (1 - np.cos(th))[:, None, None] * (K @ K)
    return u, R.astype(np.float32)


def test_rotation_step_many_batches_per_cta(vd):
    """The rotation step of an all-nodes lattice stages 128 nodes per batch; at 47 x 45 x
    43 = 90,945 nodes the 592 CTAs take 711 batches, the last one 65 nodes long, so CTAs
    run the two-stage copy pipeline over more than one batch and the ragged end.
    Rotations (Sec. 7.1), the count of nodes that keep theirs, and E_reg (Eq. 4) against
    the oracle's rotation step on the same warp."""
    fr = synth.sphere_frame(W=64, H=48, f=60.0, n=(47, 45, 43), seed=11, n_sparse=5, name="many-batches")
    lat, ref = _pair(vd, fr, "all")
    prm = vd.params()
    assert lat.nn == 90945 and lat.nn % 128 == 65
    h = fr.spacing
    for call, (su, sr) in enumerate([(0.1 * h, 0.1), (0.05 * h, 0.4)]):
        u, R = _rand_warp_fast(np.random.default_rng(500 + call), lat.nn, su, sr)
        lat.set_warp(u, R)
        ref.set_warp(u.astype(np.float64), R.astype(np.float64))
        lat.associate(prm)
        ref.associate()
        assert lat.fit_rotations() == ref.fit_rotations()
        _, Rg = lat.get_warp()
        _, R0 = ref.get_warp()
        err = np.abs(Rg - R0).max()
        assert err < 1e-5, f"call {call}: rotation error {err:.3e}"
        e, e0 = lat.energy(prm), ref.energy()
        assert abs(e[3] - e0[3]) <= 1e-5 * e0[3], f"call {call}: E_reg {e[3]} vs {e0[3]}"


@pytest.mark.parametrize("mode", ["all", "surface"])
def test_pcg_position_step(vd, mode):
    fr = FRAMES["cfg1"]
    lat, ref = _pair(vd, fr, mode)
    prm = vd.params(cg_iters=10)
    lat.associate(prm)
    ref.associate()
    x, it = lat.pcg(prm)
    x0, it0, _ = ref.pcg(10)
    assert it == it0 == 10
    assert np.abs(x - x0).max() < 1e-5 * fr.spacing + 1e-5 * np.abs(x0).max()


# ------------------------------------------------------------------ full solves

def _solve_pair(vd, fr, mode, gn, cg, fixed=True, params=None):
    lat, ref = _pair(vd, fr, mode, params=params)
    kw = params or {}
    prm = vd.params(gn_iters=gn, cg_iters=cg, fixed_association=fixed, init=vd.VD_INIT_ZERO, **kw)
    rep = lat.solve(prm)
    res = ref.solve(gn, cg, fixed_association=fixed)
    u, R = lat.get_warp()
    u0, R0 = ref.get_warp()
    return lat, ref, rep, res, u, u0, R, R0


@pytest.mark.parametrize("mode", ["all", "surface"])
@pytest.mark.parametrize("name", ["cfg1", "ragged"])
def test_solve_parity_fixed_association(vd, mode, name):
    fr = FRAMES[name]
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, mode, 5, 10)
    assert rep["gn_done"] == 5 and rep["cg_done"] == int(res["cg_done"][-1])
    assert np.abs(u - u0).max() <= 1e-4 * fr.spacing
    e0 = res["energy"][-1]
    assert abs(rep["e_total"] - e0[0]) / e0[0] <= 1e-5
    assert rep["n_valid_corr"] == res["n_valid"]
    assert rep["n_degenerate_rot"] == res["n_degenerate"]


@pytest.mark.parametrize("mode", ["all", "surface"])
def test_solve_free_association(vd, mode):
    """Re-association every iteration: the decisions are taken on slightly different
    warps (FP32 vs FP64 iterates), so a handful of correspondences may differ; the
    count is reported and must stay tiny, and the warp stays within tolerance when
    none differs."""
    fr = FRAMES["cfg1"]
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, mode, 5, 10, fixed=False)
    prm = vd.params()
    pix, _, _ = lat.association(prm)
    pix0, _, _ = ref.association()
    ndiff = int((pix != pix0).sum())
    print(f"free association: {ndiff} of {fr.C} target pixels differ")
    assert ndiff <= max(2, fr.C // 1000)
    if ndiff == 0:
        assert np.abs(u - u0).max() <= 1e-4 * fr.spacing
        assert abs(rep["e_total"] - res["energy"][-1, 0]) / res["energy"][-1, 0] <= 1e-5


@pytest.mark.parametrize("n,bricks", [(32, "2x4 rows of 32"), (48, "4x4 rows of 48")])
def test_solve_parity_brick_partition(vd, n, bricks):
    """All-nodes lattices whose persistent position step splits the slots into bricks
    of full x-rows with neighbours in other CTAs along y and z (the host's plan for
    these sizes on 148 SMs is noted); same tolerance as the other solves."""
    fr = synth.sphere_frame(W=96, H=72, f=90.0, n=n, seed=6, n_sparse=40, name=f"sphere{n}")
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, "all", 3, 10)
    assert rep["gn_done"] == 3 and rep["cg_done"] == int(res["cg_done"][-1])
    assert np.abs(u - u0).max() <= 1e-4 * fr.spacing
    e0 = res["energy"][-1]
    assert abs(rep["e_total"] - e0[0]) / e0[0] <= 1e-5


@pytest.mark.parametrize("n", [69, (75, 62, 66), 92, 93])
def test_solve_parity_padded_bricks(vd, n):
    """All-nodes lattices whose bricks are padded: nx % 4 != 0 (rows held as a multiple
    of 4 slots in shared memory, the padding kept at zero; the global vectors read and
    written element by element) and / or ny, nz that the brick does not divide (ragged
    bricks at the far faces); same tolerance as the other solves, and the plan is the
    padded one (lattices of at least 2,048 slots per SM)."""
    fr = synth.capsule_frame(W=320, H=240, f=262.5, n=n, seed=11, n_sparse=60, name=f"capsules{n}")
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, "all", 3, 10)
    plan = lat.pcg_plan()
    print(f"{fr.dims}: plan {plan}, |du|max = {np.abs(u - u0).max() / fr.spacing:.2e} h")
    assert plan["padded"] == 1 and plan["by"] > 0
    assert rep["gn_done"] == 3 and rep["cg_done"] == int(res["cg_done"][-1])
    assert np.abs(u - u0).max() <= 1e-4 * fr.spacing
    assert np.abs(R - R0).max() <= 1e-4
    e0 = res["energy"][-1]
    assert abs(rep["e_total"] - e0[0]) / e0[0] <= 1e-5


def test_solve_parity_config2_surface(vd, cfg2):
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, cfg2, "surface", 10, 20)
    assert np.abs(u - u0).max() <= 1e-4 * cfg2.spacing
    assert abs(rep["e_total"] - res["energy"][-1, 0]) / res["energy"][-1, 0] <= 1e-5


_CFG2_ORACLE = {}


def _cfg2_oracle(cfg2):
    """The FP64 oracle's fixed-association 10 x 20 solve of the 96^3 frame (cached)."""
    if "res" not in _CFG2_ORACLE:
        ref = oracle.Oracle.from_frame(cfg2, oracle.ACTIVE_ALL)
        res = ref.solve(10, 20, fixed_association=True)
        u0, R0 = ref.get_warp()
        _CFG2_ORACLE.update(res=res, u0=u0)
    return _CFG2_ORACLE["res"], _CFG2_ORACLE["u0"]


@pytest.mark.slow
def test_solve_parity_config2_all(vd, cfg2):
    """96^3 lattice, 640x480 depth, 10 x 20 schedule: the benchmark's workload."""
    res, u0 = _cfg2_oracle(cfg2)
    lat = vd.Lattice(cfg2.dims, cfg2.origin, cfg2.spacing, vd.VD_ACTIVE_ALL)
    lat.set_frame_from(cfg2)
    rep = lat.solve(vd.params(gn_iters=10, cg_iters=20, fixed_association=True, init=vd.VD_INIT_ZERO))
    u, _ = lat.get_warp()
    err = float(np.abs(u - u0).max())
    rel = abs(rep["e_total"] - res["energy"][-1, 0]) / res["energy"][-1, 0]
    print(f"config 2 all-nodes FP32: |du|max = {err:.3e} m (tol {1e-4 * cfg2.spacing:.3e}), dE/E = {rel:.3e}")
    assert err <= 1e-4 * cfg2.spacing
    assert rel <= 1e-5


_CFG2_FREE = {}


def _cfg2_oracle_free(cfg2, gn=10, cg=20):
    """The oracle's 10 x 20 solve of the 96^3 frame with re-association at every
    iteration, stage by stage in the order of Sec. 7.1 (the same as vdo_solve, pinned by
    test_solve_is_the_stages_in_the_papers_order), keeping each iteration's target
    pixels (cached)."""
    if not _CFG2_FREE:
        ref = oracle.Oracle.from_frame(cfg2, oracle.ACTIVE_ALL)
        pix = []
        for g in range(gn):
            ref.associate()
            pix.append(ref.association()[0])
            x, _, _ = ref.pcg(cg)
            ref.add_increment(x)
            ref.fit_rotations()
        u0, _ = ref.get_warp()
        _CFG2_FREE.update(pix=pix, e=ref.energy(), u0=u0)
    return _CFG2_FREE


@pytest.mark.slow
def test_solve_parity_config2_free_association(vd, cfg2):
    """The benchmark's own mode: 96^3 lattice, 640x480 depth, 10 x 20, re-associated at
    every iteration.  For each iteration g the GPU solve of g + 1 iterations is stopped
    and its association (taken at the start of iteration g) compared pixel by pixel with
    the oracle's; the count of differing target pixels is printed per iteration and must
    stay tiny, and the final warp and energy must meet the parity tolerances."""
    ref = _cfg2_oracle_free(cfg2)
    lat = vd.Lattice(cfg2.dims, cfg2.origin, cfg2.spacing, vd.VD_ACTIVE_ALL)
    lat.set_frame_from(cfg2)
    diffs = []
    for g in range(10):
        prm = vd.params(gn_iters=g + 1, cg_iters=20, fixed_association=False, init=vd.VD_INIT_ZERO)
        rep = lat.solve(prm)
        pix, _, _ = lat.association(prm)
        diffs.append(int((pix != ref["pix"][g]).sum()))
    u, _ = lat.get_warp()
    err = float(np.abs(u - ref["u0"]).max())
    rel = abs(rep["e_total"] - ref["e"][0]) / ref["e"][0]
    print(f"config 2 free association: differing target pixels per iteration {diffs} of {cfg2.C}; "
          f"|du|max = {err:.3e} m (tol {1e-4 * cfg2.spacing:.3e}), dE/E = {rel:.3e}")
    assert max(diffs) <= max(2, cfg2.C // 1000)
    assert err <= 1e-4 * cfg2.spacing
    assert rel <= 1e-5


# ------------------------------------------------------------------ precision variant

def _mixed_vs_oracle(vd, fr, mode, gn, cg, res=None, u0=None):
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing,
                     vd.VD_ACTIVE_ALL if mode == "all" else vd.VD_ACTIVE_SURFACE, vd.VD_PREC_MIXED)
    lat.set_frame_from(fr)
    prm = vd.params(gn_iters=gn, cg_iters=cg, fixed_association=True, init=vd.VD_INIT_ZERO)
    if res is None:
        ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
        ref.associate()
        pix0, _, _ = ref.association()
        lat.associate(prm)
        pix, _, _ = lat.association(prm)
        assert (pix == pix0).all()          # decisions are still taken in FP64 near thresholds
        res = ref.solve(gn, cg, fixed_association=True)
        u0, _ = ref.get_warp()
    rep = lat.solve(prm)
    u, _ = lat.get_warp()
    err = float(np.abs(u - u0).max())
    rel = abs(rep["e_total"] - res["energy"][-1, 0]) / res["energy"][-1, 0]
    return err, rel, rep, res


@pytest.mark.parametrize("mode", ["all", "surface"])
def test_precision_variant_config1(vd, mode):
    """BF16 storage of target normals and per-sample records, FP32 stencil and
    accumulation: the error against the FP64 oracle is stated and bounded."""
    fr = FRAMES["cfg1"]
    err, rel, rep, res = _mixed_vs_oracle(vd, fr, mode, 5, 10)
    print(f"mixed precision, config 1 {mode}: |du|max = {err:.3e} m = {err / fr.spacing:.2e} h, dE/E = {rel:.3e}")
    assert rep["n_valid_corr"] == res["n_valid"]
    assert err <= 1e-2 * fr.spacing
    assert rel <= 1e-2
    assert err > 0.0                      # the BF16 records are really used


@pytest.mark.slow
def test_precision_variant_config2(vd, cfg2):
    res, u0 = _cfg2_oracle(cfg2)
    err, rel, rep, _ = _mixed_vs_oracle(vd, cfg2, "all", 10, 20, res=res, u0=u0)
    print(f"mixed precision, config 2 all-nodes: |du|max = {err:.3e} m = {err / cfg2.spacing:.2e} h, dE/E = {rel:.3e}")
    assert rep["n_valid_corr"] == res["n_valid"]
    assert err <= 1e-2 * cfg2.spacing
    assert rel <= 1e-2


# ------------------------------------------------------------------ edge cases

def test_arap_only_stays_at_rest(vd):
    fr = FRAMES["cfg1"]
    kw = dict(w_sparse=0.0, w_dense=0.0)
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, "all", 3, 10, params=kw)
    assert rep["cg_done"] == 0 and np.abs(u).max() == 0.0
    assert np.abs(R - np.eye(3)).max() == 0.0


def test_no_dense_samples_sparse_only(vd):
    fr = dataclasses.replace(FRAMES["cfg1"], src_pts=np.zeros((0, 3), np.float32),
                             src_nrm=np.zeros((0, 3), np.float32))
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, "surface", 3, 10)
    assert np.abs(u - u0).max() <= 1e-4 * fr.spacing
    assert rep["n_valid_corr"] == 0


def test_empty_depth_and_no_pairs(vd):
    fr = dataclasses.replace(FRAMES["cfg1"], depth=np.zeros_like(FRAMES["cfg1"].depth),
                             sp_canon=np.zeros((0, 3), np.float32), sp_target=np.zeros((0, 3), np.float32))
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, "all", 2, 5)
    assert rep["n_valid_corr"] == 0 and rep["cg_done"] == 0
    assert np.abs(u).max() == 0.0 and rep["e_total"] == 0.0


def test_samples_outside_lattice(vd):
    fr = FRAMES["cfg1"]
    out = fr.src_pts + np.float32([5.0, 0, 0])
    fr2 = dataclasses.replace(fr, src_pts=np.concatenate([fr.src_pts, out]),
                              src_nrm=np.concatenate([fr.src_nrm, fr.src_nrm]))
    lat, ref = _pair(vd, fr2, "all")
    prm = vd.params()
    lat.associate(prm)
    ref.associate()
    pix, w, _ = lat.association(prm)
    pix0, w0, _ = ref.association()
    assert (pix == pix0).all() and (pix[fr.C:] == -1).all() and (w[fr.C:] == 0).all()


def _non_finite_frame(fr, seed=7):
    """fr with NaN / +inf / -inf depth pixels on the surface, samples with a NaN or
    infinite position or normal, and one sparse pair with a NaN canonical position."""
    rng = np.random.default_rng(seed)
    on = np.argwhere(fr.depth > 0)
    pick = on[rng.choice(len(on), 12, replace=False)]
    depth = fr.depth.copy()
    depth[pick[:6, 0], pick[:6, 1]] = np.nan
    depth[pick[6:9, 0], pick[6:9, 1]] = np.inf
    depth[pick[9:, 0], pick[9:, 1]] = -np.inf
    pts, nrm = fr.src_pts.copy(), fr.src_nrm.copy()
    pts[5] = np.nan
    pts[17, 1] = np.inf
    nrm[23] = np.nan
    nrm[31, 2] = -np.inf
    nrm[40, 0] = np.inf
    fh = fr.sp_canon.copy()
    fh[3, 1] = np.nan
    return dataclasses.replace(fr, depth=depth, src_pts=pts, src_nrm=nrm, sp_canon=fh), [5, 17, 23, 31, 40]


@pytest.mark.parametrize("mode", ["all", "surface"])
def test_non_finite_inputs_treated_as_invalid(vd, mode):
    """Non-finite depth pixels are invalid and samples or pairs with a non-finite
    canonical position or normal are ignored, exactly as the oracle takes them: the
    validity map, the active set and the target pixels are bit-exact, the solve within
    the parity tolerances."""
    fr, bad = _non_finite_frame(FRAMES["cfg1"])
    lat, ref = _pair(vd, fr, mode)
    _, N, valid = ref.target_maps()
    g = lat.target_normals()
    assert ((np.abs(g).sum(-1) > 0) == valid).all()
    assert np.abs(g[valid] - N[valid]).max() < 2e-6
    assert (lat.active_mask() == ref.active_mask()).all()
    prm = vd.params()
    lat.associate(prm)
    ref.associate()
    pix, w, _ = lat.association(prm)
    pix0, w0, _ = ref.association()
    assert (pix == pix0).all() and (pix[bad] == -1).all() and (w[bad] == 0).all()
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, mode, 3, 10)
    assert rep["status"] == vd.VD_OK and np.isfinite(u).all()
    assert np.abs(u - u0).max() <= 1e-4 * fr.spacing
    assert abs(rep["e_total"] - res["energy"][-1, 0]) / res["energy"][-1, 0] <= 1e-5


def test_non_finite_target_reports_numeric_error(vd):
    """A sparse pair whose observed position is NaN makes E_sparse non-finite (the
    oracle's energy is NaN too): the solve returns VD_ERR_NUMERIC, and the lattice,
    reset by a zero-initialised solve of a clean frame, solves normally again."""
    fr = FRAMES["cfg1"]
    ft = fr.sp_target.copy()
    ft[2, 0] = np.nan
    bad = dataclasses.replace(fr, sp_target=ft)
    ref = oracle.Oracle.from_frame(bad, oracle.ACTIVE_ALL)
    assert not np.isfinite(ref.solve(2, 10)["energy"][-1, 0])
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL)
    lat.set_frame_from(bad)
    prm = vd.params(gn_iters=2, cg_iters=10, fixed_association=True, init=vd.VD_INIT_ZERO)
    rep = lat.solve(prm)
    assert rep["status"] == vd.VD_ERR_NUMERIC
    lat.set_frame_from(fr)
    rep = lat.solve(prm)
    assert rep["status"] == vd.VD_OK
    ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL)
    res = ref.solve(2, 10, fixed_association=True)
    u, _ = lat.get_warp()
    u0, _ = ref.get_warp()
    assert np.abs(u - u0).max() <= 1e-4 * fr.spacing


def test_smallest_lattice(vd):
    """One cell (2x2x2), one sparse pair: the exact step moves every node by d."""
    fr = synth.plane_frame(W=8, H=6, f=6.0, n=2)
    fr = dataclasses.replace(fr, src_pts=np.zeros((0, 3), np.float32), src_nrm=np.zeros((0, 3), np.float32),
                             sp_canon=np.float32([[0.0, 0.0, 1.0]]), sp_target=np.float32([[0.01, -0.02, 1.03]]))
    lat, ref, rep, res, u, u0, R, R0 = _solve_pair(vd, fr, "all", 2, 24)
    assert np.abs(u - u0).max() <= 1e-4 * fr.spacing


def test_errors_and_state(vd):
    fr = FRAMES["cfg1"]
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing)
    with pytest.raises(vd.VDError) as e:
        lat.solve(vd.params())
    assert e.value.status == vd.VD_ERR_STATE
    lat.set_frame_from(fr)
    with pytest.raises(vd.VDError) as e:
        lat.solve(vd.params(gn_iters=0))
    assert e.value.status == vd.VD_ERR_INVALID_ARG
    u, R = _rand_warp(np.random.default_rng(5), lat.nn)
    lat.set_warp(u, R)
    u2, R2 = lat.get_warp()
    assert (u2 == u).all() and (R2 == R).all()


def test_device_pointers_and_async(vd):
    import torch
    fr = FRAMES["cfg1"]
    prm = vd.params(gn_iters=3, cg_iters=8, fixed_association=True, init=vd.VD_INIT_ZERO)
    a = vd.Lattice(fr.dims, fr.origin, fr.spacing)
    a.set_frame_from(fr)
    ra = a.solve(prm)
    b = vd.Lattice(fr.dims, fr.origin, fr.spacing)
    b.set_frame_from(fr, device="cuda:0")
    b.solve_async(prm)
    rb = b.report()
    for k in ("gn_done", "cg_done", "n_valid_corr", "n_degenerate_rot", "status"):
        assert ra[k] == rb[k]
    assert abs(ra["e_total"] - rb["e_total"]) <= 1e-6 * ra["e_total"]
    ud = torch.zeros((b.nn, 3), dtype=torch.float32, device="cuda:0")
    Rd = torch.zeros((b.nn, 9), dtype=torch.float32, device="cuda:0")
    b.get_warp(ud, Rd)
    ua, _ = a.get_warp()
    assert np.abs(ud.cpu().numpy() - ua).max() <= 1e-6 * fr.spacing
    per_solve, per_frame = b.launch_counts(prm)
    # persistent position step: assoc once + 3 x (rhs 2, pcg 1, rotation 1, energy 1) + report
    # + reset; streamed position step: 4 launches per PCG iteration instead of the 1
    assert per_solve in (1 + 3 * 5 + 1 + 1, 1 + 3 * (3 + 4 * 8 + 3) + 1 + 1) and per_frame > 0


def test_get_warp_async_matches_get_warp(vd):
    """vd_get_warp_async (readback overlapped with the next frame's work) delivers the
    same warp as vd_get_warp: into page-locked host buffers and device buffers, u alone
    and u with R, over consecutive frames (the readback buffer reused while the next
    solve runs)."""
    import torch
    fr = FRAMES["ragged"]
    prm = vd.params(gn_iters=2, cg_iters=6, fixed_association=True)
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing)
    lat.set_frame_from(fr)
    host = [torch.empty((lat.nn, 3), dtype=torch.float32).pin_memory() for _ in range(2)]
    hostR = torch.empty((lat.nn, 9), dtype=torch.float32).pin_memory()
    dev = torch.empty((lat.nn, 3), dtype=torch.float32, device="cuda:0")
    got = []
    for k in range(3):
        lat.solve_async(prm)
        lat.report()
        if k < 2:
            lat.get_warp_async(host[k])
        else:
            lat.get_warp_async(dev, None)
        u_ref, R_ref = lat.get_warp()          # the warp of this frame, read synchronously
        got.append(u_ref)
        lat.get_warp_wait()
        out = (host[k] if k < 2 else dev).cpu().numpy()
        assert np.array_equal(out, u_ref)
    assert not np.array_equal(got[0], got[2])  # the warp moved between the frames
    lat.get_warp_async(host[0], hostR)
    lat.get_warp_wait()
    u_ref, R_ref = lat.get_warp()
    assert np.array_equal(host[0].numpy(), u_ref)
    assert np.array_equal(hostR.numpy().reshape(-1, 3, 3), R_ref)
    with pytest.raises(ValueError):
        lat.get_warp_async(host[0], dev)      # host and device outputs mixed
