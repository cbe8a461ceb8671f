"""Batched solve (vd_batch_*): many independent lattices of uneven size in one graph.

Each lattice of a batch must match the FP64 oracle within the same tolerances as a
single solve (1e-4 h per node, 1e-5 relative energy, fixed association), and match the
lattice's own vd_solve up to FP32 reduction order (the single solve may take the
persistent position step, the batch streams it)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1603_08161_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1603_08161_b300 import vd as mod
    return mod


def _frames():
    return [
        ("all", synth.config1()),
        ("all", synth.sphere_frame(W=53, H=37, f=50.0, n=(13, 11, 9), seed=3, n_sparse=7)),
        ("surface", synth.config1()),
        ("all", synth.capsule_frame(W=160, H=120, f=131.25, n=24, seed=5, n_sparse=40)),
        ("surface", synth.capsule_frame(W=160, H=120, f=131.25, n=32, seed=6, n_sparse=25)),
    ]


def _lattice(vd, mode, fr):
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL if mode == "all" else vd.VD_ACTIVE_SURFACE)
    lat.set_frame_from(fr)
    return lat


def test_batch_matches_oracle_and_single_solves(vd):
    items = _frames()
    prm = vd.params(gn_iters=4, cg_iters=10, fixed_association=True, init=vd.VD_INIT_ZERO)
    lats = [_lattice(vd, m, fr) for m, fr in items]
    batch = vd.Batch(lats)
    reps = batch.solve(prm)
    for (mode, fr), lat, rep in zip(items, lats, reps):
        u, _ = lat.get_warp()
        ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
        res = ref.solve(4, 10, fixed_association=True)
        u0, _ = ref.get_warp()
        assert np.abs(u - u0).max() <= 1e-4 * fr.spacing
        assert abs(rep["e_total"] - res["energy"][-1, 0]) <= 1e-5 * res["energy"][-1, 0]
        single = _lattice(vd, mode, fr)
        r1 = single.solve(prm)
        u1, _ = single.get_warp()
        assert np.abs(u - u1).max() <= 1e-5 * fr.spacing
        assert r1["n_valid_corr"] == rep["n_valid_corr"] and r1["cg_done"] == rep["cg_done"]
    assert batch.launch_count() > 0


def test_batch_tune_and_repeat(vd):
    items = _frames()[:4]
    prm = vd.params(gn_iters=3, cg_iters=8, init=vd.VD_INIT_ZERO)
    lats = [_lattice(vd, m, fr) for m, fr in items]
    batch = vd.Batch(lats)
    first = batch.solve(prm)
    streams, ms = batch.tune(prm)
    assert streams >= 1 and ms > 0
    again = batch.solve(prm)                   # re-captured with the tuned branches
    for a, b in zip(first, again):
        assert a["n_valid_corr"] == b["n_valid_corr"]
        assert abs(a["e_total"] - b["e_total"]) <= 1e-5 * a["e_total"]


def test_batch_needs_frames(vd):
    fr = synth.config1()
    a = _lattice(vd, "all", fr)
    b = vd.Lattice(fr.dims, fr.origin, fr.spacing)
    batch = vd.Batch([a, b])
    with pytest.raises(vd.VDError) as e:
        batch.solve(vd.params())
    assert e.value.status == vd.VD_ERR_STATE


@pytest.mark.slow
@pytest.mark.parametrize("n", [64, 69])
def test_batch_run_ahead_persistent_branch(vd, n):
    """A 64^3 (exact bricks) or 69^3 (padded bricks with unaligned rows, whose padded
    vectors the batch allocates before its capture) all-nodes lattice in a batch with
    small ones, under a plan that makes lattices of at least 2^17 active nodes run ahead
    with their persistent (cooperative) position step while the others' streamed
    schedules follow as branches; every lattice of the batch matches the oracle within the
    parity tolerances."""
    items = [("all", synth.capsule_frame(W=320, H=240, f=262.5, n=n, seed=9, n_sparse=120)),
             ("all", synth.capsule_frame(W=160, H=120, f=131.25, n=24, seed=5, n_sparse=40)),
             ("surface", synth.config1())]
    prm = vd.params(gn_iters=3, cg_iters=10, fixed_association=True, init=vd.VD_INIT_ZERO)
    lats = [_lattice(vd, m, fr) for m, fr in items]
    batch = vd.Batch(lats)
    batch.set_plan(2, True, 1 << 17)
    reps = batch.solve(prm)
    assert n ** 3 >= (1 << 17) > 24 ** 3
    assert lats[0].pcg_plan()["padded"] == (1 if n % 4 else 0)
    for (mode, fr), lat, rep in zip(items, lats, reps):
        u, _ = lat.get_warp()
        ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
        res = ref.solve(3, 10, fixed_association=True)
        u0, _ = ref.get_warp()
        err = float(np.abs(u - u0).max())
        rel = abs(rep["e_total"] - res["energy"][-1, 0]) / res["energy"][-1, 0]
        print(f"batch run-ahead {fr.dims}: |du|max = {err / fr.spacing:.2e} h, dE/E = {rel:.2e}")
        assert err <= 1e-4 * fr.spacing
        assert rel <= 1e-5


@pytest.mark.parametrize("threads,ctas,weight", [(512, 1, 2.0), (256, 2, 1.0), (256, 1, 4.0)])
def test_persistent_batch_matches_oracle(vd, threads, ctas, weight):
    """The batch's position steps as one persistent cooperative kernel per Gauss-Newton
    iteration (one CTA group per lattice, vectors in global memory), the other stages as
    branches: every lattice matches the oracle and its own vd_solve."""
    items = _frames()
    prm = vd.params(gn_iters=4, cg_iters=10, fixed_association=True, init=vd.VD_INIT_ZERO)
    lats = [_lattice(vd, m, fr) for m, fr in items]
    batch = vd.Batch(lats)
    batch.set_persistent(True, threads, ctas, weight)
    reps = batch.solve(prm)
    assert batch.plan()["persistent"]
    with pytest.raises(vd.VDError):       # more resident CTAs than the device holds
        other = vd.Batch(lats)
        other.set_persistent(True, 512, 8, 1.0)
        other.solve(prm)
    for (mode, fr), lat, rep in zip(items, lats, reps):
        assert rep["status"] == vd.VD_OK
        u, _ = lat.get_warp()
        ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
        res = ref.solve(4, 10, fixed_association=True)
        u0, _ = ref.get_warp()
        assert np.abs(u - u0).max() <= 1e-4 * fr.spacing
        assert abs(rep["e_total"] - res["energy"][-1, 0]) <= 1e-5 * res["energy"][-1, 0]
        assert rep["cg_done"] == int(res["cg_done"][-1])
    # a second solve replays the same graph
    again = batch.solve(prm)
    for a, b in zip(reps, again):
        assert abs(a["e_total"] - b["e_total"]) <= 1e-6 * a["e_total"]


def test_persistent_batch_free_association_and_tune(vd):
    items = _frames()[:4]
    prm = vd.params(gn_iters=3, cg_iters=8, init=vd.VD_INIT_ZERO)
    lats = [_lattice(vd, m, fr) for m, fr in items]
    batch = vd.Batch(lats)
    batch.set_persistent(True, 512, 1, 2.0)
    first = batch.solve(prm)
    for (mode, fr), lat, rep in zip(items, lats, first):
        ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
        res = ref.solve(3, 8, fixed_association=False)
        assert abs(rep["e_total"] - res["energy"][-1, 0]) <= 1e-5 * res["energy"][-1, 0]
    streams, ms = batch.tune(prm)
    plan = batch.plan()
    print(f"tuned batch: {plan}, {ms:.3f} ms")
    again = batch.solve(prm)
    for a, b in zip(first, again):
        assert a["n_valid_corr"] == b["n_valid_corr"]
        assert abs(a["e_total"] - b["e_total"]) <= 1e-5 * a["e_total"]


def _check_against_oracle(vd, items, lats, reps, gn, cg, single=True):
    for (mode, fr), lat, rep in zip(items, lats, reps):
        assert rep["status"] == vd.VD_OK
        u, _ = lat.get_warp()
        ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
        res = ref.solve(gn, cg, fixed_association=True)
        u0, _ = ref.get_warp()
        err = float(np.abs(u - u0).max())
        rel = abs(rep["e_total"] - res["energy"][-1, 0]) / res["energy"][-1, 0]
        print(f"wave batch {fr.dims} ({mode}): |du|max = {err / fr.spacing:.2e} h, dE/E = {rel:.2e}")
        assert err <= 1e-4 * fr.spacing
        assert rel <= 1e-5
        assert rep["cg_done"] == int(res["cg_done"][-1])
        if single:
            one = _lattice(vd, mode, fr)
            one.solve(vd.params(gn_iters=gn, cg_iters=cg, fixed_association=True, init=vd.VD_INIT_ZERO))
            u1, _ = one.get_warp()
            assert np.abs(u - u1).max() <= 1e-5 * fr.spacing


def test_wave_batch_mixed_forms_matches_oracle(vd):
    """The position steps in waves of the shared-memory persistent step (VD_BATCH_WAVES):
    all-nodes lattices of which one has nx % 4 != 0 (the scalar stencil for all of them)
    and surface-set lattices (a launch of their own); every lattice matches the oracle,
    its own vd_solve, and a replay of the same graph."""
    items = _frames()
    prm = vd.params(gn_iters=4, cg_iters=10, fixed_association=True, init=vd.VD_INIT_ZERO)
    lats = [_lattice(vd, m, fr) for m, fr in items]
    batch = vd.Batch(lats)
    batch.set_persistent(vd.VD_BATCH_WAVES)
    reps = batch.solve(prm)
    assert batch.plan()["form"] == "waves"
    _check_against_oracle(vd, items, lats, reps, 4, 10)
    again = batch.solve(prm)
    for a, b in zip(reps, again):
        assert abs(a["e_total"] - b["e_total"]) <= 1e-6 * a["e_total"]


def test_wave_batch_several_waves_matches_oracle(vd):
    """All-nodes lattices with nx % 4 == 0 (float4 groups, bricks) whose CTA groups need
    more than the SMs hold at once -- the 32^3 and 48^3 lattices see a 640x480 frame and
    their groups are sized by their samples (at most 512 per CTA) -- run in two or more
    waves inside each launch; every lattice matches the oracle and its own vd_solve."""
    import torch
    items = [("all", synth.capsule_frame(W=320, H=240, f=262.5, n=64, seed=9, n_sparse=120)),
             ("all", synth.capsule_frame(W=640, H=480, f=525.0, n=32, seed=7, n_sparse=60)),
             ("all", synth.sphere_frame(W=640, H=480, f=525.0, n=48, seed=8, n_sparse=80)),
             ("all", synth.config1())]
    prm = vd.params(gn_iters=3, cg_iters=10, fixed_association=True, init=vd.VD_INIT_ZERO)
    lats = [_lattice(vd, m, fr) for m, fr in items]
    batch = vd.Batch(lats)
    batch.set_persistent(vd.VD_BATCH_WAVES)
    batch.set_wave_share(512)
    reps = batch.solve(prm)
    need = sum(batch.groups())
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    print(f"wave batch groups {batch.groups()} ({need} CTAs, {sms} SMs), waves {batch.waves()}")
    assert need > sms and batch.waves() >= 2
    _check_against_oracle(vd, items, lats, reps, 3, 10)


def test_wave_batch_free_association_and_tune(vd):
    """The wave form with re-association at every Gauss-Newton iteration (the bench's
    mode): every lattice's final energy within 1e-5 of the oracle's free-association
    solve; then the tuner (which times the wave form beside the others) and a replay."""
    items = _frames()[:4]
    prm = vd.params(gn_iters=3, cg_iters=8, init=vd.VD_INIT_ZERO)
    lats = [_lattice(vd, m, fr) for m, fr in items]
    batch = vd.Batch(lats)
    batch.set_persistent(vd.VD_BATCH_WAVES)
    first = batch.solve(prm)
    for (mode, fr), lat, rep in zip(items, lats, first):
        ref = oracle.Oracle.from_frame(fr, oracle.ACTIVE_ALL if mode == "all" else oracle.ACTIVE_SURFACE)
        res = ref.solve(3, 8, fixed_association=False)
        assert abs(rep["e_total"] - res["energy"][-1, 0]) <= 1e-5 * res["energy"][-1, 0]
    streams, ms = batch.tune(prm)
    plan = batch.plan()
    print(f"tuned batch: {plan}, {ms:.3f} ms")
    assert plan["form"] in ("branches", "waves", "global")
    again = batch.solve(prm)
    for a, b in zip(first, again):
        assert a["n_valid_corr"] == b["n_valid_corr"]
        assert abs(a["e_total"] - b["e_total"]) <= 1e-5 * a["e_total"]


def test_batch_plan_arguments(vd):
    fr = synth.config1()
    batch = vd.Batch([_lattice(vd, "all", fr)])
    for bad in (lambda: batch.set_persistent(3), lambda: batch.set_persistent(-1),
                lambda: batch.set_wave_share(16)):
        with pytest.raises(vd.VDError) as e:
            bad()
        assert e.value.status == vd.VD_ERR_INVALID_ARG
    batch.set_persistent(vd.VD_BATCH_WAVES)
    assert batch.plan()["form"] == "waves"
    assert batch.groups() == [0] and batch.waves() == 0      # before the first build
    batch.solve(vd.params(gn_iters=1, cg_iters=4, fixed_association=True, init=vd.VD_INIT_ZERO))
    assert batch.groups()[0] >= 1 and batch.waves() == 1


def test_wave_batch_refuses_a_lattice_too_large(vd):
    """A lattice whose slots do not fit in the SMs' shared memory at one CTA per SM
    (100^3 all nodes: more than 148 x 6,144 slots) cannot take the wave form: the solve
    reports VD_ERR_INVALID_ARG and the batch still solves in the branch form."""
    import torch
    n = 100
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert n ** 3 > sms * 6144
    fr = synth.config1()
    small = _lattice(vd, "all", fr)
    big = vd.Lattice((n, n, n), fr.origin, 1.0 / n)
    big.set_frame_from(fr)
    batch = vd.Batch([small, big])
    batch.set_persistent(vd.VD_BATCH_WAVES)
    prm = vd.params(gn_iters=1, cg_iters=2, fixed_association=True, init=vd.VD_INIT_ZERO)
    with pytest.raises(vd.VDError) as e:
        batch.solve(prm)
    assert e.value.status == vd.VD_ERR_INVALID_ARG
    batch.set_persistent(vd.VD_BATCH_BRANCHES)
    reps = batch.solve(prm)
    assert all(r["status"] == vd.VD_OK for r in reps)
