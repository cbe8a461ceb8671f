"""What the trained warm-start network gains over the plain solve (test sequences, seeds
from 10001, which the training seeds 1-192 do not include).

Per frame, from the plain trajectory's previous warp, the plain solve sets E_plain with
its full schedule (10 x 20); the plain solve and the learned start are then each run
until E <= E_plain (1 + 1e-5).  The learned path must meet the same tolerance on every
frame (by itself or through its fallback) and need fewer Gauss-Newton iterations on
average than the plain solve does to reach the same energy.
"""
import os

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1603_08161_b300 import learned, synth, vd
    if not os.path.exists(learned.WEIGHTS):
        pytest.fail(f"trained weights missing: {learned.WEIGHTS}")
    return vd, learned, synth


def test_learned_warm_start_needs_fewer_iterations(env):
    vd, learned, synth = env
    net = vd.UNet(synth.lattice_for(96)[0])
    net.load(learned.WEIGHTS)
    summ, rec = learned.evaluate(net, [10001, 10002], frames=6, log=lambda m: None)
    assert summ["frames"] == 10
    for r in rec:
        assert r["e_learned"] <= r["e_plain"] * (1 + learned.E_RTOL) or r["fallback"]
        assert r["gn_plain_stop"] <= learned.GN_ITERS and r["gn_learned"] <= learned.GN_ITERS
    assert summ["prediction_used"] > 0
    assert summ["gn_mean_learned"] < summ["gn_mean_plain_same_tolerance"]
