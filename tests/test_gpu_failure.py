"""Failure detection of the persistent position step, without a GPU fault.

Every grid-barrier wait of the cooperative position step is bounded (about 2e9 SM
cycles).  vd_test_stall_barrier makes the step wait for one more arrival than it has
CTAs, an arrival that no CTA supplies, so the first wait runs out: the kernel sets its
error word and returns, the solve reports VD_ERR_TIMEOUT and leaves the warp of the last
completed iteration, and the same lattice then solves normally again on the same context.
"""
import time

import numpy as np
import pytest

from paper_1603_08161_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1603_08161_b300 import vd as _vd
    return _vd


def test_barrier_wait_runs_out_and_context_recovers(vd):
    # an all-nodes 32^3 lattice: the position step is the cooperative persistent kernel
    fr = synth.sphere_frame(W=96, H=72, f=90.0, n=32, seed=6, n_sparse=40, name="sphere32")
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL)
    lat.set_frame_from(fr)
    prm = vd.params(gn_iters=1, cg_iters=10, init=vd.VD_INIT_ZERO)
    good = lat.solve(prm)
    u_good, _ = lat.get_warp()
    assert good["cg_done"] > 0 and np.abs(u_good).max() > 0

    lat.test_stall_barrier(True)
    t0 = time.time()
    with pytest.raises(vd.VDError) as e:
        lat.solve(prm)
    assert e.value.status == vd.VD_ERR_TIMEOUT
    assert time.time() - t0 < 60
    u_stalled, _ = lat.get_warp()
    assert np.abs(u_stalled).max() == 0.0  # the step was not applied: u of the start

    lat.test_stall_barrier(False)
    again = lat.solve(prm)
    u_again, _ = lat.get_warp()
    assert again["cg_done"] == good["cg_done"]
    # FP32 atomics make repeated solves differ by rounding only
    assert np.abs(u_again - u_good).max() <= 1e-4 * fr.spacing
    assert abs(again["e_total"] - good["e_total"]) <= 1e-5 * good["e_total"]
