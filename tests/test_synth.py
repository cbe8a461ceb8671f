"""The input generator's two tracers agree: the float64 torch sphere tracing of the
capsule sequences (used on the GPU for training data) reproduces the numpy tracing."""
import numpy as np
import pytest

from paper_1603_08161_b300 import synth


def test_torch_tracer_matches_numpy():
    pytest.importorskip("torch")
    kw = dict(frames=2, W=80, H=60, f=65.625, n=16)
    a = synth.sequence_frames(7, **kw)
    b = synth.sequence_frames(7, device="cpu", **kw)
    for fa, fb in zip(a, b):
        assert fa.C == fb.C > 100
        np.testing.assert_array_equal(fa.depth > 0, fb.depth > 0)
        np.testing.assert_allclose(fa.depth, fb.depth, rtol=0, atol=1e-6)
        np.testing.assert_allclose(fa.src_pts, fb.src_pts, rtol=0, atol=1e-6)
        np.testing.assert_array_equal(fa.sp_canon, fb.sp_canon)
