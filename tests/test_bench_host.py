"""Host-side arithmetic of bench.py: the algorithmic bytes behind the roofline figures."""
import bench

# the benchmark frame: 96^3 nodes, the capsules frame's samples, 300 pairs, 640 x 480
NN, C, S, W, H = 884736, 36266, 300, 640, 480


def test_position_step_bytes_per_launch():
    # 20 CG iterations of N*108 + C*28 + S*28
    assert bench.algorithmic_bytes("pcg", NN, C, S) == 1931506720


def test_frame_bytes_hold_the_position_steps_and_the_stages():
    b = bench.frame_algorithmic_bytes(NN, C, S, W, H)
    pcg = bench.GN * bench.algorithmic_bytes("pcg", NN, C, S)
    # the position steps are most of the frame's bytes; the stages around them the rest
    assert pcg < b < 1.1 * pcg
    # no Gauss-Newton iteration: only the energy and the target maps remain
    assert bench.frame_algorithmic_bytes(NN, C, S, W, H, gn=0) == 28 * C + 48 * NN + 28 * W * H
    # no CG iteration: per Gauss-Newton iteration the association, RHS and rotation step
    once = bench.frame_algorithmic_bytes(NN, C, S, W, H, gn=1, cg=0)
    assert once - bench.frame_algorithmic_bytes(NN, C, S, W, H, gn=0) == 68 * C + 120 * NN


def test_frame_roofline_is_consistent():
    peak = 6500.6
    r = bench.frame_roofline(200.0, NN, C, S, W, H, peak)
    assert abs(r["frac"] * r["bound_frames_per_s"] - 200.0) < 1e-6
    assert abs(r["achieved_GBps"] / peak - r["frac"]) < 1e-12
    assert r["algorithmic_bytes_per_frame"] == bench.frame_algorithmic_bytes(NN, C, S, W, H)
