"""The allocation-free rotation step (vd_fit_rotations_noalloc) against the regular one.

Some callers cannot let the library allocate device memory -- they reserve their whole
device budget up front, or their memory belongs to another allocator -- so the library
offers this variant, whose scratch is a fixed array compiled into the library.  Here it
is called through the C ABI on caller-owned device tensors, twice in a row with
different warps (the second call must not see anything the first left in the shared
scratch), and each result is compared with vd_step_fit_rotations / vd_step_energy on a
lattice holding the same warp, within the stage tolerance the other GPU tests use.  A
second case fills the scratch almost to its cap (40^3 = 64,000 of 65,536 nodes, where
the plane stride and the end of the scratch matter) and checks the rotations and E_reg
(Eq. 4) directly against the FP64 oracle's rotation step on the same warp.
This file sorts last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_1603_08161_b300 import synth

pytestmark = pytest.mark.gpu


def _warp(rng, nn, su, sr):
    u = rng.normal(0, su, (nn, 3)).astype(np.float32)
    w = rng.normal(0, sr, (nn, 3))
    R = np.zeros((nn, 3, 3))
    for i in range(nn):
        th = np.linalg.norm(w[i])
        k = w[i] / th
        Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R[i] = np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx
    return u, R.astype(np.float32)


def test_noalloc_rotation_step_matches_lattice_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1603_08161_b300 import vd

    fr = synth.config1()
    nx, ny, nz = fr.dims
    nn = nx * ny * nz
    lat = vd.Lattice(fr.dims, fr.origin, fr.spacing, vd.VD_ACTIVE_ALL)
    lat.set_frame_from(fr)
    prm = vd.params()
    dev = torch.device("cuda", 0)
    for call, (su, sr) in enumerate([(0.01, 0.05), (0.004, 0.3)]):
        u, R = _warp(np.random.default_rng(100 + call), nn, su, sr)
        # regular path: the lattice's rotation step and its E_reg with the new rotations
        lat.set_warp(u, R)
        nd_ref = lat.fit_rotations()
        _, R_ref = lat.get_warp()
        e_ref = lat.energy(prm)[3]
        # allocation-free path on caller-owned device memory
        du = torch.from_numpy(u).to(dev)
        dr = torch.from_numpy(R.reshape(nn, 9)).to(dev)
        dro = torch.full((nn, 9), float("nan"), dtype=torch.float32, device=dev)
        de = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        dn = torch.full((1,), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        st = vd.vd_fit_rotations_noalloc(nx, ny, nz, ctypes.c_float(fr.spacing), du.data_ptr(), dr.data_ptr(),
                                         dro.data_ptr(), de.data_ptr(), dn.data_ptr(), None)
        assert st == vd.VD_OK
        torch.cuda.synchronize()
        R_out = dro.cpu().numpy().reshape(nn, 3, 3)
        assert np.isfinite(R_out).all()
        assert np.abs(R_out - R_ref).max() <= 2e-5
        assert int(dn.item()) == nd_ref
        assert abs(float(de.item()) - e_ref) <= 2e-5 * abs(e_ref)
    # sizes beyond the scratch are refused before any device work
    big = int(np.ceil(vd.VD_NOALLOC_MAX_NODES ** (1 / 3))) + 1
    assert vd.vd_fit_rotations_noalloc(big, big, big, ctypes.c_float(0.01), du.data_ptr(), dr.data_ptr(),
                                       dro.data_ptr(), None, None, None) == vd.VD_ERR_INVALID_ARG


def _empty_frame(dims, origin, spacing):
    """A frame with no samples or pairs: only the lattice matters to a rotation step."""
    return synth.Frame(depth=np.zeros((3, 3), np.float32), K=np.array([1, 1, 1, 1], np.float32),
                       pose=np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float32),
                       src_pts=np.zeros((0, 3), np.float32), src_nrm=np.zeros((0, 3), np.float32),
                       sp_canon=np.zeros((0, 3), np.float32), sp_target=np.zeros((0, 3), np.float32),
                       dims=dims, origin=origin, spacing=spacing)


def test_noalloc_rotation_step_near_the_cap_matches_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    from paper_1603_08161_b300 import vd

    dims, origin, h = synth.lattice_for(40)
    nx, ny, nz = dims
    nn = nx * ny * nz
    assert nn <= vd.VD_NOALLOC_MAX_NODES and 2 * nn > vd.VD_NOALLOC_MAX_NODES
    dev = torch.device("cuda", 0)
    ref = oracle.Oracle(dims, origin, h, oracle.ACTIVE_ALL)
    ref.set_frame(_empty_frame(dims, origin, h))
    for call, (su, sr) in enumerate([(0.1, 0.1), (0.05, 0.4)]):
        u, R = _warp(np.random.default_rng(300 + call), nn, su * h, sr)
        ref.set_warp(u.astype(np.float64), R.astype(np.float64))
        nd_ref = ref.fit_rotations()
        _, R_ref = ref.get_warp()
        e_ref = ref.energy()[3]
        du = torch.from_numpy(u).to(dev)
        dr = torch.from_numpy(R.reshape(nn, 9)).to(dev)
        dro = torch.full((nn, 9), float("nan"), dtype=torch.float32, device=dev)
        de = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        dn = torch.full((1,), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        st = vd.vd_fit_rotations_noalloc(nx, ny, nz, ctypes.c_float(h), du.data_ptr(), dr.data_ptr(),
                                         dro.data_ptr(), de.data_ptr(), dn.data_ptr(), None)
        assert st == vd.VD_OK
        torch.cuda.synchronize()
        R_out = dro.cpu().numpy().reshape(nn, 3, 3).astype(np.float64)
        assert np.isfinite(R_out).all()
        err = np.abs(R_out - R_ref).max()
        assert err <= 2e-5, f"call {call}: rotation error {err:.3e}"
        assert int(dn.item()) == nd_ref
        rel = abs(float(de.item()) - e_ref) / e_ref
        assert rel <= 1e-5, f"call {call}: E_reg relative error {rel:.3e}"
