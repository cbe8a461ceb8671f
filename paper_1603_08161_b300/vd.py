"""ctypes binding of libvd (include/vd.h): the same entry points, same names.

Argument marshalling only: every step of the solve runs in the CUDA library.  Arrays
may be numpy arrays (host memory, VD_MEM_HOST) or CUDA torch tensors (device memory,
VD_MEM_DEVICE); ``Lattice`` wraps a handle for convenience.  Importing this module
loads ``libvd.so`` and raises ImportError when it has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvd.so")

VD_OK, VD_ERR_INVALID_ARG, VD_ERR_OOM, VD_ERR_CUDA, VD_ERR_STATE, VD_ERR_NUMERIC, VD_ERR_TIMEOUT = range(7)
VD_ACTIVE_SURFACE, VD_ACTIVE_ALL = 0, 1
VD_PREC_FP32, VD_PREC_MIXED = 0, 1
VD_MEM_HOST, VD_MEM_DEVICE = 0, 1
VD_INIT_PREV, VD_INIT_ZERO = 0, 1
VD_APPLY_MATRIX_FREE, VD_APPLY_CACHED, VD_APPLY_AUTO = 0, 1, 2
VD_BATCH_BRANCHES, VD_BATCH_GLOBAL, VD_BATCH_WAVES = 0, 1, 2
_BATCH_FORMS = {VD_BATCH_BRANCHES: "branches", VD_BATCH_GLOBAL: "global", VD_BATCH_WAVES: "waves"}
(VD_KC_ASSOCIATE, VD_KC_RHS, VD_KC_APPLY_STENCIL, VD_KC_APPLY_SAMPLES, VD_KC_UPDATE_X,
 VD_KC_UPDATE_P, VD_KC_ROTATION, VD_KC_ENERGY, VD_KC_PCG) = range(9)
KERNEL_CLASSES = {"associate": 0, "rhs": 1, "apply_stencil": 2, "apply_samples": 3, "update_x": 4,
                  "update_p": 5, "rotation": 6, "energy": 7, "pcg": 8}

UNET_TENSORS = ["x", "e1a", "e1", "p1", "e2a", "e2", "p2", "e3a", "e3", "cat2", "d2a", "d2", "cat1", "d1a", "d1",
                "gout", "gd1", "gd1a", "gcat1", "gd2", "gd2a", "gcat2", "ge3", "ge3a", "gp2", "ge2", "ge2a", "gp1",
                "ge1", "ge1a"]  # ids VD_UNET_T_* of include/vd.h, in order

STATUS_NAMES = {0: "VD_OK", 1: "VD_ERR_INVALID_ARG", 2: "VD_ERR_OOM", 3: "VD_ERR_CUDA", 4: "VD_ERR_STATE",
                5: "VD_ERR_NUMERIC", 6: "VD_ERR_TIMEOUT"}


class vd_lattice_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("origin", ctypes.c_float * 3), ("spacing", ctypes.c_float),
                ("active_mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class vd_solve_params(ctypes.Structure):
    _fields_ = [("w_sparse", ctypes.c_float), ("w_dense", ctypes.c_float), ("w_reg", ctypes.c_float),
                ("eps_d", ctypes.c_float), ("eps_n", ctypes.c_float), ("eps_v", ctypes.c_float),
                ("gn_iters", ctypes.c_int), ("cg_iters", ctypes.c_int), ("cg_tol", ctypes.c_double),
                ("fixed_association", ctypes.c_int), ("init", ctypes.c_int)]


class vd_solve_report(ctypes.Structure):
    _fields_ = [("e_total", ctypes.c_double), ("e_dense", ctypes.c_double),
                ("e_sparse", ctypes.c_double), ("e_reg", ctypes.c_double),
                ("gn_done", ctypes.c_int), ("cg_done", ctypes.c_int), ("n_valid_corr", ctypes.c_int),
                ("n_degenerate_rot", ctypes.c_int), ("n_refined", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vd_warm_report(ctypes.Structure):
    _fields_ = [("e_start", ctypes.c_double), ("e_predicted", ctypes.c_double),
                ("used_prediction", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libvd.so is not built ({LIB_PATH}); run `python -m paper_1603_08161_b300.build` "
                      "or __graft_entry__.build()")
lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I = ctypes.c_int
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "vd_create_lattice": [ctypes.POINTER(vd_lattice_desc), ctypes.POINTER(_P)],
    "vd_destroy_lattice": [_P],
    "vd_set_frame": [_P, _P, _I, _I, _P, _P, _P, _P, _I, _I],
    "vd_set_correspondences": [_P, _P, _P, _I, _I],
    "vd_solve": [_P, ctypes.POINTER(vd_solve_params), ctypes.POINTER(vd_solve_report)],
    "vd_solve_async": [_P, ctypes.POINTER(vd_solve_params)],
    "vd_get_report": [_P, ctypes.POINTER(vd_solve_report)],
    "vd_get_warp": [_P, _P, _P, _I],
    "vd_set_warp": [_P, _P, _P, _I],
    "vd_last_error": [_P],
    "vd_num_active": [_P, _PI],
    "vd_get_active": [_P, _P, _I],
    "vd_get_target_normals": [_P, _P, _I],
    "vd_step_associate": [_P, ctypes.POINTER(vd_solve_params)],
    "vd_get_association": [_P, ctypes.POINTER(vd_solve_params), _P, _P, _P, _I],
    "vd_step_rhs": [_P, ctypes.POINTER(vd_solve_params), _P, _P, _I],
    "vd_step_apply": [_P, ctypes.POINTER(vd_solve_params), _P, _P, _PD, _I],
    "vd_step_pcg": [_P, ctypes.POINTER(vd_solve_params), _P, _PI, _I, _I],
    "vd_step_fit_rotations": [_P, _PI],
    "vd_step_energy": [_P, ctypes.POINTER(vd_solve_params), _PD],
    "vd_profile_select": [_P, _I],
    "vd_profile_read": [_P, _PD, _PI],
    "vd_launch_counts": [_P, ctypes.POINTER(vd_solve_params), _PI, _PI],
    "vd_pcg_plan": [_P, _PI, _PI, _PI, _PI, _PI],
    "vd_get_warp_async": [_P, _P, _P, _I],
    "vd_get_warp_wait": [_P],
    "vd_fit_rotations_noalloc": [_I, _I, _I, ctypes.c_float, _P, _P, _P, _P, _P, _P],
    "vd_batch_set_plan": [_P, _I, _I, ctypes.c_longlong],
    "vd_batch_set_persistent": [_P, _I, _I, _I, ctypes.c_float],
    "vd_batch_get_plan": [_P, _PI, _PI, _PI, ctypes.POINTER(ctypes.c_float), _PI],
    "vd_unet_get_tensor": [_P, _I, _P, ctypes.c_longlong, _PI],
    "vd_estimate_pose": [_P, ctypes.POINTER(vd_solve_params), _I, _P, _PI, _PD],
    "vd_mc_case": [_I, _PI],
    "vd_renderer_create": [_I, _I, _I, ctypes.POINTER(_P)],
    "vd_renderer_destroy": [_P],
    "vd_renderer_last_error": [_P],
    "vd_marching_cubes": [_P, _P, _I, _I, _I, _P, ctypes.c_float, ctypes.c_float, _I, _PI],
    "vd_get_mesh": [_P, _P, _P, _I],
    "vd_render_samples": [_P, _P, _P, _P, _I, _P, _P, _P, _I, _PI, _I],
    "vd_set_apply_mode": [_P, _I],
    "vd_test_grid_reduce": [_P, _I, _I, _P],
    "vd_get_apply_mode": [_P, _PI, _PI],
    "vd_tune_apply": [_P, ctypes.POINTER(vd_solve_params), _PI, ctypes.POINTER(ctypes.c_float)],
    "vd_hierarchy_create": [_P, _I, ctypes.POINTER(_P)],
    "vd_hierarchy_destroy": [_P],
    "vd_hierarchy_level": [_P, _I, ctypes.POINTER(_P)],
    "vd_hierarchy_solve": [_P, _P, _P],
    "vd_hierarchy_solve_async": [_P, _P],
    "vd_hierarchy_get_reports": [_P, _P],
    "vd_hierarchy_last_error": [_P],
    "vd_batch_create": [_P, _I, ctypes.POINTER(_P)],
    "vd_batch_destroy": [_P],
    "vd_batch_solve": [_P, ctypes.POINTER(vd_solve_params), _P],
    "vd_batch_solve_async": [_P, ctypes.POINTER(vd_solve_params)],
    "vd_batch_get_reports": [_P, _P],
    "vd_batch_tune": [_P, ctypes.POINTER(vd_solve_params), _PI, ctypes.POINTER(ctypes.c_float)],
    "vd_batch_launch_count": [_P, _PI],
    "vd_batch_get_groups": [_P, _PI, _PI],
    "vd_batch_set_wave_share": [_P, _I],
    "vd_batch_last_error": [_P],
    "vd_solve_batch": [_P, _I, ctypes.POINTER(vd_solve_params), _P],
    "vd_set_energy_target": [_P, ctypes.c_double],
    "vd_test_stall_barrier": [_P, _I],
    "vd_unet_create": [_I, _I, _I, ctypes.c_ulonglong, ctypes.POINTER(_P)],
    "vd_unet_destroy": [_P],
    "vd_unet_dims": [_P, _PI, _PI, _PI],
    "vd_unet_num_params": [_P, _PI],
    "vd_unet_get_params": [_P, _P, _I],
    "vd_unet_set_params": [_P, _P, _I],
    "vd_unet_get_grads": [_P, _P, _I],
    "vd_unet_forward": [_P, _P, _P],
    "vd_unet_forward_async": [_P, _P, _P, _P],
    "vd_unet_train_step": [_P, _P, _P, ctypes.c_float, ctypes.c_float, _PD],
    "vd_unet_save": [_P, ctypes.c_char_p],
    "vd_unet_load": [_P, ctypes.c_char_p],
    "vd_warm_features": [_P, ctypes.POINTER(vd_solve_params), _P, _I],
    "vd_warm_start": [_P, _P, ctypes.POINTER(vd_solve_params), ctypes.POINTER(vd_warm_report)],
    "vd_get_warm_report": [_P, ctypes.POINTER(vd_warm_report)],
}
VD_NOALLOC_MAX_NODES = 65536
for _name, _args in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = (ctypes.c_char_p if _name in ("vd_last_error", "vd_batch_last_error", "vd_hierarchy_last_error",
                                                "vd_renderer_last_error") else ctypes.c_int)
    globals()[_name] = _fn


class VDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    """(pointer, mem) of a numpy array or a torch tensor; None -> (None, host)."""
    if a is None:
        return None, VD_MEM_HOST
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, VD_MEM_HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (VD_MEM_DEVICE if a.is_cuda else VD_MEM_HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def params(w_sparse=10.0, w_dense=1.0, w_reg=1.0, eps_d=0.05, eps_n=0.5, eps_v=0.8, gn_iters=5,
           cg_iters=10, cg_tol=0.0, fixed_association=False, init=VD_INIT_PREV):
    return vd_solve_params(w_sparse, w_dense, w_reg, eps_d, eps_n, eps_v, gn_iters, cg_iters, cg_tol,
                           int(bool(fixed_association)), init)


class Lattice:
    """A lattice handle: owns the library object, marshals arrays."""

    def __init__(self, dims, origin, spacing, active_mode=VD_ACTIVE_ALL, precision=VD_PREC_FP32, stream=None):
        self.dims = tuple(int(v) for v in dims)
        self.nn = int(np.prod(self.dims))
        d = vd_lattice_desc(self.dims[0], self.dims[1], self.dims[2],
                            (ctypes.c_float * 3)(*[float(v) for v in origin]), float(spacing),
                            int(active_mode), int(precision), stream)
        h = _P()
        st = vd_create_lattice(ctypes.byref(d), ctypes.byref(h))
        if st != VD_OK:
            raise VDError(st, "vd_create_lattice failed")
        self.h = h
        self.C = 0
        self.W = self.H = 0
        self._keep = []

    def _check(self, st):
        if st != VD_OK:
            raise VDError(st, (vd_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            vd_destroy_lattice(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_frame(self, depth, K, pose, src_pts, src_nrm):
        """depth (H, W), source samples (C, 3): numpy (host) or CUDA tensors (device);
        K (4,) and pose (12,) or None are always host values."""
        H, W = depth.shape[:2]
        C = int(src_pts.shape[0])
        pd, mem = _ptr(depth)
        pp, _ = _ptr(src_pts)
        pn, _ = _ptr(src_nrm)
        kk = np.ascontiguousarray(K, np.float32)
        pz = None if pose is None else np.ascontiguousarray(pose, np.float32)
        self._check(vd_set_frame(self.h, pd, W, H, kk.ctypes.data, None if pz is None else pz.ctypes.data,
                                 pp, pn, C, mem))
        self.C, self.W, self.H = C, W, H

    def set_frame_from(self, fr, device=None):
        """Frame from a synth.Frame; ``device`` = torch device to pass device pointers."""
        if device is None:
            self.set_correspondences(fr.sp_canon, fr.sp_target)
            self.set_frame(fr.depth, fr.K, fr.pose, fr.src_pts, fr.src_nrm)
        else:
            import torch
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
            self._keep = [t(fr.depth), t(fr.src_pts), t(fr.src_nrm), t(fr.sp_canon), t(fr.sp_target)]
            d, p, n, a, b = self._keep
            self.set_correspondences(a, b)
            self.set_frame(d, fr.K, fr.pose, p, n)

    def set_correspondences(self, canon, target):
        S = int(canon.shape[0])
        pa, mem = _ptr(canon)
        pb, _ = _ptr(target)
        self._check(vd_set_correspondences(self.h, pa, pb, S, mem))

    def solve(self, prm):
        rep = vd_solve_report()
        st = vd_solve(self.h, ctypes.byref(prm), ctypes.byref(rep))
        if st not in (VD_OK, VD_ERR_NUMERIC):
            self._check(st)
        return rep.as_dict()

    def solve_async(self, prm):
        self._check(vd_solve_async(self.h, ctypes.byref(prm)))

    def report(self):
        rep = vd_solve_report()
        vd_get_report(self.h, ctypes.byref(rep))
        return rep.as_dict()

    def get_warp(self, out_u=None, out_R=None):
        """(u, R) as new numpy arrays when neither output is given; else into the given
        arrays (numpy or CUDA tensors), and with out_u alone u only (R is None)."""
        u = np.zeros((self.nn, 3), np.float32) if out_u is None else out_u
        pu, mem = _ptr(u)
        if out_R is None and out_u is not None:
            R = None
        else:
            R = np.zeros((self.nn, 9), np.float32) if out_R is None else out_R
        pr, mr = _ptr(R)
        if R is not None and mr != mem:
            raise ValueError("u and R must both be host arrays or both CUDA tensors")
        self._check(vd_get_warp(self.h, pu, pr, mem))
        if isinstance(R, np.ndarray):
            R = R.reshape(self.nn, 3, 3)
        return u, R

    def get_warp_async(self, out_u, out_R=None):
        """Enqueue the read of u (and R) into the given arrays without waiting (see
        vd_get_warp_async): page-locked host tensors or CUDA tensors, kept alive here until
        get_warp_wait."""
        pu, mem = _ptr(out_u)
        pr, mr = _ptr(out_R)
        if out_R is not None and mr != mem:
            raise ValueError("u and R must both be host arrays or both CUDA tensors")
        self._rb_keep = [out_u, out_R]
        self._check(vd_get_warp_async(self.h, pu, pr, mem))

    def get_warp_wait(self):
        self._check(vd_get_warp_wait(self.h))
        self._rb_keep = []

    def set_warp(self, u=None, R=None):
        """u (nn, 3) and R (nn, 9) or None: numpy (host) or CUDA tensors (device)."""
        dev = any(a is not None and hasattr(a, "is_cuda") and a.is_cuda for a in (u, R))
        if dev and not all(a is None or (hasattr(a, "is_cuda") and a.is_cuda) for a in (u, R)):
            raise ValueError("u and R must both be host arrays or both CUDA tensors")
        conv = (lambda a: a.contiguous()) if dev else (lambda a: np.ascontiguousarray(a, np.float32))
        uu = None if u is None else conv(u)
        RR = None if R is None else conv(R)
        pu, _ = _ptr(uu)
        pr, _ = _ptr(RR)
        self._check(vd_set_warp(self.h, pu, pr, VD_MEM_DEVICE if dev else VD_MEM_HOST))

    def estimate_pose(self, prm, iters):
        """Dense projective ICP on the global pose: (pose (12,), steps, E before each step)."""
        pose = np.zeros(12, np.float32)
        steps = ctypes.c_int()
        e = np.zeros(max(iters, 1))
        self._check(vd_estimate_pose(self.h, ctypes.byref(prm), int(iters), pose.ctypes.data, ctypes.byref(steps),
                                     e.ctypes.data_as(_PD)))
        return pose, steps.value, e[:steps.value]

    def set_apply_mode(self, mode):
        self._check(vd_set_apply_mode(self.h, int(mode)))

    def apply_mode(self):
        m, now = ctypes.c_int(), ctypes.c_int()
        self._check(vd_get_apply_mode(self.h, ctypes.byref(m), ctypes.byref(now)))
        return m.value, bool(now.value)

    def tune_apply(self, prm):
        m = ctypes.c_int()
        ms = (ctypes.c_float * 2)()
        self._check(vd_tune_apply(self.h, ctypes.byref(prm), ctypes.byref(m), ms))
        return m.value, (ms[0], ms[1])

    def test_stall_barrier(self, on):
        """Failure injection: make the position step's first grid-barrier wait run out."""
        self._check(vd_test_stall_barrier(self.h, 1 if on else 0))

    def set_energy_target(self, e_target):
        """Stop later solves after the first iteration with E_total <= e_target (< 0: off)."""
        self._check(vd_set_energy_target(self.h, float(e_target)))

    def warm_features(self, prm, out=None):
        """Network input (nn, 6) at the current warp; ``out`` may be a CUDA tensor."""
        x = np.zeros((self.nn, 6), np.float32) if out is None else out
        px, mem = _ptr(x)
        self._check(vd_warm_features(self.h, ctypes.byref(prm), px, mem))
        return x

    def warm_start(self, net, prm, wait=True):
        """Learned warm start of the current frame (see vd_warm_start)."""
        rep = vd_warm_report()
        self._check(vd_warm_start(self.h, net.h, ctypes.byref(prm), ctypes.byref(rep) if wait else None))
        return rep.as_dict() if wait else None

    def warm_report(self):
        rep = vd_warm_report()
        self._check(vd_get_warm_report(self.h, ctypes.byref(rep)))
        return rep.as_dict()

    def num_active(self):
        n = ctypes.c_int()
        self._check(vd_num_active(self.h, ctypes.byref(n)))
        return n.value

    def active_mask(self):
        m = np.zeros(self.nn, np.uint8)
        self._check(vd_get_active(self.h, m.ctypes.data, VD_MEM_HOST))
        return m.astype(bool)

    def target_normals(self):
        n = np.zeros((self.H, self.W, 3), np.float32)
        self._check(vd_get_target_normals(self.h, n.ctypes.data, VD_MEM_HOST))
        return n

    def associate(self, prm):
        self._check(vd_step_associate(self.h, ctypes.byref(prm)))

    def association(self, prm):
        pix = np.zeros(self.C, np.int32)
        w = np.zeros(self.C, np.float32)
        r = np.zeros(self.C, np.float32)
        self._check(vd_get_association(self.h, ctypes.byref(prm), pix.ctypes.data, w.ctypes.data,
                                       r.ctypes.data, VD_MEM_HOST))
        return pix, w, r

    def rhs(self, prm):
        b = np.zeros((self.nn, 3), np.float32)
        d = np.zeros((self.nn, 3), np.float32)
        self._check(vd_step_rhs(self.h, ctypes.byref(prm), b.ctypes.data, d.ctypes.data, VD_MEM_HOST))
        return b, d

    def apply(self, prm, p):
        p = np.ascontiguousarray(p, np.float32)
        q = np.zeros((self.nn, 3), np.float32)
        dot = ctypes.c_double()
        self._check(vd_step_apply(self.h, ctypes.byref(prm), p.ctypes.data, q.ctypes.data, ctypes.byref(dot),
                                  VD_MEM_HOST))
        return q, dot.value

    def pcg(self, prm, apply=False):
        x = np.zeros((self.nn, 3), np.float32)
        it = ctypes.c_int()
        self._check(vd_step_pcg(self.h, ctypes.byref(prm), x.ctypes.data, ctypes.byref(it), int(apply),
                                VD_MEM_HOST))
        return x, it.value

    def fit_rotations(self):
        n = ctypes.c_int()
        self._check(vd_step_fit_rotations(self.h, ctypes.byref(n)))
        return n.value

    def energy(self, prm):
        out = (ctypes.c_double * 4)()
        self._check(vd_step_energy(self.h, ctypes.byref(prm), out))
        return np.array(list(out))

    def profile_select(self, kernel_class):
        self._check(vd_profile_select(self.h, int(kernel_class)))

    def profile_read(self):
        ms = ctypes.c_double()
        n = ctypes.c_int()
        self._check(vd_profile_read(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def launch_counts(self, prm):
        a = ctypes.c_int()
        b = ctypes.c_int()
        self._check(vd_launch_counts(self.h, ctypes.byref(prm), ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def pcg_plan(self):
        """Partition of the persistent position step: CTAs, slots per CTA, brick rows."""
        v = [ctypes.c_int() for _ in range(5)]
        self._check(vd_pcg_plan(self.h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("ctas", "chunk", "by", "bz", "padded"), [x.value for x in v]))


class Batch:
    """Several lattices solved by one captured graph (vd_batch_*)."""

    def __init__(self, lattices):
        self.lattices = list(lattices)
        arr = (_P * len(self.lattices))(*[lt.h for lt in self.lattices])
        h = _P()
        st = vd_batch_create(arr, len(self.lattices), ctypes.byref(h))
        if st != VD_OK:
            raise VDError(st, "vd_batch_create failed")
        self.h = h

    def _check(self, st):
        if st != VD_OK:
            raise VDError(st, (vd_batch_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            vd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, prm):
        reps = (vd_solve_report * len(self.lattices))()
        st = vd_batch_solve(self.h, ctypes.byref(prm), reps)
        if st not in (VD_OK, VD_ERR_NUMERIC):
            self._check(st)
        return [r.as_dict() for r in reps]

    def solve_async(self, prm):
        self._check(vd_batch_solve_async(self.h, ctypes.byref(prm)))

    def reports(self):
        reps = (vd_solve_report * len(self.lattices))()
        vd_batch_get_reports(self.h, reps)
        return [r.as_dict() for r in reps]

    def tune(self, prm):
        n = ctypes.c_int()
        ms = ctypes.c_float()
        self._check(vd_batch_tune(self.h, ctypes.byref(prm), ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def launch_count(self):
        n = ctypes.c_int()
        self._check(vd_batch_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def set_wave_share(self, samples_per_cta):
        self._check(vd_batch_set_wave_share(self.h, int(samples_per_cta)))

    def groups(self):
        """CTAs per lattice of the last persistent build."""
        out = (ctypes.c_int * len(self.lattices))()
        self._check(vd_batch_get_groups(self.h, out, None))
        return list(out)

    def waves(self):
        w = ctypes.c_int()
        self._check(vd_batch_get_groups(self.h, None, ctypes.byref(w)))
        return w.value

    def set_plan(self, streams, largest_first=True, run_ahead_nodes=(1 << 31) - 1):
        self._check(vd_batch_set_plan(self.h, int(streams), int(bool(largest_first)), int(run_ahead_nodes)))

    def set_persistent(self, on=True, threads=512, ctas_per_sm=1, sample_weight=2.0):
        """on: a VD_BATCH_* form, or True / False for VD_BATCH_GLOBAL / VD_BATCH_BRANCHES."""
        form = int(on) if not isinstance(on, bool) else (VD_BATCH_GLOBAL if on else VD_BATCH_BRANCHES)
        self._check(vd_batch_set_persistent(self.h, form, int(threads), int(ctas_per_sm),
                                            float(sample_weight)))

    def plan(self):
        p, t, k, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        w = ctypes.c_float()
        self._check(vd_batch_get_plan(self.h, ctypes.byref(p), ctypes.byref(t), ctypes.byref(k), ctypes.byref(w),
                                      ctypes.byref(st)))
        return {"form": _BATCH_FORMS.get(p.value, p.value), "persistent": p.value != VD_BATCH_BRANCHES,
                "threads": t.value, "ctas_per_sm": k.value, "sample_weight": w.value, "branches": st.value}


class _LevelView(Lattice):
    """A level of a hierarchy: a lattice handle owned by the hierarchy (not destroyed here)."""

    def __init__(self, handle, dims, fine):
        self.h = handle
        self.dims = tuple(dims)
        self.nn = int(np.prod(self.dims))
        self._fine = fine
        self._keep = []

    # the level's frame is level 0's (same samples, same depth map)
    C = property(lambda self: self._fine.C)
    W = property(lambda self: self._fine.W)
    H = property(lambda self: self._fine.H)

    def close(self):
        self.h = None


class Hierarchy:
    """Coarse-to-fine solve (vd_hierarchy_*) on a Lattice (level 0)."""

    def __init__(self, fine, levels):
        self.fine = fine
        h = _P()
        st = vd_hierarchy_create(fine.h, int(levels), ctypes.byref(h))
        if st != VD_OK:
            raise VDError(st, "vd_hierarchy_create failed")
        self.h = h
        self.n_levels = int(levels)
        self.levels = [fine]
        dims = fine.dims
        for l in range(1, levels):
            dims = tuple(d // 2 + 1 for d in dims)
            lh = _P()
            vd_hierarchy_level(self.h, l, ctypes.byref(lh))
            self.levels.append(_LevelView(lh, dims, fine))

    def _check(self, st):
        if st != VD_OK:
            raise VDError(st, (vd_hierarchy_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            vd_hierarchy_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _params(self, schedule):
        assert len(schedule) == self.n_levels
        return (vd_solve_params * self.n_levels)(*schedule)

    def solve(self, schedule):
        """schedule: vd_solve_params per level, coarsest first; returns the reports."""
        self._prm = self._params(schedule)
        reps = (vd_solve_report * self.n_levels)()
        st = vd_hierarchy_solve(self.h, self._prm, reps)
        if st not in (VD_OK, VD_ERR_NUMERIC):
            self._check(st)
        return [r.as_dict() for r in reps]

    def solve_async(self, schedule):
        self._prm = self._params(schedule)
        self._check(vd_hierarchy_solve_async(self.h, self._prm))

    def reports(self):
        reps = (vd_solve_report * self.n_levels)()
        vd_hierarchy_get_reports(self.h, reps)
        return [r.as_dict() for r in reps]


class Renderer:
    """Canonical mesh by marching cubes and rasterised source samples (vd_renderer_*)."""

    def __init__(self, max_triangles, W, H):
        h = _P()
        st = vd_renderer_create(int(max_triangles), int(W), int(H), ctypes.byref(h))
        if st != VD_OK:
            raise VDError(st, "vd_renderer_create failed")
        self.h, self.W, self.H = h, int(W), int(H)
        self.n_tri = 0

    def _check(self, st):
        if st != VD_OK:
            raise VDError(st, (vd_renderer_last_error(self.h) or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            vd_renderer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def marching_cubes(self, grid, origin, spacing, iso=0.0):
        """grid: (sz, sy, sx) float32 numpy array or CUDA tensor; returns the triangle count."""
        sz, sy, sx = grid.shape
        pg, mem = _ptr(grid if not isinstance(grid, np.ndarray) else np.ascontiguousarray(grid, np.float32))
        if isinstance(grid, np.ndarray):
            self._g = np.ascontiguousarray(grid, np.float32)
            pg = self._g.ctypes.data
        o = np.ascontiguousarray(origin, np.float32)
        n = ctypes.c_int()
        self._check(vd_marching_cubes(self.h, pg, sx, sy, sz, o.ctypes.data, float(spacing), float(iso), mem,
                                      ctypes.byref(n)))
        self.n_tri = n.value
        return n.value

    def mesh(self):
        t = np.zeros((self.n_tri, 3, 3), np.float32)
        m = np.zeros((self.n_tri, 3, 3), np.float32)
        self._check(vd_get_mesh(self.h, t.ctypes.data, m.ctypes.data, VD_MEM_HOST))
        return t, m

    def render_into(self, pts, nrm, K, pose=None, lattice=None, stride=1):
        """Samples into CUDA tensors pts, nrm (cap x 3 float32); returns the count."""
        kk = np.ascontiguousarray(K, np.float32)
        pz = None if pose is None else np.ascontiguousarray(pose, np.float32)
        self._kp = (kk, pz)
        n = ctypes.c_int()
        self._check(vd_render_samples(self.h, None if lattice is None else lattice.h, kk.ctypes.data,
                                      None if pz is None else pz.ctypes.data, int(stride), _ptr(pts)[0],
                                      _ptr(nrm)[0], None, int(pts.shape[0]), ctypes.byref(n), VD_MEM_DEVICE))
        return n.value

    def render(self, K, pose=None, lattice=None, stride=1, cap=None):
        """(points (n, 3), normals (n, 3), pixel index (n,)) of the covered pixels, host."""
        cap = self.W * self.H if cap is None else int(cap)
        p = np.zeros((cap, 3), np.float32)
        m = np.zeros((cap, 3), np.float32)
        px = np.zeros(cap, np.int32)
        kk = np.ascontiguousarray(K, np.float32)
        pz = None if pose is None else np.ascontiguousarray(pose, np.float32)
        n = ctypes.c_int()
        self._check(vd_render_samples(self.h, None if lattice is None else lattice.h, kk.ctypes.data,
                                      None if pz is None else pz.ctypes.data, int(stride), p.ctypes.data,
                                      m.ctypes.data, px.ctypes.data, cap, ctypes.byref(n), VD_MEM_HOST))
        k = min(n.value, cap)
        return p[:k], m[:k], px[:k]


class UNet:
    """The warm-start network (vd_unet_*): device arrays in and out (CUDA tensors)."""

    def __init__(self, dims, seed=0):
        self.dims = tuple(int(v) for v in dims)
        h = _P()
        st = vd_unet_create(self.dims[0], self.dims[1], self.dims[2], int(seed), ctypes.byref(h))
        if st != VD_OK:
            raise VDError(st, "vd_unet_create failed")
        self.h = h
        n = ctypes.c_int()
        vd_unet_num_params(self.h, ctypes.byref(n))
        self.n_params = n.value

    @staticmethod
    def _check(st, what):
        if st != VD_OK:
            raise VDError(st, what)

    def close(self):
        if getattr(self, "h", None):
            vd_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        a = np.zeros(self.n_params, np.float32)
        self._check(vd_unet_get_params(self.h, a.ctypes.data, self.n_params), "vd_unet_get_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, np.float32)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {a.size}")
        self._check(vd_unet_set_params(self.h, a.ctypes.data, self.n_params), "vd_unet_set_params")

    def get_grads(self):
        a = np.zeros(self.n_params, np.float32)
        self._check(vd_unet_get_grads(self.h, a.ctypes.data, self.n_params), "vd_unet_get_grads")
        return a

    def forward(self, in6, out3):
        """out3 (nn, 3) = net(in6 (nn, 6)), both CUDA float32 tensors."""
        self._check(vd_unet_forward(self.h, _ptr(in6)[0], _ptr(out3)[0]), "vd_unet_forward")
        return out3

    def train_step(self, in6, target3, lr, surface_weight=0.0):
        loss = ctypes.c_double()
        self._check(vd_unet_train_step(self.h, _ptr(in6)[0], _ptr(target3)[0], float(surface_weight), float(lr),
                                       ctypes.byref(loss)), "vd_unet_train_step")
        return loss.value

    def tensor(self, name):
        """Intermediate tensor of the last forward / training step, (D, H, W, C) float32."""
        tid = UNET_TENSORS.index(name)
        dims = (ctypes.c_int * 4)()
        self._check(vd_unet_get_tensor(self.h, tid, None, 0, dims), "vd_unet_get_tensor")
        a = np.zeros(tuple(dims), np.float32)
        self._check(vd_unet_get_tensor(self.h, tid, a.ctypes.data, a.size, dims), "vd_unet_get_tensor")
        return a

    def save(self, path):
        self._check(vd_unet_save(self.h, os.fsencode(path)), f"vd_unet_save({path})")

    def load(self, path):
        self._check(vd_unet_load(self.h, os.fsencode(path)), f"vd_unet_load({path})")
