"""FP64 CPU oracle of the VolumeDeform lattice solve -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product path (the CUDA library and its binding) never
loads it, and the two share no code: this wrapper drives ``vd_oracle.c``, a plain
double-precision implementation written from the paper (Sec. 4-7, Eq. 1-4).

Parity status of each part (what pins it is in tests/test_oracle_pins.py):
  * S(x) and trilinear weights ............ pinned (affine reproduction, partition of 1)
  * target maps and association (Sec. 5.1). pinned (plane fixtures computed by hand)
  * E_dense / E_sparse / E_reg (Eq. 1-4) ... pinned (rigid motion, identity warp,
                                             translation closed form)
  * Jacobian .............................. pinned (central finite differences of E)
  * PCG position step ...................... pinned (dense Cholesky, closed forms)
  * rotation step .......................... pinned (brute-force search over SO(3))
  * global pose by dense projective ICP (Sec. 6) pinned (gradient of the point-to-plane
                                             energy by central differences; exact recovery of
                                             a rigid motion of a three-plane corner; fixed
                                             point at the true pose)
  * marching cubes (Sec. 4) and rasterised samples (Sec. 5.1) pinned (watertight closed
                                             surfaces, outward normals, plane fields exact,
                                             sphere volume; pixel samples on their rays and
                                             on the analytic surface)
  * hierarchy (Sec. 7.2): restriction of the constraints, injection of the state and
    trilinear prolongation ................. pinned (affine fields reproduced exactly;
                                             data energies of a coarse-trilinear warp equal
                                             on both levels; rigid targets recovered)
  * end-to-end accuracy against ground truth: parity unpinned (the paper prints no
    numbers); reported only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vd_oracle.c")
_LIB = os.path.join(_HERE, "libvd_oracle.so")

ACTIVE_SURFACE = 0
ACTIVE_ALL = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    F = ctypes.POINTER(ctypes.c_float)
    I = ctypes.POINTER(ctypes.c_int)
    U8 = ctypes.POINTER(ctypes.c_ubyte)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "vdo_create": (P, [i, i, i, F, ctypes.c_float, i]),
        "vdo_destroy": (None, [P]),
        "vdo_set_params": (None, [P, d, d, d, d, d, d]),
        "vdo_set_frame": (i, [P, F, i, i, F, F, F, F, i]),
        "vdo_set_correspondences": (i, [P, F, F, i]),
        "vdo_set_warp": (None, [P, D, D]),
        "vdo_get_warp": (None, [P, D, D]),
        "vdo_num_active": (i, [P]),
        "vdo_get_active": (None, [P, U8]),
        "vdo_target_maps": (None, [P, D, D, U8]),
        "vdo_sample_cells": (None, [P, I, D]),
        "vdo_associate": (i, [P]),
        "vdo_get_association": (None, [P, I, D, D]),
        "vdo_energy": (None, [P, D]),
        "vdo_rhs": (None, [P, D, D]),
        "vdo_apply": (None, [P, D, D]),
        "vdo_pcg": (i, [P, i, d, D, D]),
        "vdo_cholesky": (i, [P, D]),
        "vdo_add_increment": (None, [P, D]),
        "vdo_svd3": (None, [D, D, D, D]),
        "vdo_procrustes": (i, [D, D]),
        "vdo_fit_rotations": (i, [P]),
        "vdo_solve": (i, [P, i, i, d, i, i, D, I, I]),
        "vdo_set_domain": (None, [P, i, i, i, ctypes.c_float]),
        "vdo_restrict_state": (None, [P, P]),
        "vdo_prolongate": (None, [P, D, P]),
        "vdo_set_pose": (None, [P, D]),
        "vdo_get_pose": (None, [P, D]),
        "vdo_icp_system": (i, [P, D, D, D]),
        "vdo_icp": (i, [P, i, D]),
        "vdo_mc_case": (i, [i, I]),
        "vdo_marching_cubes": (ctypes.c_long, [F, i, i, i, D, d, d, D, D, ctypes.c_long]),
        "vdo_render_samples": (ctypes.c_long, [P, D, D, ctypes.c_long, i, i, D, D, I, D, D, D, D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def svd3(A):
    lib = _load()
    A = np.ascontiguousarray(A, np.float64).reshape(9)
    U, s, V = np.zeros(9), np.zeros(3), np.zeros(9)
    lib.vdo_svd3(_ptr(A, ctypes.c_double), _ptr(U, ctypes.c_double), _ptr(s, ctypes.c_double),
                 _ptr(V, ctypes.c_double))
    return U.reshape(3, 3), s, V.reshape(3, 3)


def procrustes(A):
    """Best rotation argmax tr(R^T A); None when it is not unique."""
    lib = _load()
    A = np.ascontiguousarray(A, np.float64).reshape(9)
    R = np.zeros(9)
    bad = lib.vdo_procrustes(_ptr(A, ctypes.c_double), _ptr(R, ctypes.c_double))
    return None if bad else R.reshape(3, 3)


class Oracle:
    """One lattice with its frame, correspondences and warp state, solved in FP64."""

    def __init__(self, dims, origin, spacing, active_mode=ACTIVE_ALL):
        lib = _load()
        self.dims = tuple(int(v) for v in dims)
        self.nn = int(np.prod(self.dims))
        o = _f32(origin)
        self._o = o
        self._c = lib.vdo_create(self.dims[0], self.dims[1], self.dims[2], _ptr(o, ctypes.c_float),
                                 ctypes.c_float(spacing), int(active_mode))
        if not self._c:
            raise ValueError("invalid lattice")
        self.W = self.H = self.C = 0

    @classmethod
    def from_frame(cls, fr, active_mode=ACTIVE_ALL, params=None, dims=None, spacing=None):
        """Lattice with the frame's input; dims / spacing override the frame's lattice
        (a coarse level, whose constraints are gathered from the frame's own lattice)."""
        o = cls(dims or fr.dims, fr.origin, spacing or fr.spacing, active_mode)
        if dims is not None:
            _load().vdo_set_domain(o._c, int(fr.dims[0]), int(fr.dims[1]), int(fr.dims[2]),
                                   ctypes.c_float(fr.spacing))
        if params is not None:
            o.set_params(**params)
        o.set_correspondences(fr.sp_canon, fr.sp_target)
        o.set_frame(fr)
        return o

    def close(self):
        if self._c:
            _load().vdo_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, w_sparse=10.0, w_dense=1.0, w_reg=1.0, eps_d=0.05, eps_n=0.5, eps_v=0.8):
        _load().vdo_set_params(self._c, w_sparse, w_dense, w_reg, eps_d, eps_n, eps_v)

    def set_frame(self, fr):
        self._depth = _f32(fr.depth)
        self._K = _f32(fr.K)
        self._pose = _f32(fr.pose)
        self._sp = _f32(fr.src_pts).reshape(-1, 3)
        self._sn = _f32(fr.src_nrm).reshape(-1, 3)
        self.H, self.W = self._depth.shape
        self.C = self._sp.shape[0]
        rc = _load().vdo_set_frame(self._c, _ptr(self._depth, ctypes.c_float), self.W, self.H,
                                   _ptr(self._K, ctypes.c_float), _ptr(self._pose, ctypes.c_float),
                                   _ptr(self._sp, ctypes.c_float), _ptr(self._sn, ctypes.c_float), self.C)
        if rc:
            raise ValueError("vdo_set_frame failed")

    def set_correspondences(self, canon, target):
        self._fh = _f32(canon).reshape(-1, 3)
        self._ft = _f32(target).reshape(-1, 3)
        _load().vdo_set_correspondences(self._c, _ptr(self._fh, ctypes.c_float),
                                        _ptr(self._ft, ctypes.c_float), self._fh.shape[0])

    def set_warp(self, u=None, R=None):
        uu = None if u is None else np.ascontiguousarray(u, np.float64).reshape(self.nn * 3)
        RR = None if R is None else np.ascontiguousarray(R, np.float64).reshape(self.nn * 9)
        _load().vdo_set_warp(self._c, _ptr(uu, ctypes.c_double), _ptr(RR, ctypes.c_double))

    def get_warp(self):
        u = np.zeros(self.nn * 3)
        R = np.zeros(self.nn * 9)
        _load().vdo_get_warp(self._c, _ptr(u, ctypes.c_double), _ptr(R, ctypes.c_double))
        return u.reshape(self.nn, 3), R.reshape(self.nn, 3, 3)

    def num_active(self):
        return _load().vdo_num_active(self._c)

    def active_mask(self):
        m = np.zeros(self.nn, np.uint8)
        _load().vdo_get_active(self._c, _ptr(m, ctypes.c_ubyte))
        return m.astype(bool)

    def target_maps(self):
        V = np.zeros(self.W * self.H * 3)
        N = np.zeros(self.W * self.H * 3)
        v = np.zeros(self.W * self.H, np.uint8)
        _load().vdo_target_maps(self._c, _ptr(V, ctypes.c_double), _ptr(N, ctypes.c_double),
                                _ptr(v, ctypes.c_ubyte))
        return V.reshape(self.H, self.W, 3), N.reshape(self.H, self.W, 3), v.reshape(self.H, self.W).astype(bool)

    def sample_cells(self):
        cell = np.zeros(self.C, np.int32)
        frac = np.zeros(self.C * 3)
        _load().vdo_sample_cells(self._c, _ptr(cell, ctypes.c_int), _ptr(frac, ctypes.c_double))
        return cell, frac.reshape(self.C, 3)

    def associate(self):
        return _load().vdo_associate(self._c)

    def association(self):
        pix = np.zeros(self.C, np.int32)
        w = np.zeros(self.C)
        r = np.zeros(self.C)
        _load().vdo_get_association(self._c, _ptr(pix, ctypes.c_int), _ptr(w, ctypes.c_double),
                                    _ptr(r, ctypes.c_double))
        return pix, w, r

    def energy(self):
        e = np.zeros(4)
        _load().vdo_energy(self._c, _ptr(e, ctypes.c_double))
        return e

    def rhs(self):
        b = np.zeros(self.nn * 3)
        d = np.zeros(self.nn * 3)
        _load().vdo_rhs(self._c, _ptr(b, ctypes.c_double), _ptr(d, ctypes.c_double))
        return b.reshape(self.nn, 3), d.reshape(self.nn, 3)

    def apply(self, p):
        p = np.ascontiguousarray(p, np.float64).reshape(self.nn * 3)
        q = np.zeros(self.nn * 3)
        _load().vdo_apply(self._c, _ptr(p, ctypes.c_double), _ptr(q, ctypes.c_double))
        return q.reshape(self.nn, 3)

    def pcg(self, iters, tol=0.0):
        x = np.zeros(self.nn * 3)
        hist = np.zeros(iters + 1)
        it = _load().vdo_pcg(self._c, iters, tol, _ptr(x, ctypes.c_double), _ptr(hist, ctypes.c_double))
        return x.reshape(self.nn, 3), it, hist[:it + 1]

    def cholesky(self):
        x = np.zeros(self.nn * 3)
        bad = _load().vdo_cholesky(self._c, _ptr(x, ctypes.c_double))
        if bad:
            raise np.linalg.LinAlgError("normal matrix not positive definite")
        return x.reshape(self.nn, 3)

    def add_increment(self, delta):
        d = np.ascontiguousarray(delta, np.float64).reshape(self.nn * 3)
        _load().vdo_add_increment(self._c, _ptr(d, ctypes.c_double))

    def fit_rotations(self):
        return _load().vdo_fit_rotations(self._c)

    def set_pose(self, pose):
        p = np.ascontiguousarray(pose, np.float64).reshape(12)
        _load().vdo_set_pose(self._c, _ptr(p, ctypes.c_double))

    def get_pose(self):
        p = np.zeros(12)
        _load().vdo_get_pose(self._c, _ptr(p, ctypes.c_double))
        return p

    def icp_system(self):
        """(A 6x6, b 6, E, samples used) of the pose's normal equations at the current
        pose and association (Sec. 6, dense projective ICP)."""
        A, b, E = np.zeros(36), np.zeros(6), np.zeros(1)
        n = _load().vdo_icp_system(self._c, _ptr(A, ctypes.c_double), _ptr(b, ctypes.c_double),
                                   _ptr(E, ctypes.c_double))
        return A.reshape(6, 6), b, float(E[0]), n

    def icp(self, iters):
        """Dense projective ICP on the global pose; returns (steps, E before each)."""
        e = np.zeros(max(iters, 1))
        it = _load().vdo_icp(self._c, iters, _ptr(e, ctypes.c_double))
        return it, e[:it]

    def solve(self, gn_iters, cg_iters, cg_tol=0.0, fixed_association=False, cholesky=False):
        e = np.zeros(gn_iters * 4)
        cg = np.zeros(gn_iters, np.int32)
        st = np.zeros(2, np.int32)
        g = _load().vdo_solve(self._c, gn_iters, cg_iters, cg_tol, int(bool(fixed_association)),
                              int(bool(cholesky)), _ptr(e, ctypes.c_double), _ptr(cg, ctypes.c_int),
                              _ptr(st, ctypes.c_int))
        return {"gn_done": g, "energy": e.reshape(gn_iters, 4)[:g], "cg_done": cg[:g],
                "n_valid": int(st[0]), "n_degenerate": int(st[1])}


def mc_case(cs):
    """Triangles (edge triples) of marching-cubes case cs (bit k: corner k inside)."""
    e = np.zeros(36, np.int32)
    n = _load().vdo_mc_case(int(cs), _ptr(e, ctypes.c_int))
    return e[:3 * n].reshape(n, 3)


def marching_cubes(grid, origin, spacing, iso=0.0):
    """Triangles (n, 3, 3) and vertex normals (n, 3, 3) of the iso-surface of a grid
    (sz, sy, sx) of float32 values at `origin`, `spacing` (Sec. 4)."""
    g = np.ascontiguousarray(grid, np.float32)
    sz, sy, sx = g.shape
    o = np.ascontiguousarray(origin, np.float64)
    lib = _load()
    n = lib.vdo_marching_cubes(_ptr(g, ctypes.c_float), sx, sy, sz, _ptr(o, ctypes.c_double), float(spacing),
                               float(iso), None, None, 0)
    tri, nrm = np.zeros(9 * max(n, 1)), np.zeros(9 * max(n, 1))
    lib.vdo_marching_cubes(_ptr(g, ctypes.c_float), sx, sy, sz, _ptr(o, ctypes.c_double), float(spacing),
                           float(iso), _ptr(tri, ctypes.c_double), _ptr(nrm, ctypes.c_double), n)
    return tri[:9 * n].reshape(n, 3, 3), nrm[:9 * n].reshape(n, 3, 3)


def render_samples(ctx, tri, nrm, W, H, K, pose=None):
    """Rasterise the mesh deformed by ctx's warp and `pose` (Sec. 5.1): per pixel the
    winning triangle, depth, canonical point and normal, and the decision margin."""
    tri = np.ascontiguousarray(tri, np.float64).reshape(-1, 9)
    nrm = np.ascontiguousarray(nrm, np.float64).reshape(-1, 9)
    Kd = np.ascontiguousarray(K, np.float64)
    Pd = np.ascontiguousarray(np.eye(3).ravel().tolist() + [0, 0, 0] if pose is None else pose, np.float64)
    win = np.zeros(W * H, np.int32)
    dep, mar = np.zeros(W * H), np.zeros(W * H)
    cp, cn = np.zeros(3 * W * H), np.zeros(3 * W * H)
    cnt = _load().vdo_render_samples(ctx._c, _ptr(tri, ctypes.c_double), _ptr(nrm, ctypes.c_double), tri.shape[0],
                                     W, H, _ptr(Kd, ctypes.c_double), _ptr(Pd, ctypes.c_double),
                                     _ptr(win, ctypes.c_int), _ptr(dep, ctypes.c_double), _ptr(cp, ctypes.c_double),
                                     _ptr(cn, ctypes.c_double), _ptr(mar, ctypes.c_double))
    return {"count": int(cnt), "win": win.reshape(H, W), "depth": dep.reshape(H, W),
            "point": cp.reshape(H, W, 3), "normal": cn.reshape(H, W, 3), "margin": mar.reshape(H, W)}


def coarse_dims(dims):
    """Node counts of the next coarser level (Sec. 7.2): every coarse cell is the parent
    voxel of 2 x 2 x 2 finer cells, so n nodes per axis become n // 2 + 1 (the nodes
    0, 2, 4, ... of the finer axis; one past its end when n - 1 is odd)."""
    return tuple(int(n) // 2 + 1 for n in dims)


class Hierarchy:
    """Nested coarse-to-fine solve of one frame (Sec. 7.2): level 0 is the frame's own
    lattice, level l has spacing 2^l h and the same origin, and gathers every constraint
    of the finest level into its coarse cells (each expressed trilinearly in the coarse
    nodes).  A solve restricts the state to every coarse level (injection), then from
    the coarsest level up: flip-flop solve of the level, prolongation of its
    displacement increment to the next finer level, one rotation step there (Sec. 7.1,
    with the prolongated positions); finally the flip-flop solve of level 0."""

    def __init__(self, fr, levels, active_mode=ACTIVE_ALL, params=None):
        assert levels >= 1
        self.levels = [Oracle.from_frame(fr, active_mode, params)]
        dims, h = tuple(fr.dims), float(np.float32(fr.spacing))
        for _ in range(1, levels):
            dims = coarse_dims(dims)
            h = float(np.float32(2.0 * h))
            self.levels.append(Oracle.from_frame(fr, active_mode, params, dims=dims, spacing=h))

    def restrict(self):
        """Injection of the state into every coarse level; returns the start displacements."""
        lib = _load()
        starts = [None]
        for l in range(1, len(self.levels)):
            lib.vdo_restrict_state(self.levels[l - 1]._c, self.levels[l]._c)
            starts.append(self.levels[l].get_warp()[0].copy())
        return starts

    def prolongate(self, l, start):
        """Add level l's increment (u - start) to level l - 1, trilinearly."""
        s = np.ascontiguousarray(start, np.float64).reshape(-1)
        _load().vdo_prolongate(self.levels[l]._c, _ptr(s, ctypes.c_double), self.levels[l - 1]._c)

    def solve(self, schedule, fixed_association=False):
        """schedule: (gn_iters, cg_iters) per level, coarsest first.  Returns the
        per-level results of Oracle.solve, coarsest first."""
        assert len(schedule) == len(self.levels)
        starts = self.restrict()
        out = []
        for l in range(len(self.levels) - 1, 0, -1):
            gn, cg = schedule[len(self.levels) - 1 - l]
            out.append(self.levels[l].solve(gn, cg, fixed_association=fixed_association))
            self.prolongate(l, starts[l])
            self.levels[l - 1].fit_rotations()
        gn, cg = schedule[-1]
        out.append(self.levels[0].solve(gn, cg, fixed_association=fixed_association))
        return out
