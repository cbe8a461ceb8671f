"""Seeded synthetic RGB-D-shaped workloads for the lattice solve.

This module only builds inputs: it renders depth maps of deforming surfaces with a
pinhole camera, and emits the canonical surface samples, the sparse feature pairs and
the lattice placement. It holds none of the method's arithmetic (no space deformation
S(x), no association, no energy, no solve), so the FP64 oracle and the CUDA path can
both consume its arrays without sharing any solver code.

Scene conventions (the paper leaves them open, Sec. 4-5):
  * camera at the origin looking down +z, pixel (u, v) has the ray
    ((u - cx) / fx, (v - cy) / fy, 1) and depth = z; cx = (W-1)/2, cy = (H-1)/2;
  * lattice over the cube [-0.5, 0.5]^2 x [0.5, 1.5] m with cell-centred nodes:
    origin = cube_min + h/2, spacing h = 1/n;
  * the "source samples" stand in for the rasterised model of Sec. 5.1: the canonical
    (undeformed) surface rendered by the same camera, one sample per covered pixel,
    with its analytic normal.

All arrays are returned as float32 (what both implementations read); random numbers
come from numpy's PCG64 ``default_rng`` with the documented seeds.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Frame", "sphere_frame", "capsule_frame", "config1", "config2",
           "batch_frames", "sequence_frames", "sequences", "lattice_for", "plane_frame", "corner_frame", "sdf_grid"]


@dataclasses.dataclass
class Frame:
    """One frame of input: depth map, intrinsics, source samples, sparse pairs."""
    depth: np.ndarray          # (H, W) float32, metres, 0 = invalid
    K: np.ndarray              # (4,) float32: fx, fy, cx, cy
    pose: np.ndarray           # (12,) float32: row-major R_g (3x3) then t_g
    src_pts: np.ndarray        # (C, 3) float32 canonical sample positions p^_c
    src_nrm: np.ndarray        # (C, 3) float32 canonical sample normals n^_c
    sp_canon: np.ndarray       # (S, 3) float32 canonical feature positions f^_s
    sp_target: np.ndarray      # (S, 3) float32 observed feature positions f_s
    dims: tuple                # lattice nodes (nx, ny, nz)
    origin: np.ndarray         # (3,) float32 position of node (0, 0, 0)
    spacing: float             # lattice spacing h (float32 value)
    name: str = ""

    @property
    def W(self) -> int:
        return int(self.depth.shape[1])

    @property
    def H(self) -> int:
        return int(self.depth.shape[0])

    @property
    def C(self) -> int:
        return int(self.src_pts.shape[0])

    @property
    def S(self) -> int:
        return int(self.sp_canon.shape[0])


def lattice_for(n, cube_min=(-0.5, -0.5, 0.5), cube_size=1.0):
    """Cell-centred lattice of n^3 nodes (or n = (nx, ny, nz)) over a cube of side 1 m."""
    if np.isscalar(n):
        n = (int(n),) * 3
    nmax = max(n)
    h = np.float32(cube_size / nmax)
    origin = (np.asarray(cube_min, np.float64) + 0.5 * float(h)).astype(np.float32)
    return tuple(int(v) for v in n), origin, float(h)


def _intrinsics(W, H, f):
    return np.array([f, f, (W - 1) / 2.0, (H - 1) / 2.0], np.float64)


def _rays(W, H, K):
    fx, fy, cx, cy = K
    u = np.arange(W, dtype=np.float64)
    v = np.arange(H, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    d = np.stack([(uu - cx) / fx, (vv - cy) / fy, np.ones_like(uu)], -1)
    return d.reshape(-1, 3)


def _identity_pose():
    return np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float32)


def _march(phi, dirs, z0, z1, step, iters_bisect=48):
    """First zero crossing (+ to -) of phi(z * d) along each ray in [z0, z1]; 0 if none."""
    n = dirs.shape[0]
    zs = np.arange(z0, z1 + step, step)
    hit = np.zeros(n, bool)
    lo = np.zeros(n)
    hi = np.zeros(n)
    prev = phi(zs[0] * dirs)
    for k in range(1, len(zs)):
        cur = phi(zs[k] * dirs)
        new = (~hit) & (prev > 0) & (cur <= 0)
        lo[new] = zs[k - 1]
        hi[new] = zs[k]
        hit |= new
        prev = cur
    idx = np.nonzero(hit)[0]
    a, b, d = lo[idx], hi[idx], dirs[idx]
    for _ in range(iters_bisect):          # bracket shrinks to < 1e-7 m well before 48
        m = 0.5 * (a + b)
        f = phi(m[:, None] * d)
        pos = f > 0
        a = np.where(pos, m, a)
        b = np.where(pos, b, m)
    z = np.zeros(n)
    z[idx] = 0.5 * (a + b)
    return z, hit


def _sphere_trace(sdf, dirs, z0, z1, iters=160, eps=2e-6, iters_bisect=40, step=1.0):
    """First surface hit of a signed distance function along each ray (sphere tracing,
    then bisection of the last bracket to well below 1e-7 m); 0 where no hit.  ``step``
    < 1 scales the steps for a function that over-estimates the distance by up to 1/step."""
    n = dirs.shape[0]
    L = np.linalg.norm(dirs, axis=1)
    z = np.full(n, float(z0))
    live = np.ones(n, bool)
    conv = np.zeros(n, bool)
    for _ in range(iters):
        idx = np.nonzero(live)[0]
        if idx.size == 0:
            break
        d = sdf(z[idx, None] * dirs[idx])
        done = d < eps
        conv[idx[done]] = True
        z[idx[~done]] += step * d[~done] / L[idx[~done]]
        live[idx] = ~done
        live &= z < z1
    idx = np.nonzero(conv)[0]
    lo = z[idx]
    hi = lo + 4 * eps / L[idx] + 1e-6
    for _ in range(8):                    # widen until the far end is inside
        out = sdf(hi[:, None] * dirs[idx]) > 0
        if not out.any():
            break
        hi = np.where(out, hi + 1e-5, hi)
    inside = sdf(hi[:, None] * dirs[idx]) <= 0
    idx, lo, hi = idx[inside], lo[inside], hi[inside]
    for _ in range(iters_bisect):
        m = 0.5 * (lo + hi)
        pos = sdf(m[:, None] * dirs[idx]) > 0
        lo = np.where(pos, m, lo)
        hi = np.where(pos, hi, m)
    zz = np.zeros(n)
    hit = np.zeros(n, bool)
    zz[idx] = 0.5 * (lo + hi)
    hit[idx] = True
    return zz, hit


def _rotation(axis, angle):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    x, y, z = axis
    c, s = math.cos(angle), math.sin(angle)
    C = 1 - c
    return np.array([[c + x * x * C, x * y * C - z * s, x * z * C + y * s],
                     [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
                     [z * x * C - y * s, z * y * C + x * s, c + z * z * C]])


# ---------------------------------------------------------------------------
# sphere bent by a smooth sinusoidal displacement field
# ---------------------------------------------------------------------------

def _sine_field(centre, amp, wavelength):
    k = 2.0 * math.pi / wavelength

    def d(x):
        return amp * np.stack([np.sin(k * (x[..., 1] - centre[1])),
                               np.sin(k * (x[..., 2] - centre[2])),
                               np.sin(k * (x[..., 0] - centre[0]))], -1)
    return d


def sphere_frame(W=64, H=48, f=60.0, n=16, radius=0.3, centre=(0.0, 0.0, 1.0),
                 amp=0.02, wavelength=0.5, noise=1e-3, n_sparse=20, sparse_noise=1e-3,
                 invalid_frac=0.0, seed=0, name="sphere", tracer="march"):
    """A sphere bent by d(x) = A sin(...) and seen by a W x H pinhole camera.

    The observed surface is {y : |x(y) - c| = r} with x(y) the preimage of y under
    y = x + d(x), found by 8 fixed-point steps x <- y - d(x).
    """
    rng = np.random.default_rng(seed)
    c = np.asarray(centre, np.float64)
    K = _intrinsics(W, H, f)
    dirs = _rays(W, H, K)
    disp = _sine_field(c, amp, wavelength)

    def phi_deformed(y):
        x = y.copy()
        for _ in range(8):
            x = y - disp(x)
        return np.linalg.norm(x - c, axis=-1) - radius

    if tracer == "march":
        z, hit = _march(phi_deformed, dirs, c[2] - radius - 0.1, c[2] + radius + 0.1, 2.5e-3)
    else:  # the warp's gradient is at most 2 pi A / wavelength, so 0.75 steps never overshoot
        z, hit = _sphere_trace(phi_deformed, dirs, c[2] - radius - 0.1, c[2] + radius + 0.1, iters=400,
                               step=0.75)
    z = z + rng.normal(0.0, noise, z.shape) * hit
    if invalid_frac > 0:
        z[rng.random(z.shape) < invalid_frac] = 0.0
    depth = np.where(hit, z, 0.0).reshape(H, W)

    # canonical render: analytic ray/sphere intersection
    a = np.einsum("ij,ij->i", dirs, dirs)
    b = -2.0 * dirs @ c
    cc = c @ c - radius * radius
    disc = b * b - 4 * a * cc
    ok = disc > 0
    t = np.where(ok, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), 0.0)
    pts = t[:, None] * dirs
    ok &= t > 0
    src = pts[ok]
    nrm = (src - c) / radius

    m = min(n_sparse, src.shape[0])
    pick = rng.choice(src.shape[0], size=m, replace=False) if m > 0 else np.zeros(0, int)
    f_hat = src[pick]
    f_tgt = f_hat + disp(f_hat) + rng.normal(0.0, sparse_noise, f_hat.shape)

    dims, origin, h = lattice_for(n)
    return Frame(depth.astype(np.float32), K.astype(np.float32), _identity_pose(),
                 src.astype(np.float32), nrm.astype(np.float32),
                 f_hat.astype(np.float32).reshape(-1, 3), f_tgt.astype(np.float32).reshape(-1, 3),
                 dims, origin, h, name)


# ---------------------------------------------------------------------------
# articulated union of three capsules
# ---------------------------------------------------------------------------

def _capsule_sdf(x, a, b, r):
    ab = b - a
    t = np.clip(((x - a) @ ab) / (ab @ ab), 0.0, 1.0)
    q = a + t[..., None] * ab
    return np.linalg.norm(x - q, axis=-1) - r, q


class _Capsules:
    """Three capsules chained along x; joints 1 and 2 bent about axes normal to x."""

    def __init__(self, radii, angles, axes, seg=0.2, centre=(0.0, 0.0, 1.0)):
        c = np.asarray(centre, np.float64)
        ex = np.array([1.0, 0.0, 0.0])
        self.a = [c - 1.5 * seg * ex, c - 0.5 * seg * ex, c + 0.5 * seg * ex]
        self.b = [c - 0.5 * seg * ex, c + 0.5 * seg * ex, c + 1.5 * seg * ex]
        self.r = list(radii)
        self.J = [self.b[0], self.b[1]]
        self.Q = [_rotation(axes[0], angles[0]), np.eye(3), _rotation(axes[1], angles[1])]
        self.piv = [self.J[0], self.J[0], self.J[1]]

    def canon_sdf(self, x):
        return np.min([_capsule_sdf(x, self.a[k], self.b[k], self.r[k])[0] for k in range(3)], 0)

    def posed_sdf(self, y):
        out = []
        for k in range(3):
            x = self.piv[k] + (y - self.piv[k]) @ self.Q[k]       # Q^T (y - J) + J
            out.append(_capsule_sdf(x, self.a[k], self.b[k], self.r[k])[0])
        return np.min(out, 0)

    def canon_normal_and_segment(self, x):
        d = []
        qs = []
        for k in range(3):
            s, q = _capsule_sdf(x, self.a[k], self.b[k], self.r[k])
            d.append(s)
            qs.append(q)
        d = np.stack(d, 0)
        k = np.argmin(d, 0)
        q = np.stack(qs, 0)[k, np.arange(x.shape[0])]
        nrm = x - q
        nrm /= np.linalg.norm(nrm, axis=-1, keepdims=True)
        return nrm, k

    def pose_points(self, x, seg):
        y = np.empty_like(x)
        for k in range(3):
            m = seg == k
            y[m] = self.piv[k] + (x[m] - self.piv[k]) @ self.Q[k].T
        return y


def _capsules_torch(caps, which, dirs, device):
    """The same sphere tracing as _sphere_trace, of the posed or canonical capsules, in
    float64 torch on ``device`` (every ray takes every step; a ray that has converged or
    left the range keeps its z, which is what the numpy version's compaction does)."""
    import torch
    T = lambda a: torch.as_tensor(np.asarray(a, np.float64), device=device)
    d = T(dirs)
    parts = []
    for k in range(3):
        Q = caps.Q[k] if which == "posed" else np.eye(3)
        parts.append((T(caps.piv[k]), T(Q), T(caps.a[k]), T(caps.b[k]), float(caps.r[k])))

    def sdf(y):
        out = None
        for piv, Q, a, b, r in parts:
            x = piv + (y - piv) @ Q
            ab = b - a
            t = (((x - a) @ ab) / (ab @ ab)).clamp(0.0, 1.0)
            dist = torch.linalg.norm(x - (a + t[:, None] * ab), dim=1) - r
            out = dist if out is None else torch.minimum(out, dist)
        return out

    z0, z1, eps = 0.3, 1.6, 2e-6
    L = torch.linalg.norm(d, dim=1)
    z = torch.full((d.shape[0],), z0, dtype=torch.float64, device=device)
    live = torch.ones(d.shape[0], dtype=torch.bool, device=device)
    conv = torch.zeros_like(live)
    for it in range(160):
        if it % 8 == 0 and not bool(live.any()):
            break  # no ray left to step (further steps would change nothing)
        dist = sdf(z[:, None] * d)
        done = live & (dist < eps)
        conv |= done
        step = live & ~done
        z = torch.where(step, z + dist / L, z)
        live = step & (z < z1)
    lo = z
    hi = lo + 4 * eps / L + 1e-6
    for _ in range(8):
        out = conv & (sdf(hi[:, None] * d) > 0)
        hi = torch.where(out, hi + 1e-5, hi)
    conv &= sdf(hi[:, None] * d) <= 0
    for _ in range(40):
        m = 0.5 * (lo + hi)
        pos = sdf(m[:, None] * d) > 0
        lo = torch.where(pos, m, lo)
        hi = torch.where(pos, hi, m)
    zz = torch.where(conv, 0.5 * (lo + hi), torch.zeros_like(lo))
    return zz.cpu().numpy(), conv.cpu().numpy()


def _trace_capsules(caps, which, dirs, device):
    if device is None:
        return _sphere_trace(caps.posed_sdf if which == "posed" else caps.canon_sdf, dirs, 0.3, 1.6)
    return _capsules_torch(caps, which, dirs, device)


def _canonical_capsules(caps, dirs, device=None):
    """Canonical (unbent) surface samples seen by the camera: points, normals, segment."""
    zc, hitc = _trace_capsules(caps, "canon", dirs, device)
    src = zc[hitc, None] * dirs[hitc]
    nrm, seg = caps.canon_normal_and_segment(src)
    return src, nrm, seg


def capsule_frame(W=640, H=480, f=525.0, n=96, seed=0, angles=None, axes=None, radii=None,
                  rel_noise=0.005, invalid_frac=0.05, n_sparse=300, outlier_frac=0.05,
                  outlier_max=0.10, sparse_noise=1e-3, name="capsules", canon=None, device=None):
    """Three chained capsules (radii U(5, 15) cm) bent at two joints by U(10, 30) degrees.

    Depth noise N(0, (rel_noise * z)^2), ``invalid_frac`` of pixels dropped, sparse pairs
    with ``outlier_frac`` outliers displaced by a uniform length in [0, outlier_max] m.
    ``canon`` = the canonical samples of the same capsules (reused along a sequence; the
    result is the same as without it).  ``device`` = a torch CUDA device: trace the rays
    there (same algorithm in float64; depths agree with the numpy trace to rounding).
    """
    rng = np.random.default_rng(seed)
    if radii is None:
        radii = rng.uniform(0.05, 0.15, 3)
    if angles is None:
        angles = np.deg2rad(rng.uniform(10.0, 30.0, 2))
    if axes is None:
        phis = rng.uniform(0.0, 2 * math.pi, 2)
        axes = [np.array([0.0, math.cos(p), math.sin(p)]) for p in phis]
    caps = _Capsules(radii, angles, axes)
    K = _intrinsics(W, H, f)
    dirs = _rays(W, H, K)

    z, hit = _trace_capsules(caps, "posed", dirs, device)
    z = z + rng.normal(0.0, 1.0, z.shape) * rel_noise * z
    z[rng.random(z.shape) < invalid_frac] = 0.0
    depth = np.where(hit, z, 0.0).reshape(H, W)

    src, nrm, seg = canon if canon is not None else _canonical_capsules(caps, dirs, device)

    m = min(n_sparse, src.shape[0])
    pick = rng.choice(src.shape[0], size=m, replace=False) if m > 0 else np.zeros(0, int)
    f_hat = src[pick]
    f_tgt = caps.pose_points(f_hat, seg[pick]) + rng.normal(0.0, sparse_noise, f_hat.shape)
    n_out = int(round(outlier_frac * m))
    if n_out > 0:
        which = rng.choice(m, size=n_out, replace=False)
        dirv = rng.normal(size=(n_out, 3))
        dirv /= np.linalg.norm(dirv, axis=1, keepdims=True)
        f_tgt[which] += dirv * rng.uniform(0.0, outlier_max, (n_out, 1))

    dims, origin, h = lattice_for(n)
    return Frame(depth.astype(np.float32), K.astype(np.float32), _identity_pose(),
                 src.astype(np.float32), nrm.astype(np.float32),
                 f_hat.astype(np.float32).reshape(-1, 3), f_tgt.astype(np.float32).reshape(-1, 3),
                 dims, origin, h, name)


def plane_frame(W=32, H=24, f=30.0, n=8, depth=1.0, tilt_deg=0.0, shift=(0.0, 0.0, 0.0),
                noise=0.0, name="plane"):
    """A plane at ``depth`` tilted about the camera's y axis; source = the same plane.

    With ``shift`` = 0 and no noise the observed surface equals the canonical one.
    """
    K = _intrinsics(W, H, f)
    dirs = _rays(W, H, K)
    th = math.radians(tilt_deg)
    nrm = np.array([math.sin(th), 0.0, -math.cos(th)])       # faces the camera
    p0 = np.array([0.0, 0.0, depth])
    # canonical plane: n . (x - p0) = 0; observed plane: shifted by ``shift``
    t = (nrm @ p0) / (dirs @ nrm)
    src = t[:, None] * dirs
    p1 = p0 + np.asarray(shift, np.float64)
    t1 = (nrm @ p1) / (dirs @ nrm)
    dep = (t1 + (np.random.default_rng(0).normal(0, noise, t1.shape) if noise else 0.0))
    dims, origin, h = lattice_for(n)
    return Frame(dep.reshape(H, W).astype(np.float32), K.astype(np.float32), _identity_pose(),
                 src.astype(np.float32), np.tile(nrm, (src.shape[0], 1)).astype(np.float32),
                 np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32),
                 dims, origin, h, name)


def corner_frame(W=64, H=48, f=60.0, n=16, rot=None, shift=(0.0, 0.0, 0.0), vertex=(0.02, -0.03, 0.7),
                 step=2, margin=4, name="corner"):
    """A cube corner pointing at the camera -- the three faces around the vertex, whose
    outward normals each make the same angle (arccos 1/sqrt 3) with the view axis --
    moved by the rigid motion (rot, shift): x -> rot x + shift.  Source = the unmoved
    corner rendered by the same camera (every ``step``-th pixel), with the faces'
    normals, kept only at pixels at least ``margin`` pixels from a face edge or the
    silhouette (so that, for motions of a pixel or two, a sample's target pixel and its
    central-difference neighbours lie on its own face).  Point-to-plane residuals then
    vanish exactly at the true pose, and three independent planes fix all six pose
    parameters."""
    K = _intrinsics(W, H, f)
    dirs = _rays(W, H, K)
    Q = np.eye(3) if rot is None else np.asarray(rot, np.float64)
    c = np.asarray(shift, np.float64)
    # orthonormal outward normals with n_k . (0, 0, -1) = 1 / sqrt(3): the coordinate
    # axes turned so that (1, 1, 1) / sqrt(3) points at the camera
    a = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    b = np.array([0.0, 0.0, -1.0])
    v = np.cross(a, b)
    Kx = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    Ralign = np.eye(3) + Kx + Kx @ Kx / (1.0 + a @ b)
    nrm0 = (Ralign @ np.eye(3)).T                  # rows: the three outward normals
    C0 = np.asarray(vertex, np.float64)

    def render(Q, c):
        n_k = nrm0 @ Q.T                           # moved planes n_k . x = n_k . (Q C0 + c)
        d_k = n_k @ (Q @ C0 + c)
        den = dirs @ n_k.T
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(den < 0, d_k[None, :] / den, -np.inf)
        k = np.argmax(t, axis=1)                   # the ray enters the corner's solid last
        tt = t[np.arange(len(k)), k]
        p = tt[:, None] * dirs
        inside = np.all(p @ n_k.T <= d_k[None, :] + 1e-12, axis=1)
        ok = np.isfinite(tt) & (tt > 0) & inside
        return np.where(ok, tt, 0.0), k, n_k, ok

    t1, _, _, _ = render(Q, c)
    dep = (t1 * dirs[:, 2]).reshape(H, W)
    t0, k0, n0, ok0 = render(np.eye(3), np.zeros(3))
    pts = t0[:, None] * dirs
    face = np.where(ok0, k0, -1).reshape(H, W)
    same = np.ones((H, W), bool)
    for dy in range(-margin, margin + 1):
        for dx in range(-margin, margin + 1):
            sh = np.full((H, W), -2)
            ys, xs = slice(max(dy, 0), H + min(dy, 0)), slice(max(dx, 0), W + min(dx, 0))
            yd, xd = slice(max(-dy, 0), H + min(-dy, 0)), slice(max(-dx, 0), W + min(-dx, 0))
            sh[yd, xd] = face[ys, xs]
            same &= sh == face
    sel = np.zeros(H * W, bool)
    sel.reshape(H, W)[::step, ::step] = True
    sel &= ok0 & same.ravel()
    dims, origin, h = lattice_for(n)
    return Frame(dep.astype(np.float32), K.astype(np.float32), _identity_pose(),
                 pts[sel].astype(np.float32), n0[k0[sel]].astype(np.float32),
                 np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), dims, origin, h, name)


def sdf_grid(kind="sphere", n=64, seed=0, cube_min=(-0.5, -0.5, 0.5), cube_size=1.0, **kw):
    """Signed distance of a canonical surface (negative inside) on an n^3 grid of nodes
    over the 1 m cube, float32 array (z, y, x), with its origin and spacing: the input
    of the marching cubes.  kind "sphere": radius kw.get("radius", 0.3) at (0, 0, 1);
    "capsules": the unbent three-capsule surface of capsule_frame(seed)."""
    hs = cube_size / (n - 1)
    ax = np.asarray(cube_min, np.float64)[:, None] + hs * np.arange(n)[None, :]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    pts = np.stack([x, y, z], -1).reshape(-1, 3)
    if kind == "sphere":
        d = np.linalg.norm(pts - np.array([0.0, 0.0, 1.0]), axis=1) - kw.get("radius", 0.3)
    else:
        rng = np.random.default_rng(seed)
        radii = rng.uniform(0.05, 0.15, 3)
        caps = _Capsules(radii, [0.0, 0.0], [np.array([0.0, 0.0, 1.0])] * 2)
        d = caps.canon_sdf(pts)
    return d.reshape(n, n, n).astype(np.float32), np.asarray(cube_min, np.float64), hs


def config1(seed=0):
    """16^3 lattice, 64x48 depth (f = 60) of a bent 0.3 m sphere, 20 sparse pairs."""
    return sphere_frame(W=64, H=48, f=60.0, n=16, seed=seed, name="sphere16")


def config2(seed=0):
    """96^3 lattice, 640x480 depth (f = 525) of three bent capsules, 300 sparse pairs."""
    return capsule_frame(W=640, H=480, f=525.0, n=96, seed=seed, name="capsules96")


def batch_frames(count=32, base_seed=4, workers=1):
    """Lattices of uneven size: n ~ round(exp(U(ln 16, ln 96))), image 160s x 120s with
    s ~ logU(1, 4), sphere or capsules with probability 1/2, S ~ U{20..300}.
    ``workers`` > 1 renders the frames in a spawned process pool (same results)."""
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, count)) as pool:
            return pool.starmap(_batch_frame, [(k, base_seed) for k in range(count)])
    return [_batch_frame(k, base_seed) for k in range(count)]


def _batch_frame(k, base_seed):
    out = []
    for k in [k]:
        rng = np.random.default_rng([base_seed, k])
        n = int(round(math.exp(rng.uniform(math.log(16), math.log(96)))))
        s = math.exp(rng.uniform(0.0, math.log(4.0)))
        W, H = int(round(160 * s)), int(round(120 * s))
        f = 525.0 * W / 640.0
        S = int(rng.integers(20, 301))
        sub = int(rng.integers(0, 2**31 - 1))
        if rng.random() < 0.5:
            fr = sphere_frame(W=W, H=H, f=f, n=n, seed=sub, n_sparse=S, noise=2e-3,
                              name=f"batch{k}-sphere{n}", tracer="sphere")
        else:
            fr = capsule_frame(W=W, H=H, f=f, n=n, seed=sub, n_sparse=S,
                               name=f"batch{k}-capsules{n}")
        out.append(fr)
    return out[0]


def sequence_frames(seed, frames=64, n=96, W=640, H=480, f=525.0, max_step_deg=5.0, device=None):
    """Config-2 surfaces whose two bend angles random-walk by U(-5, 5) degrees per frame
    (reflected into [0, 30]); frame t's source samples are the canonical surface.
    ``device``: trace on that torch CUDA device (see capsule_frame)."""
    rng = np.random.default_rng(seed)
    radii = rng.uniform(0.05, 0.15, 3)
    phis = rng.uniform(0.0, 2 * math.pi, 2)
    axes = [np.array([0.0, math.cos(p), math.sin(p)]) for p in phis]
    ang = rng.uniform(10.0, 30.0, 2)
    canon = _canonical_capsules(_Capsules(radii, np.deg2rad(ang), axes), _rays(W, H, _intrinsics(W, H, f)), device)
    out = []
    for t in range(frames):
        if t > 0:
            ang = ang + rng.uniform(-max_step_deg, max_step_deg, 2)
            ang = np.abs(ang)
            ang = np.where(ang > 30.0, 60.0 - ang, ang)
        out.append(capsule_frame(W=W, H=H, f=f, n=n, seed=int(rng.integers(0, 2**31 - 1)),
                                 angles=np.deg2rad(ang), axes=axes, radii=radii,
                                 name=f"seq{seed}-{t}", canon=canon, device=device))
    return out


def sequences(seeds, frames=64, workers=1, device=None, **kw):
    """sequence_frames for several seeds, in a spawned process pool when workers > 1
    (or traced on a torch CUDA ``device`` in this process); yields (seed, frames) in the
    order of ``seeds``."""
    seeds = list(seeds)
    if device is not None:
        for s in seeds:
            yield s, sequence_frames(s, frames, device=device, **kw)
        return
    if workers <= 1:
        for s in seeds:
            yield s, sequence_frames(s, frames, **kw)
        return
    import functools
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(workers, len(seeds))) as pool:
        fn = functools.partial(sequence_frames, frames=frames, **kw)
        for s, fr in zip(seeds, pool.imap(fn, seeds)):
            yield s, fr
