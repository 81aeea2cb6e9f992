"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module only *creates inputs*: point clouds, Gaussian sets made directly
from a surface's analytic normals, cameras and the analytic scene description
that the oracle ray-caster reads.  It holds none of the renderer's or the
estimator's arithmetic (no projection, no compositing, no kNN, no PCA), so
both sides of every parity test can draw from it without sharing method code.

Conventions
-----------
* Gaussian set: dict of float32 numpy arrays
  ``mean (n,3)``, ``scale (n,3)`` (linear, > 0), ``quat (n,4)`` as
  ``(w, x, y, z)`` (raw, normalised by the renderer), ``opacity (n,)`` in
  [0, 1], ``rgb (n,3)``, ``normal (n,3)``.
* Camera: dict with ``viewmat`` float32 (3,4) row-major ``[T | t]`` mapping
  world to camera coordinates (OpenCV axes: x right, y down, z forward),
  ``fx, fy, cx, cy`` (pixels), ``width, height`` and ``near``.
* The humanoid proxy stands along world +y, feet at y = 0, head near y = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Primitive", "look_at_camera", "sphere_camera", "sphere_cloud",
    "humanoid_primitives", "sample_surface", "texture", "surface_gaussians",
    "humanoid_cloud", "deform_primitives", "circle_cameras",
]


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------
def look_at_camera(eye, target, up, fov_deg: float, width: int, height: int,
                   near: float = 0.01) -> dict:
    """Pinhole camera at ``eye`` looking at ``target``.

    ``up`` is the world direction that appears upwards in the image.  The
    vertical field of view is ``fov_deg``; fx = fy = (height/2)/tan(fov/2),
    principal point at the image centre (width/2, height/2).
    """
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    down = -np.asarray(up, np.float64)
    x = np.cross(down, f)
    if np.linalg.norm(x) < 1e-6:                    # looking along `up`
        alt = np.array([1.0, 0.0, 0.0]) if abs(f[0]) < 0.9 else np.array([0.0, 0.0, 1.0])
        x = np.cross(alt, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    rot = np.stack([x, y, f])                       # rows: camera axes in world
    t = -rot @ eye
    view = np.concatenate([rot, t[:, None]], axis=1).astype(np.float32)
    foc = (height / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return dict(viewmat=view, fx=float(foc), fy=float(foc), cx=width / 2.0,
                cy=height / 2.0, width=int(width), height=int(height),
                near=float(near))


def sphere_camera(center, radius: float, rng: np.random.Generator,
                  width: int, height: int, fov_deg: float = 60.0) -> dict:
    """Camera placed uniformly at random on a sphere, looking at ``center``."""
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    eye = np.asarray(center, np.float64) + radius * d
    return look_at_camera(eye, center, (0.0, 1.0, 0.0), fov_deg, width, height)


def circle_cameras(center, radius: float, n: int, width: int, height: int,
                   fov_deg: float = 60.0, elevation: float = 0.0) -> list:
    """``n`` cameras on a horizontal circle around ``center`` (12 views in the
    paper's evaluation protocol, Sec. 4.1)."""
    cams = []
    for k in range(n):
        a = 2.0 * math.pi * k / n
        eye = np.asarray(center, np.float64) + np.array(
            [radius * math.cos(a), elevation, radius * math.sin(a)])
        cams.append(look_at_camera(eye, center, (0.0, 1.0, 0.0), fov_deg, width, height))
    return cams


# ----------------------------------------------------------------------------
# config 1: points on a unit sphere
# ----------------------------------------------------------------------------
def sphere_cloud(n: int = 4096, seed: int = 1, scale: float = 0.02,
                 opacity: float = 0.8) -> dict:
    """Uniform points on the unit sphere, isotropic Gaussians.

    rgb = 0.5 + 0.5 sin(3 xyz), identity quaternion, radial normal.
    """
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((n, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    p = p.astype(np.float32)
    return dict(
        mean=p,
        scale=np.full((n, 3), scale, np.float32),
        quat=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
        opacity=np.full((n,), opacity, np.float32),
        rgb=(0.5 + 0.5 * np.sin(3.0 * p)).astype(np.float32),
        normal=p.copy(),
    )


# ----------------------------------------------------------------------------
# analytic humanoid proxy (ellipsoids and capped cylinders)
# ----------------------------------------------------------------------------
@dataclass
class Primitive:
    """An ellipsoid (``kind='ell'``: centre, radii, rotation matrix whose
    columns are the local axes) or a capped cylinder (``kind='cyl'``: axis
    from ``p0`` to ``p1``, radius ``r``, closed by two flat disks)."""
    kind: str
    center: np.ndarray = field(default_factory=lambda: np.zeros(3))
    radii: np.ndarray = field(default_factory=lambda: np.ones(3))
    rot: np.ndarray = field(default_factory=lambda: np.eye(3))
    p0: np.ndarray = field(default_factory=lambda: np.zeros(3))
    p1: np.ndarray = field(default_factory=lambda: np.zeros(3))
    r: float = 0.0

    def area(self, rng: np.random.Generator) -> float:
        if self.kind == "cyl":
            h = float(np.linalg.norm(self.p1 - self.p0))
            return 2.0 * math.pi * self.r * h + 2.0 * math.pi * self.r ** 2
        u = _unit_sphere(rng, 200_000)
        a, b, c = self.radii
        g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
        return float(4.0 * math.pi * g.mean())

    def inside(self, p: np.ndarray) -> np.ndarray:
        """Strictly inside (open set)."""
        if self.kind == "ell":
            q = (p - self.center) @ self.rot / self.radii
            return (q * q).sum(1) < 1.0
        ax = self.p1 - self.p0
        h = np.linalg.norm(ax)
        ax = ax / h
        d = p - self.p0
        s = d @ ax
        rad = np.linalg.norm(d - s[:, None] * ax, axis=1)
        return (s > 0) & (s < h) & (rad < self.r)

    def sample(self, rng: np.random.Generator, n: int):
        """``n`` points uniform by area on the surface, with outward normals."""
        if self.kind == "ell":
            a, b, c = self.radii
            gmax = max(b * c, a * c, a * b)
            pts, nrm = [], []
            got = 0
            while got < n:
                u = _unit_sphere(rng, max(2 * (n - got), 1024))
                g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
                keep = rng.random(len(u)) * gmax < g
                u = u[keep]
                loc = u * self.radii
                nl = u / self.radii
                nl /= np.linalg.norm(nl, axis=1, keepdims=True)
                pts.append(loc @ self.rot.T + self.center)
                nrm.append(nl @ self.rot.T)
                got += len(u)
            return np.concatenate(pts)[:n], np.concatenate(nrm)[:n]
        ax = self.p1 - self.p0
        h = float(np.linalg.norm(ax))
        e3 = ax / h
        e1 = np.cross(e3, [1.0, 0.0, 0.0])
        if np.linalg.norm(e1) < 1e-3:
            e1 = np.cross(e3, [0.0, 0.0, 1.0])
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(e3, e1)
        a_tube = 2.0 * math.pi * self.r * h
        a_disk = math.pi * self.r ** 2
        which = rng.choice(3, size=n, p=np.array([a_tube, a_disk, a_disk]) / (a_tube + 2 * a_disk))
        th = rng.random(n) * 2.0 * math.pi
        pts = np.empty((n, 3))
        nrm = np.empty((n, 3))
        t = which == 0
        s = rng.random(n) * h
        radial = np.cos(th)[:, None] * e1 + np.sin(th)[:, None] * e2
        pts[t] = self.p0 + s[t, None] * e3 + self.r * radial[t]
        nrm[t] = radial[t]
        rr = self.r * np.sqrt(rng.random(n))
        for k, base, nn in ((1, self.p0, -e3), (2, self.p1, e3)):
            m = which == k
            pts[m] = base + rr[m, None] * radial[m]
            nrm[m] = nn
        return pts, nrm


def _unit_sphere(rng, n):
    u = rng.standard_normal((n, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def _rot_axis(axis, ang):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    k = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * k + (1 - math.cos(ang)) * (k @ k)


def humanoid_primitives(seed: int | None = None, jitter: float = 0.0) -> list:
    """12 primitives forming a 1 m tall human proxy.

    With ``jitter > 0`` the sizes and limb poses are perturbed by a seeded
    relative amount (used for the many-scene training set).
    """
    rng = np.random.default_rng(seed)

    def j(x):
        return x * (1.0 + jitter * (2.0 * rng.random() - 1.0)) if jitter else x

    def v(*a):
        return np.array(a, np.float64)

    prims = [
        Primitive("ell", center=v(0, 0.915, 0), radii=v(j(0.070), j(0.085), j(0.078))),  # head
        Primitive("cyl", p0=v(0, 0.79, 0), p1=v(0, 0.845, 0), r=j(0.035)),               # neck
        Primitive("ell", center=v(0, 0.675, 0), radii=v(j(0.155), j(0.140), j(0.090))),  # torso
        Primitive("ell", center=v(0, 0.515, 0), radii=v(j(0.135), j(0.075), j(0.088))),  # pelvis
    ]
    limbs = []
    for sgn in (-1.0, 1.0):
        sh = v(sgn * 0.175, 0.775, 0.0)
        el = v(sgn * j(0.215), 0.600, j(0.01) if jitter else 0.0)
        wr = v(sgn * j(0.245), 0.440, j(0.03))
        hp = v(sgn * 0.078, 0.50, 0.0)
        kn = v(sgn * j(0.088), 0.270, j(0.01) if jitter else 0.0)
        an = v(sgn * j(0.092), 0.035, 0.0)
        if jitter:  # seeded pose: swing each limb about its proximal joint
            el = sh + _rot_axis([1, 0, 0], jitter * 2.0 * (rng.random() - 0.5)) @ (el - sh)
            wr = el + _rot_axis([1, 0, 0], jitter * 3.0 * (rng.random() - 0.5)) @ (wr - el)
            kn = hp + _rot_axis([1, 0, 0], jitter * 1.5 * (rng.random() - 0.5)) @ (kn - hp)
            an = kn + _rot_axis([1, 0, 0], jitter * 1.5 * (rng.random() - 0.5)) @ (an - kn)
        limbs += [
            Primitive("cyl", p0=sh, p1=el, r=j(0.036)),   # upper arm
            Primitive("cyl", p0=el, p1=wr, r=j(0.030)),   # forearm
            Primitive("cyl", p0=hp, p1=kn, r=j(0.056)),   # thigh
            Primitive("cyl", p0=kn, p1=an, r=j(0.041)),   # shin
        ]
    return prims + limbs


def limb_motion(prims: list, t: float, amp: float = 0.35, period: float = 4.0) -> list:
    """Per primitive the rigid motion ``x -> b + R (x - a)``, as ``(R, a, b)``,
    that swings the limbs sinusoidally about their proximal joints at time
    ``t`` (s); identity for head, neck, torso and pelvis.  Joint chains
    follow the primitive order of :func:`humanoid_primitives` (upper arm,
    forearm, thigh, shin per side)."""
    eye = np.eye(3)
    out = [(eye, np.zeros(3), np.zeros(3)) for _ in prims]
    w = 2.0 * math.pi * t / period
    for side in range(2):
        base = 4 + 4 * side
        ua, fa, th, sh = prims[base], prims[base + 1], prims[base + 2], prims[base + 3]
        ph = math.pi * side
        r1 = _rot_axis([1, 0, 0], amp * math.sin(w + ph))
        r2 = _rot_axis([1, 0, 0], 0.5 * amp * math.sin(w + ph + 0.7))
        r3 = _rot_axis([1, 0, 0], -amp * math.sin(w + ph))
        r4 = _rot_axis([1, 0, 0], 0.5 * amp * (1 + math.sin(w + ph + 0.5)))
        el = ua.p0 + r1 @ (ua.p1 - ua.p0)          # moved elbow
        kn = th.p0 + r3 @ (th.p1 - th.p0)          # moved knee
        out[base] = (r1, ua.p0, ua.p0)
        out[base + 1] = (r1 @ r2, fa.p0, el)
        out[base + 2] = (r3, th.p0, th.p0)
        out[base + 3] = (r3 @ r4, sh.p0, kn)
    return out


def deform_primitives(prims: list, t: float, amp: float = 0.35,
                      period: float = 4.0) -> list:
    """The primitives moved by :func:`limb_motion` at time ``t`` (s)."""
    out = []
    for p, (R, a, b) in zip(prims, limb_motion(prims, t, amp, period)):
        q = Primitive(p.kind, p.center.copy(), p.radii.copy(), p.rot.copy(), p.p0.copy(), p.p1.copy(), p.r)
        if p.kind == "cyl":
            q.p0, q.p1 = b + R @ (p.p0 - a), b + R @ (p.p1 - a)
        out.append(q)
    return out


class DynamicCloud:
    """A moving, resampled humanoid point-cloud video.

    One ``n_max``-point coloured sample of the rest pose is drawn once; frame
    ``k`` of ``frames`` (spread over one ``period``) keeps the first
    ``n(t) = mid + amp sin(2 pi t / period)`` points of a fixed random
    permutation (a uniform subsample, so the point count swings between the
    ends of ``n_range``) and moves each point with its primitive's limb
    motion at ``t = k period / frames``.  Colours travel with the surface.
    """

    def __init__(self, n_range=(300_000, 1_200_000), seed: int = 0, frames: int = 16, period: float = 4.0):
        self.prims = humanoid_primitives()
        lo, hi = int(n_range[0]), int(n_range[1])
        pts, _, pid = sample_surface(self.prims, hi, seed)
        rng = np.random.default_rng(seed + 1)
        perm = rng.permutation(hi)
        self.pts, self.pid = pts[perm], pid[perm]
        self.rgb = texture(self.pts).astype(np.float32)
        self.frames, self.period = int(frames), float(period)
        self.mid, self.amp = (lo + hi) / 2.0, (hi - lo) / 2.0

    def time_of(self, k: int) -> float:
        return (k % self.frames) * self.period / self.frames

    def count(self, k: int) -> int:
        return int(round(self.mid + self.amp * math.sin(2.0 * math.pi * self.time_of(k) / self.period)))

    def frame(self, k: int):
        """``(xyz float32 (n,3), rgb float32 (n,3))`` of frame ``k``."""
        n = self.count(k)
        x, pid = self.pts[:n], self.pid[:n]
        out = x.copy()
        for i, (R, a, b) in enumerate(limb_motion(self.prims, self.time_of(k))):
            m = pid == i
            if m.any():
                out[m] = b + (x[m] - a) @ R.T
        return out.astype(np.float32), self.rgb[:n]


def sample_surface(prims: list, n: int, seed: int, noise: float = 1e-3):
    """``n`` points uniform by area on the boundary of the primitives' union.

    Each primitive gets an area-proportional share of an oversampled set;
    points inside any other primitive are dropped; ``n`` survivors are drawn
    uniformly; N(0, ``noise``) position noise is added.  Returns float64
    ``(points, normals, prim_id)`` where normals are the exact outward
    normals before noise.
    """
    rng = np.random.default_rng(seed)
    areas = np.array([p.area(rng) for p in prims])
    share = areas / areas.sum()
    over = 1.8
    pts, nrm, pid = [], [], []
    for k, p in enumerate(prims):
        m = int(math.ceil(over * n * share[k])) + 16
        x, nn = p.sample(rng, m)
        keep = np.ones(len(x), bool)
        for q_i, q in enumerate(prims):
            if q_i != k:
                keep &= ~q.inside(x)
        pts.append(x[keep])
        nrm.append(nn[keep])
        pid.append(np.full(keep.sum(), k, np.int32))
    pts = np.concatenate(pts)
    nrm = np.concatenate(nrm)
    pid = np.concatenate(pid)
    if len(pts) < n:
        raise RuntimeError("oversampling too small for the union boundary")
    sel = rng.choice(len(pts), size=n, replace=False)
    sel.sort()
    pts = pts[sel] + noise * rng.standard_normal((n, 3))
    return pts, nrm[sel], pid[sel]


def texture(points: np.ndarray, seed: int = 7) -> np.ndarray:
    """Smooth 3D colour field in [0,1]^3: per channel a sum of 8 seeded
    random-direction sinusoids squashed by a logistic."""
    rng = np.random.default_rng(10_000 + seed)
    p = np.asarray(points, np.float64)
    out = np.empty((len(p), 3))
    for ch in range(3):
        d = _unit_sphere(rng, 8)
        f = 6.0 + 34.0 * rng.random(8)
        ph = 2.0 * math.pi * rng.random(8)
        s = np.sin((p @ d.T) * f + ph).sum(1) / math.sqrt(8.0)
        out[:, ch] = 1.0 / (1.0 + np.exp(-2.0 * s))
    return out


def _quat_from_z(nrm: np.ndarray) -> np.ndarray:
    """Unit quaternions (w,x,y,z) whose rotation maps +z onto ``nrm``."""
    z = np.array([0.0, 0.0, 1.0])
    n = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    c = n @ z
    ax = np.cross(np.broadcast_to(z, n.shape), n)
    q = np.concatenate([(1.0 + c)[:, None], ax], axis=1)
    flip = c < -0.999999
    q[flip] = [0.0, 1.0, 0.0, 0.0]
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def surface_gaussians(points, normals, rgb, spacing: float, rng=None,
                      opacity: float = 0.9, flat: float = 0.1) -> dict:
    """Gaussians built straight from a surface sample: tangent disks of radius
    ``spacing`` (``flat`` times thinner along the normal), oriented by the
    sample's analytic normal with a seeded random spin about it."""
    n = len(points)
    q = _quat_from_z(normals)
    if rng is not None:                       # random spin about the normal
        ang = rng.random(n) * 2.0 * math.pi
        spin = np.stack([np.cos(ang / 2), 0 * ang, 0 * ang, np.sin(ang / 2)], 1)
        w1, x1, y1, z1 = q.T
        w2, x2, y2, z2 = spin.T
        q = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                      w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                      w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                      w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)
    scale = np.tile([spacing, spacing, flat * spacing], (n, 1))
    if rng is not None:
        scale = scale * (0.8 + 0.4 * rng.random((n, 3)))
    return dict(
        mean=np.asarray(points, np.float32),
        scale=scale.astype(np.float32),
        quat=q.astype(np.float32),
        opacity=np.full((n,), opacity, np.float32),
        rgb=np.asarray(rgb, np.float32),
        normal=(normals / np.linalg.norm(normals, axis=1, keepdims=True)).astype(np.float32),
    )


def humanoid_cloud(n: int, seed: int, prims=None, noise: float = 1e-3):
    """Coloured point cloud on the humanoid proxy.

    Returns ``(xyz float32 (n,3), rgb float32 (n,3), normals float64 (n,3),
    prims)``.
    """
    if prims is None:
        prims = humanoid_primitives()
    pts, nrm, _ = sample_surface(prims, n, seed, noise)
    rgb = texture(pts)
    return pts.astype(np.float32), rgb.astype(np.float32), nrm, prims


def quantize_cloud(xyz, rgb, alpha: float = 1.0, bits: int = 10):
    """Voxelised input as in the paper's training data (Sec. 3.3): the cloud
    is normalised into the 2 x 2 x 2 box centred at the origin (its largest
    extent fills the box), coordinates are scaled by 2^(bits - 1) (512 for
    10 bits) and rounded to integers; ``alpha`` in (0, 1] further coarsens
    them (round(alpha x) / alpha, the density augmentation of quantised
    inputs).  Points falling into one voxel merge (mean colour).  Returns
    float32 ``(xyz, rgb)`` back in the cloud's original frame."""
    p = np.asarray(xyz, np.float64)
    lo, hi = p.min(0), p.max(0)
    c = 0.5 * (lo + hi)
    s = 2.0 / max(float((hi - lo).max()), 1e-12)
    u = (p - c) * s * 2.0 ** (bits - 1)              # in [-512, 512] for 10 bits
    q = np.round(alpha * u).astype(np.int64)           # voxel ids at the (alpha-coarsened) step
    _, first, inv, cnt = np.unique(q, axis=0, return_index=True, return_inverse=True, return_counts=True)
    inv = inv.reshape(-1)
    col = np.zeros((len(first), 3))
    np.add.at(col, inv, np.asarray(rgb, np.float64))
    col /= cnt[:, None]
    grid = q[first].astype(np.float64) / alpha         # back to the 10-bit scale
    out = grid / 2.0 ** (bits - 1) / s + c
    return out.astype(np.float32), col.astype(np.float32)


def subsample_cloud(xyz, rgb, beta: float, seed: int):
    """Random subset of round(beta N) points (the density augmentation of
    non-quantised inputs, Sec. 3.3)."""
    rng = np.random.default_rng(seed)
    n = len(xyz)
    k = max(17, int(round(beta * n)))
    idx = np.sort(rng.choice(n, size=min(k, n), replace=False))
    return np.asarray(xyz, np.float32)[idx], np.asarray(rgb, np.float32)[idx]


def mean_spacing(n: int, prims, rng=None) -> float:
    """Average point spacing sqrt(area / n) of an n-point sample on ``prims``."""
    rng = rng or np.random.default_rng(0)
    area = sum(p.area(rng) for p in prims)
    return math.sqrt(area / n)


# ----------------------------------------------------------------------------
# ground-truth views of the analytic scenes (training targets)
# ----------------------------------------------------------------------------
def gt_views(prims: list, cams: list, bg=(0.0, 0.0, 0.0)) -> list:
    """Ray-cast views of the union of the primitives: per camera a dict with
    planar ``rgb (3,H,W)`` (the scene texture at the hit), outward ``normal
    (3,H,W)``, camera ``depth (H,W)`` and coverage ``hit (H,W)``.  One ray per
    pixel centre, nearest positive hit over every primitive surface (the
    first surface a ray meets is on the union's boundary).  These are
    synthetic inputs, the stand-in for images rasterised from meshes."""
    out = []
    for cam in cams:
        V = np.asarray(cam["viewmat"], np.float64)
        T, t = V[:, :3], V[:, 3]
        W, H = cam["width"], cam["height"]
        f32 = lambda k: float(np.float32(cam[k]))  # noqa: E731
        ii, jj = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
        dc = np.stack([(ii - f32("cx")) / f32("fx"), (jj - f32("cy")) / f32("fy"), np.ones_like(ii)], -1)
        d = dc.reshape(-1, 3) @ T               # T^T dc, camera z of the ray = 1
        o = -T.T @ t
        tb = np.full(len(d), np.inf)
        nb = np.zeros((len(d), 3))
        for p in prims:
            if p.kind == "ell":
                R = np.asarray(p.rot, np.float64)
                ol = (R.T @ (o - p.center)) / p.radii
                dl = (d @ R) / p.radii
                a = (dl * dl).sum(1)
                b = 2 * dl @ ol
                c = ol @ ol - 1
                disc = b * b - 4 * a * c
                ok = disc >= 0
                sq = np.sqrt(np.where(ok, disc, 0))
                t1 = (-b - sq) / (2 * a)
                t2 = (-b + sq) / (2 * a)
                tt = np.where(t1 > 0, t1, t2)
                use = ok & (tt > 0) & (tt < tb)
                g = (ol[None, :] + tt[:, None] * dl) / p.radii
                n = g @ R.T
                n /= np.linalg.norm(n, axis=1, keepdims=True) + 1e-300
                tb = np.where(use, tt, tb)
                nb[use] = n[use]
            else:
                ax = p.p1 - p.p0
                h = np.linalg.norm(ax)
                ax = ax / h
                w = o - p.p0
                wa, da = w @ ax, d @ ax
                wp = w - wa * ax
                dp = d - da[:, None] * ax
                A = (dp * dp).sum(1)
                B = 2 * dp @ wp
                Cc = wp @ wp - p.r ** 2
                disc = B * B - 4 * A * Cc
                ok = (disc >= 0) & (A > 0)
                sq = np.sqrt(np.where(ok, disc, 0))
                Aq = np.where(A > 0, A, 1.0)
                for tt in ((-B - sq) / (2 * Aq), (-B + sq) / (2 * Aq)):
                    s = wa + tt * da
                    use = ok & (tt > 0) & (tt < tb) & (s >= 0) & (s <= h)
                    n = (wp[None, :] + tt[:, None] * dp) / p.r
                    tb = np.where(use, tt, tb)
                    nb[use] = n[use]
                    ok = ok & ~use
                with np.errstate(divide="ignore", invalid="ignore"):
                    for s_end, sgn in ((0.0, -1.0), (h, 1.0)):
                        tt = (s_end - wa) / da
                        q = wp[None, :] + tt[:, None] * dp
                        use = (da != 0) & (tt > 0) & (tt < tb) & ((q * q).sum(1) <= p.r ** 2)
                        tb = np.where(use, tt, tb)
                        nb[use] = sgn * ax
        hit = np.isfinite(tb)
        pts = o + np.where(hit, tb, 0)[:, None] * d
        rgb = np.tile(np.asarray(bg, np.float64), (len(d), 1))
        if hit.any():
            rgb[hit] = texture(pts[hit])
        out.append(dict(rgb=rgb.T.reshape(3, H, W), normal=nb.T.reshape(3, H, W),
                        depth=np.where(hit, tb, 0).reshape(H, W), hit=hit.reshape(H, W)))
    return out
