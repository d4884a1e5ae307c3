"""Seeded synthetic scenes, meshes and hypothesis sets for the PERCH 2.0 scorer.

This module makes inputs only. It holds none of the scoring arithmetic (no
rasterisation, no back-projection, no neighbour search, no colour difference):
observations are made by analytic ray casting of the primitive shapes in
float64, and poses are composed in float64 and rounded once to float32. Both the
CUDA path and the CPU oracle receive exactly the arrays built here.

Workloads (the paper's datasets are not available; these stand in for them):

* ``tabletop_small``  - 3-DoF, one 6x8x12 cm box (516 triangles) on a table,
  160x120 camera, fx=fy=150, 11x11 positions (2 cm) x 8 yaws = 968 hypotheses,
  delta = 1 cm, colour check off, depth noise N(0, 2 mm).  (Sec. VI-A setting,
  reduced.)
* ``tabletop_3obj``   - 3-DoF, an ellipsoid (20k triangles) and two cylinders of
  the same shape but different colour (10k triangles each) on a table, 640x480,
  fx=fy=615, depth noise N(0, 3 mm), 20 % random occluder pixels, 43x43
  positions (1 cm) x 16 yaws = 29,584 hypotheses per object around the ground
  truth (on the grid), colour check on.  (Sec. VI-A: same-shape objects of
  different colour, occlusion.)
* ``sixdof_5obj``     - 6-DoF, five 30k-triangle meshes at 0.7-1.0 m in front of
  a wall, labels from perturbed ground-truth masks, ROI = mask bounding box,
  4,096 hypotheses per object = GT + N(0, 2 cm) translation + N(0, 15 deg)
  rotation.  (Sec. V: label-based admissible set and occluders.)

Pose convention: float32 row-major 3x4 [R | t], object frame -> camera frame
(OpenCV camera: x right, y down, z forward), metres.  Depth: uint16 in 0.1 mm
units, 0 = no return.  Labels: int32, object index or -1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DEPTH_SCALE = 10000.0  # depth units per metre (0.1 mm)


# --------------------------------------------------------------------------
# small float64 geometry helpers (input construction only)
# --------------------------------------------------------------------------

def rot_z(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rodrigues(axis: np.ndarray, theta: float) -> np.ndarray:
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    k = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(theta) * k + (1.0 - math.cos(theta)) * (k @ k)


def rodrigues_batch(axes: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Rotation matrices (n,3,3) about unit(axes) by theta, float64."""
    a = axes / np.linalg.norm(axes, axis=1, keepdims=True)
    k = np.zeros((len(a), 3, 3))
    k[:, 0, 1], k[:, 0, 2] = -a[:, 2], a[:, 1]
    k[:, 1, 0], k[:, 1, 2] = a[:, 2], -a[:, 0]
    k[:, 2, 0], k[:, 2, 1] = -a[:, 1], a[:, 0]
    s, c = np.sin(theta)[:, None, None], np.cos(theta)[:, None, None]
    return np.eye(3)[None] + s * k + (1.0 - c) * (k @ k)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def look_at(dist: float, elev_deg: float, target=(0.0, 0.0, 0.05)):
    """World (table, z up) -> camera (OpenCV) rotation and translation, float64."""
    el = math.radians(elev_deg)
    target = np.asarray(target, np.float64)
    cam = target + dist * np.array([0.0, -math.cos(el), math.sin(el)])
    fwd = (target - cam) / np.linalg.norm(target - cam)
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    r_wc = np.stack([right, down, fwd])
    t_wc = -r_wc @ cam
    return r_wc, t_wc


def pose_rows(r_oc: np.ndarray, t_oc: np.ndarray) -> np.ndarray:
    """Pack an object->camera pose as 12 float64 values (row-major [R|t])."""
    return np.concatenate([r_oc, t_oc[:, None]], axis=1).reshape(12)


def tabletop_pose(r_wc, t_wc, x, y, yaw) -> np.ndarray:
    r_ow = rot_z(yaw)
    t_ow = np.array([x, y, 0.0])
    return pose_rows(r_wc @ r_ow, r_wc @ t_ow + t_wc)


# --------------------------------------------------------------------------
# procedural colour functions: smooth, asymmetric under yaw
# --------------------------------------------------------------------------

def _u8(c: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(c), 0, 255).astype(np.uint8)


def colour_gradient(extent, base=(60.0, 60.0, 60.0), span=(180.0, 180.0, 180.0), order=(1, 2, 0)):
    """RGB that ramps linearly along the object's axes (no symmetry)."""
    lo = np.array([-extent[0] / 2, -extent[1] / 2, 0.0])
    size = np.array(extent, np.float64)

    def fn(p):
        f = (p - lo) / size
        f = np.clip(f, 0.0, 1.0)
        return np.stack([base[i] + span[i] * f[:, order[i]] for i in range(3)], axis=1)
    return fn


def colour_wheel(hue0: float, sat: float, val: float, height: float, radius: float | None = None,
                 turns: int = 1):
    """RGB from the angle around the z axis (`turns` hue turns per revolution,
    negative: the hue runs the other way round) plus a height ramp.  With a
    radius, the saturation fades linearly to grey towards the axis (full at
    the radius), so that the end caps' vertex colours -- a fan around a centre
    vertex -- interpolate to the same colour the ray caster sees."""
    def fn(p):
        ang = np.arctan2(p[:, 1], p[:, 0])
        hue = (turns * ang / (2 * math.pi) + hue0) % 1.0
        v = val * (0.75 + 0.25 * np.clip(p[:, 2] / height, 0.0, 1.0))
        s = sat if radius is None else sat * np.clip(np.hypot(p[:, 0], p[:, 1]) / radius, 0.0, 1.0)
        k = (np.array([5.0, 3.0, 1.0])[None, :] + hue[:, None] * 6.0) % 6.0
        rgb = v[:, None] - (v * s)[:, None] * np.clip(np.minimum(k, 4.0 - k), 0.0, 1.0)
        return 255.0 * rgb
    return fn


# --------------------------------------------------------------------------
# meshes (object frame, z up, base on z = 0)
# --------------------------------------------------------------------------

@dataclass
class Mesh:
    name: str
    verts: np.ndarray          # (V,3) float32
    rgb: np.ndarray            # (V,3) uint8
    tris: np.ndarray           # (T,3) int32
    vol_radius: float          # admissible cylinder V(O): radius about z
    vol_height: float          # admissible cylinder V(O): height from z = 0
    shape: tuple = ()          # analytic description for ray casting
    colour_fn: object = field(default=None, repr=False)

    @property
    def n_tris(self):
        return int(self.tris.shape[0])


def _finish(name, v, t, colour_fn, vol_r, vol_h, shape):
    v = np.asarray(v, np.float64)
    return Mesh(name, v.astype(np.float32), _u8(colour_fn(v)), np.asarray(t, np.int32),
                float(vol_r), float(vol_h), shape, colour_fn)


def _grid_face(origin, du, dv, nu, nv, verts, tris):
    base = len(verts)
    for j in range(nv + 1):
        for i in range(nu + 1):
            verts.append(origin + du * (i / nu) + dv * (j / nv))
    for j in range(nv):
        for i in range(nu):
            a = base + j * (nu + 1) + i
            b, c, d = a + 1, a + nu + 1, a + nu + 2
            tris.append((a, b, d))
            tris.append((a, d, c))


def box_mesh(sx, sy, sz, nx, ny, nz, colour_fn=None, name="box", vol_r=None, vol_h=None):
    """Closed box [-sx/2,sx/2]x[-sy/2,sy/2]x[0,sz]; each face an nu x nv grid."""
    colour_fn = colour_fn or colour_gradient((sx, sy, sz))
    verts, tris = [], []
    x0, y0 = -sx / 2, -sy / 2
    ex, ey, ez = np.array([sx, 0, 0.0]), np.array([0, sy, 0.0]), np.array([0, 0, sz])
    o = np.array([x0, y0, 0.0])
    _grid_face(o, ex, ey, nx, ny, verts, tris)                 # bottom
    _grid_face(o + ez, ex, ey, nx, ny, verts, tris)            # top
    _grid_face(o, ex, ez, nx, nz, verts, tris)                 # front (y = y0)
    _grid_face(o + ey, ex, ez, nx, nz, verts, tris)            # back
    _grid_face(o, ey, ez, ny, nz, verts, tris)                 # left (x = x0)
    _grid_face(o + ex, ey, ez, ny, nz, verts, tris)            # right
    vol_r = min(sx, sy) / 2 if vol_r is None else vol_r
    vol_h = sz if vol_h is None else vol_h
    return _finish(name, np.array(verts), tris, colour_fn, vol_r, vol_h, ("box", sx, sy, sz))


def cylinder_mesh(r, h, nseg, nrow, colour_fn=None, name="cylinder"):
    """Closed cylinder x^2+y^2<=r^2, 0<=z<=h: nseg x nrow side quads and two fans."""
    colour_fn = colour_fn or colour_wheel(0.0, 0.7, 0.9, h)
    verts, tris = [], []
    for j in range(nrow + 1):
        z = h * j / nrow
        for i in range(nseg):
            a = 2 * math.pi * i / nseg
            verts.append((r * math.cos(a), r * math.sin(a), z))
    for j in range(nrow):
        for i in range(nseg):
            a = j * nseg + i
            b = j * nseg + (i + 1) % nseg
            tris.append((a, b, b + nseg))
            tris.append((a, b + nseg, a + nseg))
    for z, ring in ((0.0, 0), (h, nrow)):
        c = len(verts)
        verts.append((0.0, 0.0, z))
        for i in range(nseg):
            a = ring * nseg + i
            b = ring * nseg + (i + 1) % nseg
            tris.append((c, b, a) if z == 0.0 else (c, a, b))
    return _finish(name, np.array(verts), tris, colour_fn, r, h, ("cylinder", r, h))


def ellipsoid_mesh(a, b, c, nlat, nlon, colour_fn=None, name="ellipsoid", vol_r=None, vol_h=None):
    """Ellipsoid with semi-axes (a,b,c) centred at (0,0,c): a UV sphere, scaled."""
    colour_fn = colour_fn or colour_gradient((2 * a, 2 * b, 2 * c), order=(2, 0, 1))
    verts, tris = [(0.0, 0.0, 0.0)], []
    for j in range(1, nlat):
        th = math.pi * j / nlat
        for i in range(nlon):
            ph = 2 * math.pi * i / nlon
            verts.append((a * math.sin(th) * math.cos(ph), b * math.sin(th) * math.sin(ph),
                          c - c * math.cos(th)))
    top = len(verts)
    verts.append((0.0, 0.0, 2 * c))
    ring = lambda j, i: 1 + (j - 1) * nlon + (i % nlon)
    for i in range(nlon):
        tris.append((0, ring(1, i + 1), ring(1, i)))
        tris.append((top, ring(nlat - 1, i), ring(nlat - 1, i + 1)))
    for j in range(1, nlat - 1):
        for i in range(nlon):
            p, q = ring(j, i), ring(j, i + 1)
            r_, s = ring(j + 1, i), ring(j + 1, i + 1)
            tris.append((p, q, s))
            tris.append((p, s, r_))
    vol_r = min(a, b) * 0.7 if vol_r is None else vol_r
    vol_h = 2 * c if vol_h is None else vol_h
    return _finish(name, np.array(verts), tris, colour_fn, vol_r, vol_h, ("ellipsoid", a, b, c))


# --------------------------------------------------------------------------
# analytic ray casting (float64) for observations
# --------------------------------------------------------------------------

def _hit_box(o, d, sx, sy, sz):
    lo = np.array([-sx / 2, -sy / 2, 0.0])
    hi = np.array([sx / 2, sy / 2, sz])
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (lo - o) * inv
        t2 = (hi - o) * inv
    tmin = np.nanmax(np.minimum(t1, t2), axis=1)
    tmax = np.nanmin(np.maximum(t1, t2), axis=1)
    ok = (tmax >= tmin) & (tmax > 0)
    return np.where(ok, np.where(tmin > 0, tmin, np.inf), np.inf)


def _quad_roots(A, B, C):
    disc = B * B - 4 * A * C
    ok = (disc >= 0) & (A != 0)
    sq = np.sqrt(np.where(ok, disc, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (-B - sq) / (2 * A)
        t1 = (-B + sq) / (2 * A)
    return np.where(ok, t0, np.inf), np.where(ok, t1, np.inf)


def _hit_cylinder(o, d, r, h):
    A = d[:, 0] ** 2 + d[:, 1] ** 2
    B = 2 * (o[:, 0] * d[:, 0] + o[:, 1] * d[:, 1])
    C = o[:, 0] ** 2 + o[:, 1] ** 2 - r * r
    best = np.full(len(o), np.inf)
    for t in _quad_roots(A, B, C):
        z = o[:, 2] + t * d[:, 2]
        ok = np.isfinite(t) & (t > 0) & (z >= 0) & (z <= h)
        best = np.where(ok & (t < best), t, best)
    for zc in (0.0, h):
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (zc - o[:, 2]) / d[:, 2]
        x = o[:, 0] + t * d[:, 0]
        y = o[:, 1] + t * d[:, 1]
        ok = np.isfinite(t) & (t > 0) & (x * x + y * y <= r * r)
        best = np.where(ok & (t < best), t, best)
    return best


def _hit_ellipsoid(o, d, a, b, c):
    s = np.array([1 / a, 1 / b, 1 / c])
    oo = (o - np.array([0.0, 0.0, c])) * s
    dd = d * s
    A = np.sum(dd * dd, axis=1)
    B = 2 * np.sum(oo * dd, axis=1)
    C = np.sum(oo * oo, axis=1) - 1.0
    t0, t1 = _quad_roots(A, B, C)
    return np.where(t0 > 0, t0, np.where(t1 > 0, t1, np.inf))


def _hit_shape(shape, o, d):
    kind = shape[0]
    if kind == "box":
        return _hit_box(o, d, *shape[1:])
    if kind == "cylinder":
        return _hit_cylinder(o, d, *shape[1:])
    if kind == "ellipsoid":
        return _hit_ellipsoid(o, d, *shape[1:])
    raise ValueError(kind)


def raycast(W, H, fx, fy, cx, cy, objects, background):
    """Ray-cast analytic shapes.

    objects: list of (Mesh, R_oc (3x3 float64), t_oc (3,), label).
    background: ("table", R_wc, t_wc, half_extent, rgb) or ("wall", z, rgb) or None.
    Returns camera-frame Z (float64, inf = no hit), RGB float64 and labels int32.
    """
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    dirs = np.stack([(u - cx) / fx, (v - cy) / fy, np.ones_like(u)], axis=-1).reshape(-1, 3)
    n = dirs.shape[0]
    zbest = np.full(n, np.inf)
    rgb = np.zeros((n, 3))
    label = np.full(n, -1, np.int32)
    if background is not None:
        if background[0] == "table":
            _, r_wc, t_wc, half, col = background
            # plane z_w = 0: camera ray p_c = t * dir, p_w = R^T (p_c - t_wc)
            rt = r_wc.T
            o_w = -rt @ t_wc
            d_w = dirs @ rt.T
            with np.errstate(divide="ignore", invalid="ignore"):
                t = -o_w[2] / d_w[:, 2]
            pw = o_w[None, :] + t[:, None] * d_w
            ok = np.isfinite(t) & (t > 0) & (np.abs(pw[:, 0]) <= half) & (np.abs(pw[:, 1]) <= half)
            zbest = np.where(ok, t, zbest)
            tex = 8.0 * np.sin(40.0 * pw[:, 0]) * np.cos(40.0 * pw[:, 1])
            rgb = np.where(ok[:, None], np.array(col)[None, :] + tex[:, None], rgb)
        elif background[0] == "wall":
            _, zw, col = background
            zbest[:] = zw
            rgb[:] = col
    for mesh, r_oc, t_oc, lab in objects:
        # object frame: p_o = R^T (p_c - t)
        o = np.broadcast_to(-(r_oc.T @ t_oc), (n, 3))
        d = dirs @ r_oc            # (R^T dir) for each row
        t = _hit_shape(mesh.shape, o, d)
        closer = t < zbest
        if np.any(closer):
            p = o[closer] + t[closer, None] * d[closer]
            rgb[closer] = mesh.colour_fn(p)
            zbest = np.where(closer, t, zbest)
            label = np.where(closer, lab, label)
    return zbest.reshape(H, W), rgb.reshape(H, W, 3), label.reshape(H, W)


def quantise_depth(z, rng=None, noise_m=0.0):
    zz = np.array(z, np.float64)
    hit = np.isfinite(zz)
    if rng is not None and noise_m > 0:
        zz = zz + rng.normal(0.0, noise_m, size=zz.shape)
    d = np.where(hit, np.rint(zz * DEPTH_SCALE), 0.0)
    d = np.where(hit, np.clip(d, 1, 65535), 0)
    return d.astype(np.uint16)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclass
class Params:
    delta_m: float = 0.01
    tau_c: float = 12.5
    color_check: int = 0
    stride: int = 1
    occ_margin_units: int = 100
    z_near_m: float = 0.05
    jo_mode: int = 0


@dataclass
class Request:
    mesh_index: int
    label: int                   # -1: cylinder V(O); >= 0: labels == label
    roi: tuple                   # (u0, v0, u1, v1), half-open
    poses: np.ndarray            # (n,12) float32
    gt_index: int = -1           # index of the ground-truth pose in poses, if on the grid


@dataclass
class Scene:
    name: str
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    depth: np.ndarray            # (H,W) uint16
    rgb: np.ndarray              # (H,W,3) uint8
    labels: np.ndarray | None    # (H,W) int32 or None
    params: Params
    meshes: list
    requests: list
    gt_poses: list = field(default_factory=list)

    @property
    def n_hyp(self):
        return int(sum(r.poses.shape[0] for r in self.requests))


def _grid_poses(r_wc, t_wc, xs, ys, yaws):
    out = np.empty((len(xs) * len(ys) * len(yaws), 12), np.float64)
    k = 0
    for x in xs:
        for y in ys:
            for a in yaws:
                out[k] = tabletop_pose(r_wc, t_wc, x, y, a)
                k += 1
    return out.astype(np.float32)


def tabletop_small(seed=1001, noise_m=0.002, colour=False, on_grid=True, W=160, H=120):
    """One box on a table, 968 grid hypotheses (11x11 positions x 8 yaws)."""
    rng = np.random.default_rng(seed)
    f = 150.0 * W / 160.0
    cx, cy = W / 2.0, H / 2.0
    r_wc, t_wc = look_at(0.53, 50.0)
    box = box_mesh(0.06, 0.08, 0.12, 5, 6, 9, name="box")
    xs = np.arange(-5, 6) * 0.02
    yaws = np.arange(8) * (math.pi / 4)
    ix, iy, ia = rng.integers(2, 9), rng.integers(2, 9), rng.integers(0, 8)
    if on_grid:
        gx, gy, ga = xs[ix], xs[iy], yaws[ia]
    else:
        gx, gy, ga = rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), rng.uniform(0, 2 * math.pi)
    gt = tabletop_pose(r_wc, t_wc, gx, gy, ga)
    r_oc = gt.reshape(3, 4)[:, :3]
    t_oc = gt.reshape(3, 4)[:, 3]
    z, rgbf, _ = raycast(W, H, f, f, cx, cy, [(box, r_oc, t_oc, 0)],
                         ("table", r_wc, t_wc, 1.0, (128.0, 128.0, 128.0)))
    depth = quantise_depth(z, rng, noise_m)
    rgb = _u8(rgbf)
    poses = _grid_poses(r_wc, t_wc, xs, xs, yaws)
    gt_index = int((ix * len(xs) + iy) * len(yaws) + ia) if on_grid else -1
    params = Params(delta_m=0.01, color_check=int(colour), occ_margin_units=100)
    req = Request(0, -1, (0, 0, W, H), poses, gt_index)
    return Scene("tabletop_small", W, H, f, f, cx, cy, depth, rgb, None, params, [box], [req], [gt])


# Table-frame positions (m) of the three tabletop objects: the ellipsoid on
# the left, the two cans on the right.  The ellipsoid is the shorter object, so
# it is the one a pose could hide completely behind (or inside) a can; its
# centre is kept more than 25 cm (Chebyshev, in the table plane) from both
# cans, so that no pose of its +-21 cm grid comes near one.  Equal-height
# objects cannot hide each other from this camera (the farther top shows).
_TABLETOP_LAYOUT = ((-0.15, 0.01), (0.12, -0.09), (0.11, 0.08))
# Camera distance of the 3-object tabletop: far enough that every pose of
# every grid lies wholly inside the 640x480 image (a pose partly outside the
# image has fewer points to pay for and would undercut the true one).
_TABLETOP_3OBJ_DIST = 1.05


def tabletop_3obj(seed=1002, noise_m=0.003, occluder_frac=0.2, grid_half=21, n_yaw=16,
                  W=640, H=480, tri_scale=1.0, yaw_phase=0.0):
    """Ellipsoid + two same-shape cylinders of different colour on a table.

    Ground truth on the hypothesis grid: positions on the 1 cm lattice (the
    layout above plus a seeded offset of -1..1 cm) and yaws from the n_yaw
    set, so that Request.gt_index names the true pose.  Hypotheses per
    object: (2*grid_half+1)^2 positions at 1 cm x n_yaw yaws centred on the
    object's position.  yaw_phase (a fraction of the yaw step) shifts the
    hypotheses' yaws, not the scene: shards of a finer yaw grid for several
    processes; gt_index is then -1.
    """
    rng = np.random.default_rng(seed)
    f = 615.0 * W / 640.0
    cx, cy = W / 2.0, H / 2.0
    r_wc, t_wc = look_at(_TABLETOP_3OBJ_DIST, 50.0)
    nlon = max(8, int(round(100 * math.sqrt(tri_scale))))
    nseg = max(8, int(round(128 * math.sqrt(tri_scale))))
    ell = ellipsoid_mesh(0.04, 0.03, 0.05, nlon + 1, nlon, name="ellipsoid", vol_r=0.03, vol_h=0.10)
    nrow = max(2, int(round(38 * math.sqrt(tri_scale))))
    can_a = cylinder_mesh(0.033, 0.12, nseg, nrow, colour_wheel(0.0, 0.75, 0.95, 0.12, 0.033), name="can_a")
    # same shape, different colour: no yaw of one can matches the other's
    # colours (its hue wheel runs the other way round, and it is darker)
    can_b = cylinder_mesh(0.033, 0.12, nseg, nrow, colour_wheel(0.45, 0.6, 0.62, 0.12, 0.033, turns=-1),
                          name="can_b")
    meshes = [ell, can_a, can_b]
    pos = [np.round((np.array(xy) + 0.01 * rng.integers(-1, 2, size=2)) * 100) / 100 for xy in _TABLETOP_LAYOUT]
    yaw_index = rng.integers(0, n_yaw, size=3)
    yaws_gt = yaw_index * (2 * math.pi / n_yaw)
    objs, gts = [], []
    for k, m in enumerate(meshes):
        g = tabletop_pose(r_wc, t_wc, pos[k][0], pos[k][1], yaws_gt[k])
        gts.append(g)
        objs.append((m, g.reshape(3, 4)[:, :3], g.reshape(3, 4)[:, 3], k))
    z, rgbf, labels = raycast(W, H, f, f, cx, cy, objs, ("table", r_wc, t_wc, 1.0, (128.0, 128.0, 128.0)))
    depth = quantise_depth(z, rng, noise_m).astype(np.int64)
    rgb = _u8(rgbf)
    if occluder_frac > 0:
        occ = (rng.random(depth.shape) < occluder_frac) & (depth > 0)
        lift = np.rint(rng.uniform(0.02, 0.10, size=depth.shape) * DEPTH_SCALE).astype(np.int64)
        depth = np.where(occ, np.maximum(depth - lift, 1), depth)
        rnd = rng.integers(0, 256, size=rgb.shape, dtype=np.int64).astype(np.uint8)
        rgb = np.where(occ[..., None], rnd, rgb)
    depth = depth.astype(np.uint16)
    params = Params(delta_m=0.01, tau_c=12.5, color_check=1, occ_margin_units=100)
    steps = np.arange(-grid_half, grid_half + 1) * 0.01
    yaws = (np.arange(n_yaw) + yaw_phase) * (2 * math.pi / n_yaw)
    reqs = []
    for k in range(3):
        cxg, cyg = pos[k]
        poses = _grid_poses(r_wc, t_wc, cxg + steps, cyg + steps, yaws)
        gt_index = int((grid_half * len(steps) + grid_half) * n_yaw + yaw_index[k]) if yaw_phase == 0 else -1
        reqs.append(Request(k, -1, (0, 0, W, H), poses, gt_index))
    return Scene("tabletop_3obj", W, H, f, f, cx, cy, depth, rgb, None, params, meshes, reqs, gts)


def _dilate(mask, k):
    if k <= 0:
        return mask
    out = mask.copy()
    H, W = mask.shape
    p = np.pad(mask, k)
    for dy in range(-k, k + 1):
        for dx in range(-k, k + 1):
            out |= p[k + dy:k + dy + H, k + dx:k + dx + W]
    return out


def _erode(mask, k):
    return ~_dilate(~mask, k) if k > 0 else mask


def _shift(mask, dx, dy):
    out = np.zeros_like(mask)
    H, W = mask.shape
    ys, yd = (slice(0, H - dy), slice(dy, H)) if dy >= 0 else (slice(-dy, H), slice(0, H + dy))
    xs, xd = (slice(0, W - dx), slice(dx, W)) if dx >= 0 else (slice(-dx, W), slice(0, W + dx))
    out[yd, xd] = mask[ys, xs]
    return out


def sixdof_5obj(seed=1003, n_hyp=4096, W=640, H=480, tri_scale=1.0, noise_m=0.002):
    """Five 30k-triangle meshes at random 6-DoF poses, label-based V and ROI."""
    rng = np.random.default_rng(seed)
    f = 615.0 * W / 640.0
    cx, cy = W / 2.0, H / 2.0
    s = math.sqrt(tri_scale)
    n_e = max(8, int(round(122 * s)))
    meshes = [
        ellipsoid_mesh(0.05, 0.035, 0.04, n_e + 1, n_e, name="ellipsoid_a"),
        cylinder_mesh(0.04, 0.10, max(8, int(round(250 * s))), max(2, int(round(59 * s))),
                      colour_wheel(0.1, 0.8, 0.9, 0.10), name="cylinder_a"),
        box_mesh(0.07, 0.05, 0.09, max(1, int(round(52 * s))), max(1, int(round(37 * s))),
                 max(1, int(round(66 * s))), name="box_a"),
        cylinder_mesh(0.03, 0.14, max(8, int(round(250 * s))), max(2, int(round(59 * s))),
                      colour_wheel(0.6, 0.6, 0.85, 0.14), name="cylinder_b"),
        ellipsoid_mesh(0.045, 0.045, 0.06, n_e + 1, n_e, name="ellipsoid_b",
                       colour_fn=colour_gradient((0.09, 0.09, 0.12), base=(40, 90, 30), span=(200, 120, 200))),
    ]
    objs, gts = [], []
    for k, m in enumerate(meshes):
        zc = rng.uniform(0.7, 1.0)
        u = rng.uniform(0.25 * W, 0.75 * W)
        v = rng.uniform(0.25 * H, 0.75 * H)
        r = random_rotation(rng)
        centre_o = np.array([0.0, 0.0, m.vol_height / 2])
        c_cam = np.array([(u - cx) / f * zc, (v - cy) / f * zc, zc])
        t = c_cam - r @ centre_o
        gts.append(pose_rows(r, t))
        objs.append((m, r, t, k))
    z, rgbf, labels = raycast(W, H, f, f, cx, cy, objs, ("wall", 1.3, (110.0, 115.0, 120.0)))
    depth = quantise_depth(z, rng, noise_m)
    rgb = _u8(rgbf)
    lab = np.full((H, W), -1, np.int32)
    rois = []
    for k in range(len(meshes)):
        m = labels == k
        m = _shift(m, int(rng.integers(-3, 4)), int(rng.integers(-3, 4)))
        op = int(rng.integers(-3, 4))
        m = _dilate(m, op) if op > 0 else _erode(m, -op)
        lab[m] = k
        ys, xs = np.nonzero(m)
        if len(xs) == 0:
            rois.append((0, 0, 1, 1))
        else:
            rois.append((int(xs.min()), int(ys.min()), int(xs.max()) + 1, int(ys.max()) + 1))
    params = Params(delta_m=0.01, tau_c=12.5, color_check=1, occ_margin_units=100)
    reqs = []
    for k in range(len(meshes)):
        g = gts[k].reshape(3, 4)
        poses = np.empty((n_hyp, 12), np.float64)
        for i in range(n_hyp):
            axis = rng.normal(size=3)
            th = math.radians(rng.normal(0.0, 15.0))
            r = rodrigues(axis, th) @ g[:, :3]
            t = g[:, 3] + rng.normal(0.0, 0.02, size=3)
            poses[i] = pose_rows(r, t)
        reqs.append(Request(k, k, rois[k], poses.astype(np.float32)))
    return Scene("sixdof_5obj", W, H, f, f, cx, cy, depth, rgb, lab, params, meshes, reqs, gts)


def mesh_pool(seed=77, tri_counts=(500, 2000, 5000, 10000, 20000, 30000)):
    """Meshes of three shapes at several triangle counts, shared by batched scenes."""
    rng = np.random.default_rng(seed)
    pool = []
    for k, t in enumerate(tri_counts):
        kind = k % 3
        if kind == 0:
            n = max(4, int(round(math.sqrt(t / 2))))
            a, b, c = rng.uniform(0.03, 0.06, size=3)
            pool.append(ellipsoid_mesh(a, b, c, n + 1, n, name=f"ellipsoid_{t}"))
        elif kind == 1:
            nseg = max(8, int(round(math.sqrt(t * 3))))
            nrow = max(1, int(round(t / (2 * nseg))))
            pool.append(cylinder_mesh(rng.uniform(0.025, 0.045), rng.uniform(0.08, 0.15), nseg, nrow,
                                      colour_wheel(rng.uniform(), 0.7, 0.9, 0.12), name=f"cylinder_{t}"))
        else:
            q = max(1, int(round(math.sqrt(t / 12))))
            pool.append(box_mesh(*rng.uniform(0.04, 0.10, size=3), q, q, q, name=f"box_{t}"))
    return pool


def batched_scenes(seed=1004, n_scenes=64, W=320, H=240, hyp_range=(500, 40000), max_objects=6,
                   pool=None):
    """Scenes of uneven size for the batched form: 1-6 objects each (meshes from a
    shared pool of 500-30k triangles), 6-DoF ground truth, labels and ROIs from
    perturbed masks (ROI clamped to 64x64 .. 320x240 around the mask), and a
    per-scene hypothesis budget drawn from hyp_range, split over the objects."""
    rng = np.random.default_rng(seed)
    pool = pool if pool is not None else mesh_pool()
    f = 615.0 * W / 640.0
    cx, cy = W / 2.0, H / 2.0
    out = []
    for sidx in range(n_scenes):
        k = int(rng.integers(1, max_objects + 1))
        picks = rng.choice(len(pool), size=k, replace=True)
        meshes = [pool[i] for i in picks]
        objs, gts = [], []
        for j, m in enumerate(meshes):
            zc = rng.uniform(0.45, 0.9)
            u = rng.uniform(0.2 * W, 0.8 * W)
            v = rng.uniform(0.2 * H, 0.8 * H)
            r = random_rotation(rng)
            c_cam = np.array([(u - cx) / f * zc, (v - cy) / f * zc, zc])
            t = c_cam - r @ np.array([0.0, 0.0, m.vol_height / 2])
            gts.append(pose_rows(r, t))
            objs.append((m, r, t, j))
        z, rgbf, labels = raycast(W, H, f, f, cx, cy, objs, ("wall", 1.2, (100.0, 110.0, 105.0)))
        depth = quantise_depth(z, rng, 0.002)
        lab = np.full((H, W), -1, np.int32)
        rois = []
        for j in range(k):
            mk = _dilate(labels == j, int(rng.integers(0, 3)))
            lab[mk] = j
            ys, xs = np.nonzero(mk)
            if len(xs) == 0:
                xs, ys = np.array([W // 2]), np.array([H // 2])
            u0, u1, v0, v1 = xs.min(), xs.max() + 1, ys.min(), ys.max() + 1
            w = int(np.clip(u1 - u0, 64, 320))
            h = int(np.clip(v1 - v0, 64, 240))
            uc, vc = (u0 + u1) // 2, (v0 + v1) // 2
            ru0 = int(np.clip(uc - w // 2, 0, W - w))
            rv0 = int(np.clip(vc - h // 2, 0, H - h))
            rois.append((ru0, rv0, ru0 + w, rv0 + h))
        budget = int(rng.integers(hyp_range[0], hyp_range[1] + 1))
        share = np.maximum(1, rng.multinomial(budget - k, np.ones(k) / k) + 1)
        reqs = []
        for j in range(k):
            g = gts[j].reshape(3, 4)
            n = int(share[j])
            axes = rng.normal(size=(n, 3))
            th = np.radians(rng.normal(0.0, 15.0, size=n))
            rot = rodrigues_batch(axes, th) @ g[:, :3]
            trans = g[:, 3][None, :] + rng.normal(0.0, 0.02, size=(n, 3))
            poses = np.concatenate([rot, trans[:, :, None]], axis=2).reshape(n, 12)
            reqs.append(Request(j, j, rois[j], poses.astype(np.float32)))
        params = Params(delta_m=0.01, tau_c=12.5, color_check=1, occ_margin_units=100)
        out.append(Scene(f"batched_{sidx}", W, H, f, f, cx, cy, depth, _u8(rgbf), lab, params, meshes,
                         reqs, gts))
    return out


WORKLOADS = {
    "tabletop_small": tabletop_small,
    "tabletop_3obj": tabletop_3obj,
    "sixdof_5obj": sixdof_5obj,
}
