"""6-DoF pose proposals (Sec. V-B, Eq. 5 and Eq. 6) -- plain float64 oracle.

TEST INFRASTRUCTURE ONLY: the parity reference for perch_pose_proposals.  It
shares no code with the CUDA path.

H_r (Eq. 5): M viewpoints on the unit sphere taken from a Fibonacci lattice
(y_i = 1 - (2i+1)/M, azimuth i times the golden angle) -- the reading of "M
equidistant viewpoints" -- times N in-plane angles 2 pi k / N.  The viewpoint
is the object-to-camera direction in the object frame; the camera looks along
its negative, with "right" = forward x z (or forward x y when forward is
parallel to z) and "down" = forward x right; the in-plane angle rotates about
the optical axis.

H_t (Eq. 6): the centre of the object's 2-D box back-projected at K depths
from the nearest to the farthest observed depth of the box's pixels that carry
the object's label (K = 1: the mean of the two).  The translation places the
centre of the mesh's bounding box at that point.
"""
import math

import numpy as np


def depth_range(depth, labels, label, box):
    u0, v0, u1, v1 = box
    d = depth[v0:v1, u0:u1].astype(np.int64)
    m = (labels[v0:v1, u0:u1] == label) & (d > 0)
    if not m.any():
        return 0, 0
    return int(d[m].min()), int(d[m].max())


def viewpoint(i, M):
    golden = math.pi * (3.0 - math.sqrt(5.0))
    y = 1.0 - (2.0 * i + 1.0) / M
    r = math.sqrt(max(0.0, 1.0 - y * y))
    phi = golden * i
    return np.array([r * math.cos(phi), y, r * math.sin(phi)])


def view_rotation(v):
    f = -np.asarray(v, np.float64)
    r = np.cross(f, [0.0, 0.0, 1.0])
    if np.linalg.norm(r) < 1e-6:
        r = np.cross(f, [0.0, 1.0, 0.0])
    r = r / np.linalg.norm(r)
    d = np.cross(f, r)
    return np.stack([r, d, f])


def proposals(depth, labels, label, box, fx, fy, cx, cy, mesh_lo, mesh_hi, M, N, K):
    """(M*N*K, 12) float64 poses ordered ((i N + k) K + j), and (z_min, z_max)."""
    zmin_u, zmax_u = depth_range(depth, labels, label, box)
    zmin, zmax = zmin_u / 10000.0, zmax_u / 10000.0
    u0, v0, u1, v1 = box
    uc, vc = 0.5 * (u0 + u1 - 1), 0.5 * (v0 + v1 - 1)
    m = 0.5 * (np.asarray(mesh_lo, np.float64) + np.asarray(mesh_hi, np.float64))
    out = np.empty((M * N * K, 12))
    for i in range(M):
        Rv = view_rotation(viewpoint(i, M))
        for k in range(N):
            th = 2.0 * math.pi * k / N
            Rz = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0],
                           [0.0, 0.0, 1.0]])
            R = Rz @ Rv
            for j in range(K):
                z = zmin + (zmax - zmin) * j / (K - 1) if K > 1 else 0.5 * (zmin + zmax)
                c = np.array([(uc - cx) * z / fx, (vc - cy) * z / fy, z])
                out[(i * N + k) * K + j] = np.concatenate([R, (c - R @ m)[:, None]], 1).reshape(12)
    return out, (zmin_u, zmax_u)
