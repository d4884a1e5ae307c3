"""ctypes front end of the plain-C PERCH 2.0 oracle (``perch_oracle.c``).

TEST INFRASTRUCTURE ONLY: the parity reference for the CUDA path.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module.  It shares no code with the CUDA library and never imports
it.  ``build()`` compiles the C file with ``-ffp-contract=off`` (no FMA
contraction, no fast-math), which the bit-exact parity contract relies on.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "perch_oracle.c")
LIB = os.path.join(HERE, "liboracle_perch.so")
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
NWORK = 8
WORK_NAMES = ("tri_setups", "tri_culled", "fragments", "visible", "kept",
              "cell_candidates", "in_volume", "explained")


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2 -ffp-contract=off, OpenMP)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11",
           "-Wall", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


class _Scene(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("depth", C.c_void_p), ("rgb", C.c_void_p),
                ("labels", C.c_void_p), ("delta", C.c_float), ("tau_c", C.c_float),
                ("color_check", C.c_int32), ("stride", C.c_int32), ("occ_margin", C.c_int32),
                ("z_near", C.c_float), ("jo_mode", C.c_int32)]


class _Mesh(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("rgb", C.c_void_p), ("n_verts", C.c_int32),
                ("tris", C.c_void_p), ("n_tris", C.c_int32), ("vol_r", C.c_float),
                ("vol_h", C.c_float)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.c_void_p
        L.or_render_keys.argtypes = [P, P, P, P, P, P]
        L.or_observed_points.argtypes = [P, P, P, P]
        L.or_observed_points.restype = C.c_int64
        L.or_rendered_points.argtypes = [P, P, P, C.c_int32, P, P, P, P]
        L.or_rendered_points.restype = C.c_int64
        L.or_score.argtypes = [P, P, C.c_int32, P, P, C.c_int64, P, P, P, C.c_int32]
        L.or_score_nn.argtypes = [P, P, C.c_int32, P, P, C.c_int64, P, P, P, C.c_int32, C.c_int32]
        L.or_best.argtypes = [P, P, C.c_int64, P, P]
        L.or_srgb_to_lab.argtypes = [P, P]
        L.or_ciede2000.argtypes = [P, P, P]
        L.or_ciede2000.restype = C.c_float
        L.or_num_threads.restype = C.c_int
        L.or_gicp.argtypes = [P, P, C.c_int32, P, P, C.c_int64, P, P, P, C.c_int32]
        L.or_triangle_normal.argtypes = [P, C.c_int32, P]
        L.or_observed_normal.argtypes = [P, C.c_int32, C.c_int64, C.c_int64, P]
        L.or_gicp_terms.argtypes = [P, P, P, P, P, P, C.c_float, P]
        L.or_gicp_quantise.argtypes = [C.c_float]
        L.or_gicp_quantise.restype = C.c_int64
        L.or_gicp_solve.argtypes = [P, P]
        L.or_gicp_rotation.argtypes = [P, P]
        L.or_add_s.argtypes = [P, C.c_int32, P, P, C.c_int32]
        L.or_add_s.restype = C.c_double
        L.or_score_tree.argtypes = [P, P, C.c_int32, P, P, C.c_int64, P, P, P, P, P, P, P, P, C.c_int32]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class OracleScene:
    """An observation plus scoring parameters, held as contiguous arrays."""

    def __init__(self, depth, rgb, labels, fx, fy, cx, cy, delta=0.01, tau_c=12.5,
                 color_check=0, stride=1, occ_margin=100, z_near=0.05, jo_mode=0):
        self.depth = np.ascontiguousarray(depth, np.uint16)
        self.rgb = np.ascontiguousarray(rgb, np.uint8)
        self.labels = None if labels is None else np.ascontiguousarray(labels, np.int32)
        H, W = self.depth.shape
        self.W, self.H = W, H
        self.s = _Scene(W, H, fx, fy, cx, cy, _ptr(self.depth), _ptr(self.rgb), _ptr(self.labels),
                        delta, tau_c, color_check, stride, occ_margin, z_near, jo_mode)

    @classmethod
    def from_scene(cls, sc, **over):
        p = sc.params
        kw = dict(delta=p.delta_m, tau_c=p.tau_c, color_check=p.color_check, stride=p.stride,
                  occ_margin=p.occ_margin_units, z_near=p.z_near_m, jo_mode=p.jo_mode)
        kw.update(over)
        return cls(sc.depth, sc.rgb, sc.labels, sc.fx, sc.fy, sc.cx, sc.cy, **kw)


class OracleMesh:
    def __init__(self, verts, rgb, tris, vol_r, vol_h):
        self.verts = np.ascontiguousarray(verts, np.float32)
        self.rgb = np.ascontiguousarray(rgb, np.uint8)
        self.tris = np.ascontiguousarray(tris, np.int32)
        self.m = _Mesh(_ptr(self.verts), _ptr(self.rgb), self.verts.shape[0], _ptr(self.tris),
                       self.tris.shape[0], vol_r, vol_h)

    @classmethod
    def from_mesh(cls, m):
        return cls(m.verts, m.rgb, m.tris, m.vol_radius, m.vol_height)


def render_keys(scene: OracleScene, mesh: OracleMesh, pose, roi=None):
    """Key buffer (H,W) uint64: (depth << 32) | triangle id, EMPTY where uncovered."""
    roi = np.asarray(roi if roi is not None else (0, 0, scene.W, scene.H), np.int32)
    pose = np.ascontiguousarray(pose, np.float32).reshape(12)
    keys = np.empty((scene.H, scene.W), np.uint64)
    work = np.zeros(NWORK, np.int64)
    lib().or_render_keys(C.byref(scene.s), C.byref(mesh.m), _ptr(pose), _ptr(roi), _ptr(keys),
                         _ptr(work))
    return keys, work


def observed_points(scene: OracleScene):
    n = scene.W * scene.H
    xyz = np.empty((n, 3), np.float32)
    lab = np.empty((n, 3), np.float32)
    pix = np.empty(n, np.int32)
    k = lib().or_observed_points(C.byref(scene.s), _ptr(xyz), _ptr(lab), _ptr(pix))
    return xyz[:k], lab[:k], pix[:k]


def rendered_points(scene: OracleScene, mesh: OracleMesh, pose, keys, label=-1):
    n = scene.W * scene.H
    xyz = np.empty((n, 3), np.float32)
    rgb = np.empty((n, 3), np.uint8)
    pix = np.empty(n, np.int32)
    pose = np.ascontiguousarray(pose, np.float32).reshape(12)
    keys = np.ascontiguousarray(keys, np.uint64)
    k = lib().or_rendered_points(C.byref(scene.s), C.byref(mesh.m), _ptr(pose), label, _ptr(keys),
                                 _ptr(xyz), _ptr(rgb), _ptr(pix))
    return xyz[:k], rgb[:k], pix[:k]


def score(scene: OracleScene, mesh: OracleMesh, poses, label=-1, roi=None, threads=0,
          with_work=False, nn="brute"):
    """(costs (n,2) int32 [J_o, J_r], band (n,) int32[, work (n,8) int64]).
    nn: "brute" scans all of the other cloud for each nearest neighbour (Eq. 2
    as written); "grid" scans the 27 cells of edge delta (1 + 1/32) around the
    query (the same neighbour within delta, far faster; pinned equal to
    "brute"; work column 5, the delta-cell candidates, is left at 0)."""
    if nn not in ("brute", "grid"):
        raise ValueError(nn)
    poses = np.ascontiguousarray(poses, np.float32).reshape(-1, 12)
    n = poses.shape[0]
    roi = np.asarray(roi if roi is not None else (0, 0, scene.W, scene.H), np.int32)
    costs = np.zeros((n, 2), np.int32)
    band = np.zeros(n, np.int32)
    work = np.zeros((n, NWORK), np.int64) if with_work else None
    rc = lib().or_score_nn(C.byref(scene.s), C.byref(mesh.m), label, _ptr(roi), _ptr(poses), n,
                           _ptr(costs), _ptr(band), _ptr(work), threads, 1 if nn == "grid" else 0)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return (costs, band, work) if with_work else (costs, band)


def best(costs, ids=None):
    costs = np.ascontiguousarray(costs, np.int32).reshape(-1, 2)
    ids = None if ids is None else np.ascontiguousarray(ids, np.uint64)
    bi = C.c_int64()
    bc = C.c_int32()
    rc = lib().or_best(_ptr(costs), _ptr(ids), costs.shape[0], C.byref(bi), C.byref(bc))
    if rc != 0:
        raise ValueError("empty cost array")
    return bi.value, bc.value


def srgb_to_lab(rgb):
    rgb = np.ascontiguousarray(rgb, np.uint8).reshape(3)
    out = np.empty(3, np.float32)
    lib().or_srgb_to_lab(_ptr(rgb), _ptr(out))
    return out


def ciede2000(lab1, lab2):
    a = np.ascontiguousarray(lab1, np.float32).reshape(3)
    b = np.ascontiguousarray(lab2, np.float32).reshape(3)
    gap = C.c_float()
    v = lib().or_ciede2000(_ptr(a), _ptr(b), C.byref(gap))
    return float(v), float(gap.value)


class _GicpParams(C.Structure):
    _fields_ = [("max_iters", C.c_int32), ("epsilon", C.c_float), ("normal_jump", C.c_int32),
                ("min_corr", C.c_int32), ("stop_rot", C.c_float), ("stop_trans", C.c_float)]


GICP_DEFAULTS = dict(max_iters=10, epsilon=1e-3, normal_jump=200, min_corr=6, stop_rot=1e-5,
                     stop_trans=1e-5)
GICP_NVAL = 28


def gicp(scene: OracleScene, mesh: OracleMesh, poses, label=-1, roi=None, threads=0, **params):
    """Refine poses by M2M GICP: (poses_out (n,12) float32, info (n,2) int32 =
    [updates applied, correspondences of the last iteration])."""
    kw = dict(GICP_DEFAULTS)
    kw.update(params)
    gp = _GicpParams(**kw)
    poses = np.ascontiguousarray(poses, np.float32).reshape(-1, 12)
    n = poses.shape[0]
    roi = np.asarray(roi if roi is not None else (0, 0, scene.W, scene.H), np.int32)
    out = np.zeros((n, 12), np.float32)
    info = np.zeros((n, 2), np.int32)
    rc = lib().or_gicp(C.byref(scene.s), C.byref(mesh.m), label, _ptr(roi), _ptr(poses), n,
                       C.byref(gp), _ptr(out), _ptr(info), threads)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out, info


def triangle_normal(mesh: OracleMesh, t):
    out = np.empty(3, np.float32)
    lib().or_triangle_normal(C.byref(mesh.m), int(t), _ptr(out))
    return out


def observed_normal(scene: OracleScene, u, v, normal_jump=200):
    out = np.empty(3, np.float32)
    lib().or_observed_normal(C.byref(scene.s), int(normal_jump), int(u), int(v), _ptr(out))
    return out


def gicp_terms(Rf, tf, a, na, b, nb, eps=1e-3):
    """(ok, terms[28]) of one correspondence."""
    arrs = [np.ascontiguousarray(x, np.float32).reshape(-1) for x in (Rf, tf, a, na, b, nb)]
    out = np.zeros(GICP_NVAL, np.float32)
    ok = lib().or_gicp_terms(*[_ptr(x) for x in arrs], C.c_float(eps), _ptr(out))
    return bool(ok), out


def gicp_quantise(x):
    return int(lib().or_gicp_quantise(C.c_float(x)))


def gicp_solve(S):
    S = np.ascontiguousarray(S, np.int64).reshape(GICP_NVAL)
    xi = np.zeros(6, np.float64)
    ok = lib().or_gicp_solve(_ptr(S), _ptr(xi))
    return bool(ok), xi


def gicp_rotation(w):
    w = np.ascontiguousarray(w, np.float64).reshape(3)
    R = np.zeros(9, np.float64)
    lib().or_gicp_rotation(_ptr(w), _ptr(R))
    return R.reshape(3, 3)


def empty_state(scene: OracleScene):
    """Root of the Monotone Scene Generation tree: (depth u32, mark u8, vol u8) images."""
    return (np.zeros((scene.H, scene.W), np.uint32), np.zeros((scene.H, scene.W), np.uint8),
            np.zeros((scene.H, scene.W), np.uint8))


def score_tree(scene: OracleScene, mesh: OracleMesh, poses, state, label=-1, roi=None, child=False,
               threads=0):
    """Edge costs of adding the object at each pose to `state`: (costs (n,2)
    int32, (-1,-1) = refused, band (n,)[, child state]) -- child only for n == 1."""
    poses = np.ascontiguousarray(poses, np.float32).reshape(-1, 12)
    n = poses.shape[0]
    roi = np.asarray(roi if roi is not None else (0, 0, scene.W, scene.H), np.int32)
    pd, pm, pv = (np.ascontiguousarray(x) for x in state)
    costs = np.zeros((n, 2), np.int32)
    band = np.zeros(n, np.int32)
    cd = cm = cv = None
    if child:
        assert n == 1
        cd, cm, cv = np.zeros_like(pd), np.zeros_like(pm), np.zeros_like(pv)
    rc = lib().or_score_tree(C.byref(scene.s), C.byref(mesh.m), label, _ptr(roi), _ptr(poses), n,
                             _ptr(pd), _ptr(pm), _ptr(pv), _ptr(costs), _ptr(band), _ptr(cd), _ptr(cm),
                             _ptr(cv), threads)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return (costs, band, (cd, cm, cv)) if child else (costs, band)


def add_s(verts, pose_a, pose_b, symmetric=True):
    """ADD-S (symmetric) or ADD of pose_a against pose_b over the model points, float64."""
    v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
    a = np.ascontiguousarray(pose_a, np.float32).reshape(12)
    b = np.ascontiguousarray(pose_b, np.float32).reshape(12)
    return float(lib().or_add_s(_ptr(v), v.shape[0], _ptr(a), _ptr(b), int(bool(symmetric))))


def add_auc(errors, max_threshold=0.1):
    """Area under the accuracy curve acc(t) = |{i : e_i < t}| / n on [0, T],
    divided by T: the step function integrated piece by piece between its
    sorted break points."""
    e = np.sort(np.asarray(errors, np.float64))
    n, T = len(e), float(max_threshold)
    area, prev, below = 0.0, 0.0, 0
    for x in e:
        if x >= T:
            break
        area += (x - prev) * below / n if x > prev else 0.0
        prev = max(prev, x)
        below += 1
    area += (T - prev) * below / n
    return area / T


def num_threads():
    return int(lib().or_num_threads())
