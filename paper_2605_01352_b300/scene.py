"""Seeded synthetic scenes for the simulate-then-render loop.

This module only draws random numbers and builds input geometry: body
shapes and placements, mass properties from a fixed density, the mesh
library (icosphere, cube, ground quad, convex hulls) and the pinhole
cameras.  It holds none of the step's arithmetic (integration, contacts,
impulse solve, vertex transform, rasterisation); both the CUDA path and the
CPU oracle read the arrays it returns.

The paper's workloads are ManiSkill3 scenes stepped by PhysX and rendered by
Vulkan (Sec. 6.1, experimental setup); those assets are not available, so
these seeded scenes stand in for them with the batch sizes and camera
resolutions the paper reports (Sec. 6.3 data generation, Sec. 6.4 RL).

Random numbers: one SplitMix64 stream per environment, seeded with
``seed ^ (env * 0x9E3779B97F4A7C15)`` so that an environment's content does
not depend on the batch it is generated in.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

SHAPE_SPHERE = 0
SHAPE_BOX = 1
SHAPE_HULL = 2  # rendered as a convex-hull mesh, simulated as a sphere proxy

MESH_ICOSPHERE = 0
MESH_CUBE = 1
MESH_GROUND = 2

DENSITY = 1000.0  # kg / m^3
GROUND_HALF = 1.5  # m, half size of the rendered ground quad
PALETTE = [
    (230, 80, 60), (70, 160, 230), (90, 200, 90), (240, 200, 60),
    (170, 90, 210), (60, 200, 190), (240, 140, 40), (200, 200, 200),
]
GROUND_ALBEDO = (128, 128, 128)


def pack_rgb(c) -> int:
    return int(c[0]) | (int(c[1]) << 8) | (int(c[2]) << 16)


# ----------------------------------------------------------------------------
# SplitMix64, vectorised over environments (counter-based: output k of a
# stream seeded with s is mix(s + (k + 1) * GOLDEN)).
# ----------------------------------------------------------------------------
def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


class Streams:
    """One SplitMix64 stream per environment."""

    def __init__(self, seed: int, n: int, base_index: int = 0):
        idx = np.arange(base_index, base_index + n, dtype=np.uint64)
        with np.errstate(over="ignore"):
            self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (idx * GOLDEN)
        self.state = self.state.astype(np.uint64)

    def next_u64(self, mask: Optional[np.ndarray] = None) -> np.ndarray:
        with np.errstate(over="ignore"):
            if mask is None:
                self.state = self.state + GOLDEN
                return _mix(self.state.copy())
            st = self.state.copy()
            st[mask] = st[mask] + GOLDEN
            self.state = st
            return _mix(st)

    def uniform(self, lo=0.0, hi=1.0, mask=None) -> np.ndarray:
        u = (self.next_u64(mask) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


# ----------------------------------------------------------------------------
# Meshes (unit size; scaled per body by mesh_scale)
# ----------------------------------------------------------------------------
def _orient_outward(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Make every triangle counter-clockwise seen from outside a star-shaped
    mesh centred at the origin."""
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    flip = np.einsum("ij,ij->i", nrm, (v0 + v1 + v2) / 3.0) < 0
    out = tris.copy()
    out[flip, 1], out[flip, 2] = tris[flip, 2], tris[flip, 1]
    return out


def icosphere(level: int = 1):
    """Icosahedron subdivided ``level`` times, vertices on the unit sphere.
    Level 1 has 42 vertices and 80 triangles."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts, dtype=np.float64)
    T = _orient_outward(V, np.array(faces, dtype=np.int32))
    return V.astype(np.float32), T


def cube():
    V = np.array([[(1 if k & 1 else -1), (1 if k & 2 else -1), (1 if k & 4 else -1)]
                  for k in range(8)], dtype=np.float64)
    quads = [(0, 2, 6, 4), (1, 3, 7, 5), (0, 1, 5, 4), (2, 3, 7, 6), (0, 1, 3, 2), (4, 5, 7, 6)]
    T = []
    for a, b, c, d in quads:
        T += [(a, b, c), (a, c, d)]
    T = _orient_outward(V, np.array(T, dtype=np.int32))
    return V.astype(np.float32), T


def ground_quad(half: float = GROUND_HALF):
    V = np.array([[-half, -half, 0.0], [half, -half, 0.0], [half, half, 0.0], [-half, half, 0.0]],
                 dtype=np.float32)
    T = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)  # counter-clockwise seen from +z
    return V, T


def convex_hull_mesh(streams: Streams, ntri: int):
    """Convex hull of ntri/2 + 2 random points on the unit sphere.  All points
    are hull vertices, so the hull has exactly ntri triangles."""
    from scipy.spatial import ConvexHull

    nv = ntri // 2 + 2
    while True:
        pts = []
        for _ in range(nv):
            zc = float(streams.uniform(-1.0, 1.0)[0])
            ph = float(streams.uniform(0.0, 2.0 * math.pi)[0])
            s = math.sqrt(max(0.0, 1.0 - zc * zc))
            pts.append((s * math.cos(ph), s * math.sin(ph), zc))
        P = np.array(pts, dtype=np.float64)
        hull = ConvexHull(P)
        if len(hull.vertices) == nv and hull.simplices.shape[0] == ntri:
            T = _orient_outward(P, hull.simplices.astype(np.int32))
            return P.astype(np.float32), T


def hull_from_points(points) -> tuple:
    """Convex hull mesh (vertices, outward triangles) of points on the unit
    sphere, every point a vertex of the hull (e.g. octahedron())."""
    from scipy.spatial import ConvexHull

    P = np.asarray(points, np.float64)
    hull = ConvexHull(P)
    if len(hull.vertices) != len(P):
        raise ValueError("every point must be a vertex of the hull")
    return P.astype(np.float32), _orient_outward(P, hull.simplices.astype(np.int32))


def octahedron():
    """The regular octahedron with vertices +-x, +-y, +-z: 6 vertices, 8
    faces with normals (+-1, +-1, +-1) / sqrt(3) at distance 1 / sqrt(3)."""
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float32)
    T = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                T.append([sx, sy, sz])
    return V, _orient_outward(V.astype(np.float64), np.array(T, np.int32))


# ----------------------------------------------------------------------------
# Scene container
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class SimParams:
    dt: float = 1.0 / 240.0
    substeps: int = 4
    iterations: int = 8
    gravity: tuple = (0.0, 0.0, -9.81)
    restitution: float = 0.0
    restitution_threshold: float = 1.0
    friction: float = 0.5
    baumgarte: float = 0.2
    slop: float = 0.001
    margin: float = 0.02
    jacobi_omega: float = 1.0
    plane: int = 1  # 1: static ground plane z = 0 present
    max_contacts_per_body: int = 16
    # options beyond the configured workloads' physics (off there: no
    # gyroscopic term, box-box contacts from corners only)
    gyroscopic: int = 0  # 1: gyroscopic term of boxes (implicit, one Newton step)
    edge_contacts: int = 0  # 1: box-box edge-edge contacts (separating-axis test)
    hull_contacts: int = 0  # 1: hulls collide through their vertices and faces (else as spheres of their radius)


@dataclasses.dataclass
class Scene:
    body_off: np.ndarray      # int32 [E+1]
    pos: np.ndarray           # f32 [3, B]
    quat: np.ndarray          # f32 [4, B]  (w, x, y, z)
    vel: np.ndarray           # f32 [3, B]
    angvel: np.ndarray        # f32 [3, B]
    shape_type: np.ndarray    # u8  [B]
    shape_dims: np.ndarray    # f32 [3, B]
    inv_mass: np.ndarray      # f32 [B]
    inv_inertia: np.ndarray   # f32 [3, B] (body frame, principal)
    mesh_id: np.ndarray       # int32 [B]
    mesh_scale: np.ndarray    # f32 [3, B]
    albedo: np.ndarray        # u32 [B] packed r | g<<8 | b<<16
    mesh_vert_off: np.ndarray  # int32 [M+1]
    mesh_verts: np.ndarray    # f32 [V, 3]
    mesh_tri_off: np.ndarray  # int32 [M+1]
    mesh_tris: np.ndarray     # int32 [T, 3] (mesh-local vertex indices)
    ground_mesh: int
    ground_albedo: int
    cam_off: np.ndarray       # int32 [E+1]
    cam_w: np.ndarray         # int32 [C]
    cam_h: np.ndarray         # int32 [C]
    cam_eye: np.ndarray       # f32 [C, 3]
    cam_right: np.ndarray     # f32 [C, 3]
    cam_up: np.ndarray        # f32 [C, 3]
    cam_fwd: np.ndarray       # f32 [C, 3]
    cam_fpy: np.ndarray       # f32 [C]  focal length in pixels
    light: np.ndarray         # f32 [3] unit direction towards the light
    params: SimParams = dataclasses.field(default_factory=SimParams)
    name: str = ""

    @property
    def num_envs(self) -> int:
        return len(self.body_off) - 1

    @property
    def num_bodies(self) -> int:
        return int(self.body_off[-1])

    @property
    def num_cams(self) -> int:
        return int(self.cam_off[-1])

    def bodies_per_env(self) -> np.ndarray:
        return np.diff(self.body_off).astype(np.int32)

    def cam_pix_off(self) -> np.ndarray:
        px = self.cam_w.astype(np.int64) * self.cam_h.astype(np.int64)
        return np.concatenate([[0], np.cumsum(px)]).astype(np.int64)

    def tris_per_env(self) -> np.ndarray:
        ntri_mesh = np.diff(self.mesh_tri_off)
        gt = int(ntri_mesh[self.ground_mesh])
        per_body = ntri_mesh[self.mesh_id]
        cs = np.concatenate([[0], np.cumsum(per_body)])
        return (gt + cs[self.body_off[1:]] - cs[self.body_off[:-1]]).astype(np.int64)

    def state(self):
        return dict(pos=self.pos.copy(), quat=self.quat.copy(), vel=self.vel.copy(),
                    angvel=self.angvel.copy())

    def subset(self, envs: Sequence[int]) -> "Scene":
        """A scene holding only the given environments (same meshes)."""
        envs = list(envs)
        bidx = np.concatenate([np.arange(self.body_off[e], self.body_off[e + 1]) for e in envs]).astype(np.int64) \
            if envs else np.zeros(0, np.int64)
        cidx = np.concatenate([np.arange(self.cam_off[e], self.cam_off[e + 1]) for e in envs]).astype(np.int64) \
            if envs else np.zeros(0, np.int64)
        nb = [self.body_off[e + 1] - self.body_off[e] for e in envs]
        nc = [self.cam_off[e + 1] - self.cam_off[e] for e in envs]
        return dataclasses.replace(
            self,
            body_off=np.concatenate([[0], np.cumsum(nb)]).astype(np.int32),
            pos=self.pos[:, bidx].copy(), quat=self.quat[:, bidx].copy(),
            vel=self.vel[:, bidx].copy(), angvel=self.angvel[:, bidx].copy(),
            shape_type=self.shape_type[bidx].copy(), shape_dims=self.shape_dims[:, bidx].copy(),
            inv_mass=self.inv_mass[bidx].copy(), inv_inertia=self.inv_inertia[:, bidx].copy(),
            mesh_id=self.mesh_id[bidx].copy(), mesh_scale=self.mesh_scale[:, bidx].copy(),
            albedo=self.albedo[bidx].copy(),
            cam_off=np.concatenate([[0], np.cumsum(nc)]).astype(np.int32),
            cam_w=self.cam_w[cidx].copy(), cam_h=self.cam_h[cidx].copy(),
            cam_eye=self.cam_eye[cidx].copy(), cam_right=self.cam_right[cidx].copy(),
            cam_up=self.cam_up[cidx].copy(), cam_fwd=self.cam_fwd[cidx].copy(),
            cam_fpy=self.cam_fpy[cidx].copy(),
            name=self.name + "[subset]")


def mass_properties(shape_type: np.ndarray, dims: np.ndarray):
    """Inverse mass and inverse principal inertia at DENSITY (double, cast)."""
    B = shape_type.shape[0]
    im = np.zeros(B, np.float64)
    ii = np.zeros((3, B), np.float64)
    for b in range(B):
        if shape_type[b] == SHAPE_BOX:
            a, bb, c = (float(x) for x in dims[:, b])
            m = DENSITY * 8.0 * a * bb * c
            I = (m * (bb * bb + c * c) / 3.0, m * (a * a + c * c) / 3.0, m * (a * a + bb * bb) / 3.0)
        else:
            r = float(dims[0, b])
            m = DENSITY * 4.0 / 3.0 * math.pi * r ** 3
            I = (0.4 * m * r * r,) * 3
        im[b] = 1.0 / m
        ii[:, b] = [1.0 / x for x in I]
    return im.astype(np.float32), ii.astype(np.float32)


def bounding_radius(shape_type, dims):
    r = dims[0].astype(np.float64).copy()
    box = shape_type == SHAPE_BOX
    r[box] = np.sqrt((dims[:, box].astype(np.float64) ** 2).sum(0))
    return r


def look_at(eye, target, fov_deg: float, h: int):
    """Camera basis and focal length in pixels, computed in double and cast."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, [0.0, 0.0, 1.0])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    fpy = (h / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return (eye.astype(np.float32), r.astype(np.float32), u.astype(np.float32),
            f.astype(np.float32), np.float32(fpy))


def _mesh_library(hulls: List = ()):
    meshes = [icosphere(1), cube(), ground_quad()] + list(hulls)
    voff = [0]
    toff = [0]
    for V, T in meshes:
        voff.append(voff[-1] + len(V))
        toff.append(toff[-1] + len(T))
    verts = np.concatenate([V for V, _ in meshes]).astype(np.float32)
    tris = np.concatenate([T for _, T in meshes]).astype(np.int32)
    return np.array(voff, np.int32), verts, np.array(toff, np.int32), tris


def _shoemake(st: Streams, mask=None):
    u1, u2, u3 = st.uniform(mask=mask), st.uniform(mask=mask), st.uniform(mask=mask)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    t2, t3 = 2.0 * np.pi * u2, 2.0 * np.pi * u3
    q = np.stack([b * np.cos(t3), a * np.sin(t2), a * np.cos(t2), b * np.sin(t3)])  # (w, x, y, z)
    return q / np.linalg.norm(q, axis=0)


def generate(num_envs: int, bodies, seed: int, *, kinds: str = "spheres",
             res=64, cams_per_env: int = 1, substeps: int = 4, n_hull_meshes: int = 64,
             hull_tris=(500, 2000), sphere_r=(0.05, 0.1), box_h=(0.03, 0.1),
             name: str = "", env_base: int = 0, height=None) -> Scene:
    """Build a seeded batch of environments.

    bodies: int (same count everywhere) or per-env int array.
    kinds: "spheres" | "mixed" (even index sphere, odd index box) | "hulls" |
    "mixed_hulls" (index mod 3: sphere, box, hull).
    res: int or per-env int array: camera width (and height, unless given).
    height: None (square cameras), or int / per-env int array of camera heights;
    the 60 degree field of view is vertical.
    """
    E = num_envs
    nb = np.full(E, bodies, np.int32) if np.isscalar(bodies) else np.asarray(bodies, np.int32)
    resv = np.full(E, res, np.int32) if np.isscalar(res) else np.asarray(res, np.int32)
    resh = resv.copy() if height is None else (np.full(E, height, np.int32) if np.isscalar(height)
                                                else np.asarray(height, np.int32))
    body_off = np.concatenate([[0], np.cumsum(nb)]).astype(np.int32)
    B = int(body_off[-1])
    nmax = int(nb.max()) if E else 0

    hulls = []
    if kinds in ("hulls", "mixed_hulls"):
        ms = Streams(seed ^ 0x4855_4C4C, 1)
        for _ in range(n_hull_meshes):
            lo, hi = hull_tris
            t = int(lo + (ms.next_u64()[0] % np.uint64((hi - lo) // 2 + 1)) * 2)
            hulls.append(convex_hull_mesh(ms, t))
    voff, verts, toff, tris = _mesh_library(hulls)

    st = Streams(seed, E, env_base)
    shape_type = np.zeros((E, nmax), np.uint8)
    dims = np.zeros((3, E, nmax), np.float64)
    quat = np.zeros((4, E, nmax), np.float64)
    quat[0] = 1.0
    pos = np.zeros((3, E, nmax), np.float64)
    mesh_id = np.zeros((E, nmax), np.int32)
    rad = np.zeros((E, nmax), np.float64)
    for b in range(nmax):
        act = nb > b
        if kinds == "mixed" and (b & 1):
            typ = SHAPE_BOX
        elif kinds == "hulls":
            typ = SHAPE_HULL
        elif kinds == "mixed_hulls":
            typ = (SHAPE_SPHERE, SHAPE_BOX, SHAPE_HULL)[b % 3]
        else:
            typ = SHAPE_SPHERE
        shape_type[:, b] = typ
        if typ == SHAPE_BOX:
            for k in range(3):
                dims[k, :, b] = st.uniform(box_h[0], box_h[1], act)
            quat[:, :, b] = _shoemake(st, act)
            mesh_id[:, b] = MESH_CUBE
            rad[:, b] = np.sqrt((dims[:, :, b] ** 2).sum(0))
        else:
            dims[0, :, b] = st.uniform(sphere_r[0], sphere_r[1], act)
            rad[:, b] = dims[0, :, b]
            if typ == SHAPE_HULL:
                mesh_id[:, b] = 3 + (st.next_u64(act) % np.uint64(n_hull_meshes)).astype(np.int32)
            else:
                mesh_id[:, b] = MESH_ICOSPHERE
        # rejection-sample a non-overlapping position, at most 100 tries
        span = np.sqrt(np.maximum(1.0, nb / 32.0))
        pending = act.copy()
        for _ in range(100):
            if not pending.any():
                break
            x = st.uniform(-0.5, 0.5, pending) * span
            y = st.uniform(-0.5, 0.5, pending) * span
            z = st.uniform(0.0, 1.0, pending)
            z = rad[:, b] + (1.0 - rad[:, b]) * z
            ok = np.ones(E, bool)
            if b > 0:
                d2 = (pos[0, :, :b] - x[:, None]) ** 2 + (pos[1, :, :b] - y[:, None]) ** 2 + \
                    (pos[2, :, :b] - z[:, None]) ** 2
                ok = ~((d2 < (rad[:, :b] + rad[:, b:b + 1]) ** 2) & (np.arange(b)[None, :] < nb[:, None])).any(1)
            upd = pending
            pos[0, upd, b], pos[1, upd, b], pos[2, upd, b] = x[upd], y[upd], z[upd]
            pending = pending & ~ok

    # flatten [E, nmax] -> CSR order
    sel = (np.arange(nmax)[None, :] < nb[:, None])
    flat = lambda a: a[..., sel] if a.ndim == 3 else a[sel]
    st_flat = flat(shape_type)
    dims_f = flat(dims).astype(np.float32)
    im, ii = mass_properties(st_flat, dims_f)
    scale = np.where(st_flat[None, :] == SHAPE_BOX, dims_f, dims_f[0:1].repeat(3, 0)).astype(np.float32)
    bidx_env = np.repeat(np.arange(E), nb)
    local = np.concatenate([np.arange(n) for n in nb]) if E else np.zeros(0, np.int64)
    albedo = np.array([pack_rgb(PALETTE[i % 8]) for i in local], np.uint32)
    del bidx_env

    ncam = np.full(E, cams_per_env, np.int32)
    cam_off = np.concatenate([[0], np.cumsum(ncam)]).astype(np.int32)
    C = int(cam_off[-1])
    cw = np.zeros(C, np.int32)
    ch = np.zeros(C, np.int32)
    eye = np.zeros((C, 3), np.float32)
    rr, uu, ff = (np.zeros((C, 3), np.float32) for _ in range(3))
    fpy = np.zeros(C, np.float32)
    eyes = [(0.0, -2.5, 1.5), (0.0, 2.5, 1.5)]
    cache = {}
    for e in range(E):
        for c in range(cams_per_env):
            i = cam_off[e] + c
            key = (c, int(resh[e]))
            if key not in cache:
                cache[key] = look_at(eyes[c % 2], (0.0, 0.0, 0.4), 60.0, int(resh[e]))
            eye[i], rr[i], uu[i], ff[i], fpy[i] = cache[key]
            cw[i] = resv[e]
            ch[i] = resh[e]
    L = np.array([0.3, -0.5, 0.8], np.float64)
    L = (L / np.linalg.norm(L)).astype(np.float32)

    params = SimParams(substeps=substeps)
    return Scene(
        body_off=body_off, pos=flat(pos).astype(np.float32), quat=flat(quat).astype(np.float32),
        vel=np.zeros((3, B), np.float32), angvel=np.zeros((3, B), np.float32),
        shape_type=st_flat.astype(np.uint8), shape_dims=dims_f, inv_mass=im, inv_inertia=ii,
        mesh_id=flat(mesh_id).astype(np.int32), mesh_scale=scale, albedo=albedo,
        mesh_vert_off=voff, mesh_verts=verts, mesh_tri_off=toff, mesh_tris=tris,
        ground_mesh=MESH_GROUND, ground_albedo=pack_rgb(GROUND_ALBEDO),
        cam_off=cam_off, cam_w=cw, cam_h=ch, cam_eye=eye, cam_right=rr, cam_up=uu,
        cam_fwd=ff, cam_fpy=fpy, light=L, params=params, name=name)


# ----------------------------------------------------------------------------
# The five workload recipes
# ----------------------------------------------------------------------------
def config_seed(k: int) -> int:
    return 0x5EED0000 + k


def cfg1(num_envs: int = 16) -> Scene:
    """16 envs x 8 spheres, 64x64 camera, 4 substeps of dt = 1/240 s."""
    return generate(num_envs, 8, config_seed(1), kinds="spheres", res=64, substeps=4,
                    name="cfg1: %d envs x 8 spheres, 64x64" % num_envs)


def cfg2(num_envs: int = 1024, env_base: int = 0) -> Scene:
    """1024 envs x 32 bodies (half spheres, half boxes), 8 substeps, 128x128."""
    return generate(num_envs, 32, config_seed(2), kinds="mixed", res=128, substeps=8,
                    name="cfg2: %d envs x 32 sphere/box bodies, 128x128" % num_envs, env_base=env_base)


def cfg3(num_envs: int = 4096, env_base: int = 0) -> Scene:
    """4096 envs x 64 convex-hull bodies (500-2000 tris), two 128x128 cameras."""
    return generate(num_envs, 64, config_seed(3), kinds="hulls", res=128, cams_per_env=2,
                    substeps=8, name="cfg3: %d envs x 64 hulls, 2 x 128x128" % num_envs,
                    env_base=env_base)


def cfg4_shape(num_envs: int = 2048, seed: int = config_seed(4)):
    st = Streams(seed ^ 0xC0FF_EE00, 1)
    nb = np.array([int(round(math.exp(st.uniform(math.log(4), math.log(256))[0]))) for _ in range(num_envs)],
                  np.int32)
    res = np.array([(64, 128, 256)[int(st.next_u64()[0] % np.uint64(3))] for _ in range(num_envs)], np.int32)
    return nb, res


def cfg4(num_envs: int = 2048) -> Scene:
    """2048 envs, body counts log-uniform in [4, 256], square cameras of 64, 128 or 256."""
    nb, res = cfg4_shape(num_envs)
    return generate(num_envs, nb, config_seed(4), kinds="mixed", res=res, substeps=8,
                    name="cfg4: %d uneven envs" % num_envs)


def custom(bodies: List[dict], *, res: int = 64, params: Optional[SimParams] = None,
           cams: Optional[List[dict]] = None, envs: int = 1) -> Scene:
    """A hand-placed scene for tests.  Each body dict: type ('sphere'|'box'|
    'hull'), r (sphere and hull radius) or h (half extents), mesh (a hull's
    unit-size (vertices, triangles), e.g. octahedron()), pos, quat (w,x,y,z),
    vel, angvel.  The same bodies are repeated in every env."""
    hull_meshes = []
    for b in bodies:
        if b["type"] == "hull" and not any(b["mesh"] is m for m in hull_meshes):
            hull_meshes.append(b["mesh"])
    voff, verts, toff, tris = _mesh_library(hull_meshes)
    n = len(bodies)
    B = n * envs
    kind = {"box": SHAPE_BOX, "sphere": SHAPE_SPHERE, "hull": SHAPE_HULL}
    typ = np.array([kind[b["type"]] for b in bodies] * envs, np.uint8)
    dims = np.zeros((3, B), np.float32)
    pos = np.zeros((3, B), np.float32)
    quat = np.zeros((4, B), np.float32)
    vel = np.zeros((3, B), np.float32)
    ang = np.zeros((3, B), np.float32)
    for e in range(envs):
        for i, b in enumerate(bodies):
            j = e * n + i
            if b["type"] == "box":
                dims[:, j] = b["h"]
            else:
                dims[0, j] = b["r"]
            pos[:, j] = b["pos"]
            quat[:, j] = b.get("quat", (1, 0, 0, 0))
            vel[:, j] = b.get("vel", (0, 0, 0))
            ang[:, j] = b.get("angvel", (0, 0, 0))
    im, ii = mass_properties(typ, dims)
    scale = np.where(typ[None, :] == SHAPE_BOX, dims, dims[0:1].repeat(3, 0)).astype(np.float32)
    mesh = np.where(typ == SHAPE_BOX, MESH_CUBE, MESH_ICOSPHERE).astype(np.int32)
    for e in range(envs):
        for i, b in enumerate(bodies):
            if b["type"] == "hull":
                mesh[e * n + i] = 3 + next(k for k, m in enumerate(hull_meshes) if m is b["mesh"])
    cams = cams or [dict(eye=(0.0, -2.5, 1.5), target=(0.0, 0.0, 0.4), fov=60.0)]
    C = len(cams) * envs
    eye = np.zeros((C, 3), np.float32)
    rr, uu, ff = (np.zeros((C, 3), np.float32) for _ in range(3))
    fpy = np.zeros(C, np.float32)
    for e in range(envs):
        for c, cd in enumerate(cams):
            i = e * len(cams) + c
            eye[i], rr[i], uu[i], ff[i], fpy[i] = look_at(cd["eye"], cd["target"], cd.get("fov", 60.0), res)
    L = np.array([0.3, -0.5, 0.8])
    L = (L / np.linalg.norm(L)).astype(np.float32)
    return Scene(
        body_off=(np.arange(envs + 1) * n).astype(np.int32), pos=pos, quat=quat, vel=vel, angvel=ang,
        shape_type=typ, shape_dims=dims, inv_mass=im, inv_inertia=ii, mesh_id=mesh, mesh_scale=scale,
        albedo=np.array([pack_rgb(PALETTE[i % 8]) for i in range(n)] * envs, np.uint32),
        mesh_vert_off=voff, mesh_verts=verts, mesh_tri_off=toff, mesh_tris=tris,
        ground_mesh=MESH_GROUND, ground_albedo=pack_rgb(GROUND_ALBEDO),
        cam_off=(np.arange(envs + 1) * len(cams)).astype(np.int32),
        cam_w=np.full(C, res, np.int32), cam_h=np.full(C, res, np.int32),
        cam_eye=eye, cam_right=rr, cam_up=uu, cam_fwd=ff, cam_fpy=fpy, light=L,
        params=params or SimParams(), name="custom")


def cfg5_jobs(num_jobs: int = 16, max_envs: int = 1024, max_bodies: int = 256, res_choices=(64, 128, 256),
              seed: int = config_seed(5)) -> List[Scene]:
    """Serving workload: jobs of log-uniform size in [16, max_envs] envs, each
    with its own body count (log-uniform in [4, max_bodies], spheres and boxes)
    and camera resolution."""
    st = Streams(seed ^ 0x5E4F_0005, 1)
    jobs = []
    for j in range(num_jobs):
        E = int(round(math.exp(st.uniform(math.log(16), math.log(max_envs))[0])))
        N = int(round(math.exp(st.uniform(math.log(4), math.log(max_bodies))[0])))
        res = int(res_choices[int(st.next_u64()[0] % np.uint64(len(res_choices)))])
        jobs.append(generate(E, N, seed + 1000 * (j + 1), kinds="mixed", res=res, substeps=8,
                             name="cfg5 job %d: %d envs x %d bodies, %dx%d" % (j, E, N, res, res)))
    return jobs
