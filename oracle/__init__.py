"""CPU oracle for the simulate-then-render step (Python side).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of the benchmark use it; the product path never imports it.  It loads
``liboracle.so`` built from ``oracle.c`` (plain C, gcc -O2
-ffp-contract=off) and shares no code with the CUDA library.

Functions:
  sim_step(scene, nsteps, state=None, precision="f32", force=None)
  contacts(scene, env, state=None)
  render(scene, pos, quat)
  raster_screen_tris(xy, z, W, H, count=False)
  observe(scene, rgb, depth, cells, depth_scale)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "physics.inc")]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no fast-math, no FP contraction)."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
               "-o", tmp, _SRC[0], "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("substeps", C.c_int), ("iterations", C.c_int),
                ("gravity", C.c_double * 3), ("restitution", C.c_double),
                ("restitution_threshold", C.c_double), ("friction", C.c_double),
                ("baumgarte", C.c_double), ("slop", C.c_double), ("margin", C.c_double),
                ("jacobi_omega", C.c_double), ("plane", C.c_int), ("max_contacts_per_body", C.c_int),
                ("gyroscopic", C.c_int), ("edge_contacts", C.c_int), ("hull_contacts", C.c_int),
                ("mesh_id", C.c_void_p), ("mesh_vert_off", C.c_void_p), ("mesh_verts", C.c_void_p),
                ("mesh_tri_off", C.c_void_p), ("mesh_tris", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _params(p, scene=None, mesh_id=None) -> _Params:
    """Parameters; with hull contacts also the scene's meshes (mesh_id: the
    bodies' meshes in the entry point's indexing, default all the scene's)."""
    P = _Params(p.dt, p.substeps, p.iterations, (C.c_double * 3)(*p.gravity), p.restitution,
                p.restitution_threshold, p.friction, p.baumgarte, p.slop, p.margin, p.jacobi_omega,
                p.plane, p.max_contacts_per_body, p.gyroscopic, p.edge_contacts, getattr(p, "hull_contacts", 0))
    if P.hull_contacts and scene is not None:
        keep = [np.ascontiguousarray(scene.mesh_id if mesh_id is None else mesh_id, np.int32),
                np.ascontiguousarray(scene.mesh_vert_off, np.int32), np.ascontiguousarray(scene.mesh_verts, np.float32),
                np.ascontiguousarray(scene.mesh_tri_off, np.int32), np.ascontiguousarray(scene.mesh_tris, np.int32)]
        P.mesh_id, P.mesh_vert_off, P.mesh_verts, P.mesh_tri_off, P.mesh_tris = (a.ctypes.data for a in keep)
        P._keep = keep   # the arrays live as long as the parameters
    return P


def sim_step(scene, nsteps: int = 1, state: Optional[dict] = None, precision: str = "f32",
             force: Optional[np.ndarray] = None, params=None):
    """Advance all environments by nsteps.  Returns (state dict, env_flags,
    contact_count).  state defaults to the scene's initial state."""
    dt = np.float32 if precision == "f32" else np.float64
    st = state if state is not None else scene.state()
    s = {k: np.ascontiguousarray(st[k], dtype=dt).copy() for k in ("pos", "quat", "vel", "angvel")}
    dims = np.ascontiguousarray(scene.shape_dims, dtype=dt)
    im = np.ascontiguousarray(scene.inv_mass, dtype=dt)
    ii = np.ascontiguousarray(scene.inv_inertia, dtype=dt)
    f = None if force is None else np.ascontiguousarray(force, dtype=dt)
    E = scene.num_envs
    flags = np.zeros(E, np.uint32)
    cc = np.zeros(E, np.int32)
    P = _params(params or scene.params, scene)
    fn = lib().oracle_sim_step_f32 if precision == "f32" else lib().oracle_sim_step_f64
    rc = fn(C.c_int(E), _ptr(np.ascontiguousarray(scene.body_off, np.int32)), C.c_int(scene.num_bodies),
            _ptr(s["pos"]), _ptr(s["quat"]), _ptr(s["vel"]), _ptr(s["angvel"]),
            _ptr(np.ascontiguousarray(scene.shape_type, np.uint8)), _ptr(dims), _ptr(im), _ptr(ii), _ptr(f),
            C.byref(P), C.c_int(nsteps), _ptr(flags), _ptr(cc))
    if rc != 0:
        raise ValueError("oracle_sim_step rejected its arguments")
    return s, flags, cc


def contacts(scene, env: int, state: Optional[dict] = None, params=None):
    """Canonical contact list of one environment at the given state."""
    st = state if state is not None else scene.state()
    b0, b1 = int(scene.body_off[env]), int(scene.body_off[env + 1])
    n = b1 - b0
    pos = np.ascontiguousarray(st["pos"][:, b0:b1], np.float32)
    quat = np.ascontiguousarray(st["quat"][:, b0:b1], np.float32)
    dims = np.ascontiguousarray(scene.shape_dims[:, b0:b1], np.float32)
    typ = np.ascontiguousarray(scene.shape_type[b0:b1], np.uint8)
    P = _params(params or scene.params, scene, scene.mesh_id[b0:b1])
    cap = max(1, P.max_contacts_per_body * n)
    a = np.zeros(cap, np.int32)
    b = np.zeros(cap, np.int32)
    nrm = np.zeros((cap, 3), np.float32)
    pt = np.zeros((cap, 3), np.float32)
    d = np.zeros(cap, np.float32)
    nc = lib().oracle_contacts_f32(C.c_int(n), _ptr(pos), _ptr(quat), _ptr(typ), _ptr(dims), C.byref(P),
                                   C.c_int(cap), _ptr(a), _ptr(b), _ptr(nrm), _ptr(pt), _ptr(d))
    if nc < 0:
        raise ValueError("oracle_contacts rejected its arguments")
    k = min(nc, cap)
    return dict(a=a[:k], b=b[:k], n=nrm[:k], p=pt[:k], d=d[:k], count=nc)


def render(scene, pos: Optional[np.ndarray] = None, quat: Optional[np.ndarray] = None, triid: bool = True):
    """Render every camera.  Returns (rgb u8 [px,3], depth f32 [px], triid u32 [px], env_flags)."""
    pos = np.ascontiguousarray(scene.pos if pos is None else pos, np.float32)
    quat = np.ascontiguousarray(scene.quat if quat is None else quat, np.float32)
    pix = scene.cam_pix_off()
    npx = int(pix[-1])
    rgb = np.zeros((npx, 3), np.uint8)
    depth = np.zeros(npx, np.float32)
    tid = np.zeros(npx, np.uint32) if triid else None
    flags = np.zeros(scene.num_envs, np.uint32)
    c32 = lambda a: np.ascontiguousarray(a, np.int32)
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    rc = lib().oracle_render(
        C.c_int(scene.num_envs), _ptr(c32(scene.body_off)), C.c_int(scene.num_bodies), _ptr(pos), _ptr(quat),
        _ptr(c32(scene.mesh_id)), _ptr(f32(scene.mesh_scale)), _ptr(np.ascontiguousarray(scene.albedo, np.uint32)),
        _ptr(c32(scene.mesh_vert_off)), _ptr(f32(scene.mesh_verts)), _ptr(c32(scene.mesh_tri_off)),
        _ptr(c32(scene.mesh_tris)), C.c_int(scene.ground_mesh), C.c_uint32(scene.ground_albedo),
        _ptr(c32(scene.cam_off)), _ptr(c32(scene.cam_w)), _ptr(c32(scene.cam_h)),
        _ptr(f32(scene.cam_eye)), _ptr(f32(scene.cam_right)), _ptr(f32(scene.cam_up)), _ptr(f32(scene.cam_fwd)),
        _ptr(f32(scene.cam_fpy)), _ptr(f32(scene.light)), _ptr(np.ascontiguousarray(pix, np.int64)),
        _ptr(rgb), _ptr(depth), _ptr(tid), _ptr(flags))
    if rc != 0:
        raise ValueError("oracle_render rejected its arguments")
    return rgb, depth, tid, flags


def raster_screen_tris(xy: np.ndarray, z: np.ndarray, W: int, H: int, count: bool = False):
    """Rasterise snapped 24.8 fixed-point triangles xy[t,3,2] with view
    depths z[t,3].  Returns (triid u32 [H,W], depth f32 [H,W], count or None)."""
    xy = np.ascontiguousarray(xy, np.int32).reshape(-1, 3, 2)
    z = np.ascontiguousarray(z, np.float32).reshape(-1, 3)
    tid = np.zeros((H, W), np.uint32)
    dep = np.zeros((H, W), np.float32)
    cnt = np.zeros((H, W), np.int32) if count else None
    rc = lib().oracle_raster_screen_tris(_ptr(xy), _ptr(z), C.c_int(xy.shape[0]), C.c_int(W), C.c_int(H),
                                         _ptr(tid), _ptr(dep), _ptr(cnt))
    if rc != 0:
        raise ValueError("oracle_raster_screen_tris rejected its arguments")
    return tid, dep, cnt


def observe(scene, rgb: np.ndarray, depth: np.ndarray, cells: int, depth_scale: float) -> np.ndarray:
    """Pooled observation of a rendered frame, the policy input of the RL
    rollout (Sec. 3.1 and 6.4: the policy acts on what the renderer produced
    for the step; the pooling itself is a reading, since the paper's
    policies read full frames): every camera is cut into cells x cells
    cells of (W / cells) x (H / cells) pixels, row-major; per cell the mean
    view depth (background 0) times depth_scale, and the mean luminance
    (0.299 R + 0.587 G + 0.114 B) / 255.  Output [E][2 * cams_per_env *
    cells^2]: the depth cells of the environment's cameras in order, then
    their luminance cells.  Plain float64, no blocking."""
    off = scene.cam_pix_off()
    ncam = np.diff(scene.cam_off)
    cpe = int(ncam[0]) if len(ncam) else 0
    if len(ncam) and not (ncam == cpe).all():
        raise ValueError("observe needs the same number of cameras in every environment")
    E = len(ncam)
    n = cells * cells
    out = np.zeros((E, 2 * cpe * n), np.float64)
    for c in range(int(scene.cam_off[-1]) if E else 0):
        e, k = c // cpe, c % cpe
        W, H = int(scene.cam_w[c]), int(scene.cam_h[c])
        if W % cells or H % cells:
            raise ValueError("camera %d: %d x %d pixels do not divide into %d x %d cells" % (c, W, H, cells, cells))
        cw, ch = W // cells, H // cells
        d = np.asarray(depth[off[c]:off[c + 1]], np.float64).reshape(H, W)
        px = np.asarray(rgb[off[c]:off[c + 1]], np.float64).reshape(H, W, 3)
        lum = (0.299 * px[:, :, 0] + 0.587 * px[:, :, 1] + 0.114 * px[:, :, 2]) / 255.0
        for cy in range(cells):
            for cx in range(cells):
                ys, xs = slice(cy * ch, (cy + 1) * ch), slice(cx * cw, (cx + 1) * cw)
                out[e, k * n + cy * cells + cx] = d[ys, xs].mean() * depth_scale
                out[e, (cpe + k) * n + cy * cells + cx] = lum[ys, xs].mean()
    return out
