"""Thin ctypes binding of libvuda.so (include/vuda.h).

Argument marshalling only: every step of the simulate-then-render path runs
in the library's CUDA kernels.  PyTorch supplies device memory (frames,
forces) and streams.  Importing this module raises if the library has not
been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# VUDA_LIBRARY selects another build of the same library (e.g. an instrumented one)
LIB_PATH = os.environ.get("VUDA_LIBRARY") or os.path.join(_HERE, "libvuda.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libvuda.so is not built (python -m paper_2605_01352_b300.build); "
                      "the CUDA library is required and there is no fallback")

lib = C.CDLL(LIB_PATH)

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_OVERFLOW, ERR_TIMEOUT, ERR_BUSY, ERR_UNSUPPORTED = range(8)
FLAG_CONTACT_OVERFLOW, FLAG_CLIP_CAPACITY, FLAG_GUARD_DISCARD, FLAG_MESH_CAPACITY, FLAG_BAD_RANGE = 1, 2, 4, 8, 16
COSCHED_STREAMS, COSCHED_GREEN, COSCHED_SHARED = 1, 2, 3
RENDER_AUTO, RENDER_BAND, RENDER_TILED = 0, 1, 2
PRIORITY_NONE, PRIORITY_SIM, PRIORITY_RENDER = 0, 1, 2

vp = C.c_void_p


class SimParams(C.Structure):
    _fields_ = [("dt", C.c_float), ("substeps", C.c_int32), ("iterations", C.c_int32),
                ("gravity", C.c_float * 3), ("restitution", C.c_float), ("restitution_threshold", C.c_float),
                ("friction", C.c_float), ("baumgarte", C.c_float), ("slop", C.c_float), ("margin", C.c_float),
                ("jacobi_omega", C.c_float), ("plane", C.c_int32), ("max_contacts_per_body", C.c_int32),
                ("gyroscopic", C.c_int32), ("edge_contacts", C.c_int32), ("hull_contacts", C.c_int32)]


class Scene(C.Structure):
    _fields_ = [("num_envs", C.c_int32), ("body_off", vp), ("pos", vp), ("quat", vp), ("vel", vp),
                ("angvel", vp), ("shape_type", vp), ("shape_dims", vp), ("inv_mass", vp), ("inv_inertia", vp),
                ("mesh_id", vp), ("mesh_scale", vp), ("albedo", vp), ("num_meshes", C.c_int32),
                ("mesh_vert_off", vp), ("mesh_verts", vp), ("mesh_tri_off", vp), ("mesh_tris", vp),
                ("ground_mesh", C.c_int32), ("ground_albedo", C.c_uint32), ("cam_off", vp), ("cam_w", vp),
                ("cam_h", vp), ("cam_eye", vp), ("cam_right", vp), ("cam_up", vp), ("cam_fwd", vp),
                ("cam_fpy", vp), ("light", C.c_float * 3)]


class EnvOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("device", C.c_int32), ("render_band_rows", C.c_int32),
                ("phys_smem_bytes", C.c_int32), ("persistent", C.c_int32), ("render_path", C.c_int32),
                ("tile_size", C.c_int32), ("tile_bin_limit", C.c_int32)]


class EnvInfo(C.Structure):
    _fields_ = [("num_envs", C.c_int32), ("num_bodies", C.c_int32), ("num_cams", C.c_int32),
                ("max_bodies", C.c_int32), ("num_pixels", C.c_int64), ("num_tris", C.c_int64),
                ("device_bytes", C.c_int64), ("steps_enqueued", C.c_int64), ("render_path", C.c_int32),
                ("tile_size", C.c_int32), ("tile_bin_limit", C.c_int32)]


class Frame(C.Structure):
    _fields_ = [("rgb", vp), ("depth", vp), ("triid", vp)]


class State(C.Structure):
    _fields_ = [("pos", vp), ("quat", vp), ("vel", vp), ("angvel", vp)]


class Timing(C.Structure):
    _fields_ = [("step_ms", vp), ("sim_ms", vp), ("render_ms", vp), ("total_ms", C.c_float)]


class TuneOpts(C.Structure):
    _fields_ = [("steps", C.c_int32), ("use_cache", C.c_int32)]


class TuneResult(C.Structure):
    _fields_ = [("band_rows", C.c_int32), ("cosched_mode", C.c_int32), ("sim_sms", C.c_int32),
                ("graph_steps", C.c_int32), ("ms_per_step", C.c_float), ("ms_per_step_serialized", C.c_float),
                ("trials", C.c_int32), ("from_cache", C.c_int32), ("sim_ctas_per_sm", C.c_int32),
                ("render_ctas_per_sm", C.c_int32), ("priority", C.c_int32), ("tile_size", C.c_int32),
                ("tile_bin_limit", C.c_int32)]


class CoschedOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("sim_sms", C.c_int32), ("sim_ctas_per_sm", C.c_int32),
                ("render_ctas_per_sm", C.c_int32), ("priority", C.c_int32)]


class CoschedInfo(C.Structure):
    _fields_ = [("mode", C.c_int32), ("sim_sms", C.c_int32), ("render_sms", C.c_int32),
                ("sm_granularity", C.c_int32), ("sim_ctas_per_sm", C.c_int32), ("render_ctas_per_sm", C.c_int32),
                ("priority", C.c_int32)]


def _sig(name, args, res=C.c_int):
    f = getattr(lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("vuda_status_str", [C.c_int], C.c_char_p)
_sig("vuda_last_error", [], C.c_char_p)
_sig("vuda_abi_version", [], C.c_int32)
_sig("vuda_env_create", [C.POINTER(Scene), C.POINTER(SimParams), C.POINTER(EnvOpts), C.POINTER(vp)])
_sig("vuda_env_destroy", [vp])
_sig("vuda_env_estimate_bytes", [C.POINTER(Scene), C.POINTER(SimParams), C.POINTER(C.c_int64)])
_sig("vuda_env_info_get", [vp, C.POINTER(EnvInfo)])
_sig("vuda_env_cam_pix_off", [vp, vp])
_sig("vuda_sim_step", [vp, C.c_int32, vp, vp])
_sig("vuda_render", [vp, C.c_int32, C.POINTER(Frame), vp])
_sig("vuda_coschedule", [vp, C.POINTER(CoschedOpts), C.POINTER(vp), C.POINTER(vp), C.POINTER(CoschedInfo)])
_sig("vuda_coschedule_reset", [vp])
_sig("vuda_pipeline_run", [vp, C.c_int32, C.POINTER(Frame), vp, C.POINTER(Timing)])
_sig("vuda_pipeline_run_host", [vp, C.c_int32, vp, C.c_int32, vp, vp, C.POINTER(Frame), vp, C.POINTER(Timing)])
_sig("vuda_pipeline_capture", [vp, C.c_int32, C.POINTER(Frame), vp])
_sig("vuda_pipeline_release_graph", [vp])
_sig("vuda_autotune", [vp, C.POINTER(TuneOpts), C.POINTER(Frame), C.POINTER(TuneResult)])
_sig("vuda_set_tiling", [vp, C.c_int32, C.c_int32])
_sig("vuda_wait", [vp, C.c_int32])
_sig("vuda_env_get_state", [vp, C.POINTER(State)])
_sig("vuda_env_set_state", [vp, C.POINTER(State)])
_sig("vuda_env_get_pose", [vp, C.c_int32, vp, vp])
_sig("vuda_env_set_pose", [vp, C.c_int32, vp, vp])
_sig("vuda_env_status", [vp, vp, vp, C.c_int32])
_sig("vuda_env_contact_counts", [vp, vp])
_sig("vuda_raster_screen_tris", [vp, vp, C.c_int32, C.c_int32, C.c_int32, vp, vp, vp, vp])
_sig("vuda_observe", [vp, C.POINTER(Frame), C.c_int32, C.c_float, vp, vp])
PolicyFn = C.CFUNCTYPE(C.c_int32, vp, C.c_int32, C.c_int64, C.POINTER(Frame), vp, vp)
_sig("vuda_rollout_run", [vp, vp, C.c_int32, C.POINTER(Frame), C.POINTER(Frame), vp, vp, PolicyFn, vp, vp,
                          C.POINTER(Timing)])
_sig("vuda_sim_step_noalloc", [C.c_int32, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                               C.POINTER(SimParams), C.c_int32, vp, vp, vp, C.c_int32, vp])


class VudaError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib.vuda_last_error().decode(errors="replace")
        super().__init__("%s: %s (%s)" % (where, lib.vuda_status_str(status).decode(), msg))
        self.status = status


def check(status: int, where: str):
    if status != OK:
        raise VudaError(status, where)


def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _ptr(a):
    return None if a is None else vp(a.ctypes.data)


def _dptr(t):
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return vp(t.data_ptr())


def _stream(s):
    if s is None:
        import torch
        return vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return vp(s)
    return vp(s.cuda_stream)


def sim_params(p) -> SimParams:
    return SimParams(p.dt, p.substeps, p.iterations, (C.c_float * 3)(*p.gravity), p.restitution,
                     p.restitution_threshold, p.friction, p.baumgarte, p.slop, p.margin, p.jacobi_omega,
                     p.plane, p.max_contacts_per_body, p.gyroscopic, p.edge_contacts,
                     getattr(p, "hull_contacts", 0))


def scene_struct(scene):
    """vuda_scene view of a paper_2605_01352_b300.scene.Scene; the second value
    keeps the numpy buffers alive for the duration of the call."""
    keep = []

    def h(a, dt):
        x = _np(a, dt)
        keep.append(x)
        return _ptr(x)

    sc = Scene()
    sc.num_envs = scene.num_envs
    sc.body_off = h(scene.body_off, np.int32)
    sc.pos = h(scene.pos, np.float32)
    sc.quat = h(scene.quat, np.float32)
    sc.vel = h(scene.vel, np.float32)
    sc.angvel = h(scene.angvel, np.float32)
    sc.shape_type = h(scene.shape_type, np.uint8)
    sc.shape_dims = h(scene.shape_dims, np.float32)
    sc.inv_mass = h(scene.inv_mass, np.float32)
    sc.inv_inertia = h(scene.inv_inertia, np.float32)
    sc.mesh_id = h(scene.mesh_id, np.int32)
    sc.mesh_scale = h(scene.mesh_scale, np.float32)
    sc.albedo = h(scene.albedo, np.uint32)
    sc.num_meshes = len(scene.mesh_vert_off) - 1
    sc.mesh_vert_off = h(scene.mesh_vert_off, np.int32)
    sc.mesh_verts = h(scene.mesh_verts, np.float32)
    sc.mesh_tri_off = h(scene.mesh_tri_off, np.int32)
    sc.mesh_tris = h(scene.mesh_tris, np.int32)
    sc.ground_mesh = scene.ground_mesh
    sc.ground_albedo = scene.ground_albedo
    sc.cam_off = h(scene.cam_off, np.int32)
    sc.cam_w = h(scene.cam_w, np.int32)
    sc.cam_h = h(scene.cam_h, np.int32)
    sc.cam_eye = h(scene.cam_eye, np.float32)
    sc.cam_right = h(scene.cam_right, np.float32)
    sc.cam_up = h(scene.cam_up, np.float32)
    sc.cam_fwd = h(scene.cam_fwd, np.float32)
    sc.cam_fpy = h(scene.cam_fpy, np.float32)
    sc.light = (C.c_float * 3)(*[float(x) for x in scene.light])
    return sc, keep


def estimate_bytes(scene, params=None) -> int:
    """Device bytes a batch of this scene would hold (host-side estimate)."""
    sc, keep = scene_struct(scene)
    out = C.c_int64()
    check(lib.vuda_env_estimate_bytes(C.byref(sc), C.byref(sim_params(params or scene.params)), C.byref(out)),
          "vuda_env_estimate_bytes")
    return out.value


class Env:
    """A batch of environments resident on the GPU."""

    def __init__(self, scene, params=None, hbm_budget_bytes: int = 0, device: int = 0, band_rows: int = 0,
                 phys_smem_bytes: int = 0, persistent: bool = False, render_path: int = 0, tile_size: int = 0,
                 tile_bin_limit: int = 0, _handle=None):
        self.scene = scene
        if _handle is not None:            # a handle owned elsewhere (a serving job)
            self.h = _handle
            self._owned = False
            self._read_info()
            return
        self._owned = True
        sc, keep = scene_struct(scene)
        self.params = params or scene.params
        prm = sim_params(self.params)
        opts = EnvOpts(hbm_budget_bytes, device, band_rows, phys_smem_bytes, int(persistent), render_path,
                       tile_size, tile_bin_limit)
        handle = vp()
        check(lib.vuda_env_create(C.byref(sc), C.byref(prm), C.byref(opts), C.byref(handle)), "vuda_env_create")
        del keep
        self.h = handle
        self._read_info()

    def _read_info(self):
        info = EnvInfo()
        check(lib.vuda_env_info_get(self.h, C.byref(info)), "vuda_env_info_get")
        self.E, self.B, self.C = info.num_envs, info.num_bodies, info.num_cams
        self.P = info.num_pixels
        self.T = info.num_tris
        self.device_bytes = info.device_bytes
        pix = np.zeros(self.C + 1, np.int64)
        check(lib.vuda_env_cam_pix_off(self.h, _ptr(pix)), "vuda_env_cam_pix_off")
        self.cam_pix_off = pix
        self.sim_stream = None
        self.render_stream = None
        self.cosched = None

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lib.vuda_env_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> EnvInfo:
        i = EnvInfo()
        check(lib.vuda_env_info_get(self.h, C.byref(i)), "vuda_env_info_get")
        return i

    def set_tiling(self, tile_size: int, bin_limit: int):
        """Tile edge (8, 16, 32) and bin limit of the tiled render path."""
        check(lib.vuda_set_tiling(self.h, tile_size, bin_limit), "vuda_set_tiling")

    # -- frames -------------------------------------------------------------------
    def alloc_frame(self, triid: bool = True):
        import torch
        dev = torch.device("cuda")
        return dict(rgb=torch.empty((self.P, 3), dtype=torch.uint8, device=dev),
                    depth=torch.empty(self.P, dtype=torch.float32, device=dev),
                    triid=torch.empty(self.P, dtype=torch.int32, device=dev) if triid else None)

    @staticmethod
    def frame_struct(fr) -> Frame:
        return Frame(_dptr(fr["rgb"]), _dptr(fr["depth"]), _dptr(fr.get("triid")))

    # -- the two phases -----------------------------------------------------------
    def sim_step(self, nsteps: int = 1, force=None, stream=None):
        check(lib.vuda_sim_step(self.h, nsteps, _dptr(force), _stream(stream)), "vuda_sim_step")

    def render(self, frame, pose_slot: int = -1, stream=None):
        fs = self.frame_struct(frame)
        check(lib.vuda_render(self.h, pose_slot, C.byref(fs), _stream(stream)), "vuda_render")

    def observe(self, frame, cells: int, depth_scale: float, out, stream=None):
        """Pooled observation of a frame (vuda_observe) into the device tensor
        out [E, 2 * cameras per env * cells^2] (float32)."""
        fs = self.frame_struct(frame)
        check(lib.vuda_observe(self.h, C.byref(fs), cells, depth_scale, _dptr(out), _stream(stream)), "vuda_observe")

    # -- co-scheduling ----------------------------------------------------------------
    def coschedule(self, mode: int = COSCHED_GREEN, sim_sms: int = 0, sim_ctas_per_sm: int = 0,
                   render_ctas_per_sm: int = 0, priority: int = 0):
        import torch
        s1, s2 = vp(), vp()
        info = CoschedInfo()
        opts = CoschedOpts(mode, sim_sms, sim_ctas_per_sm, render_ctas_per_sm, priority)
        check(lib.vuda_coschedule(self.h, C.byref(opts), C.byref(s1), C.byref(s2), C.byref(info)),
              "vuda_coschedule")
        self.sim_stream = torch.cuda.ExternalStream(s1.value)
        self.render_stream = torch.cuda.ExternalStream(s2.value)
        self.cosched = dict(mode=info.mode, sim_sms=info.sim_sms, render_sms=info.render_sms,
                            sm_granularity=info.sm_granularity, sim_ctas_per_sm=info.sim_ctas_per_sm,
                            render_ctas_per_sm=info.render_ctas_per_sm, priority=info.priority)
        return self.cosched

    def coschedule_reset(self):
        check(lib.vuda_coschedule_reset(self.h), "vuda_coschedule_reset")
        self.sim_stream = self.render_stream = None
        self.cosched = None

    @staticmethod
    def _timing(n):
        arr = {k: np.zeros(max(n, 1), np.float32) for k in ("step_ms", "sim_ms", "render_ms")}
        tm = Timing(_ptr(arr["step_ms"]), _ptr(arr["sim_ms"]), _ptr(arr["render_ms"]), 0.0)
        return tm, arr

    @staticmethod
    def _timing_out(tm, arr, n):
        out = {k: v[:n] for k, v in arr.items()}
        out["total_ms"] = float(tm.total_ms)
        return out

    def pipeline_run(self, nsteps: int, ring: Sequence[dict], stream=None, timing: bool = False):
        """Run the loop (pipelined when co-scheduled).  With timing=True
        returns dict(step_ms, sim_ms, render_ms, total_ms)."""
        frames = (Frame * 2)(self.frame_struct(ring[0]), self.frame_struct(ring[1 % len(ring)]))
        tm, arr = self._timing(nsteps) if timing else (None, None)
        check(lib.vuda_pipeline_run(self.h, nsteps, frames, _stream(stream), C.byref(tm) if timing else None),
              "vuda_pipeline_run")
        return self._timing_out(tm, arr, nsteps) if timing else None

    def pipeline_run_host(self, nsteps: int, ring: Sequence[dict], h_rgb, h_depth, h_force=None,
                          force_per_step: bool = False, stream=None, timing: bool = False):
        """Loop with host buffers: h_force (pinned torch CPU tensor [3,B] or
        [nsteps,3,B]) in, frames out into the pinned host ring h_rgb [2,P,3],
        h_depth [2,P]."""
        frames = (Frame * 2)(self.frame_struct(ring[0]), self.frame_struct(ring[1 % len(ring)]))
        tm, arr = self._timing(nsteps) if timing else (None, None)
        hf = None if h_force is None else vp(h_force.data_ptr())
        check(lib.vuda_pipeline_run_host(self.h, nsteps, hf, int(force_per_step), vp(h_rgb.data_ptr()),
                                         vp(h_depth.data_ptr()), frames, _stream(stream),
                                         C.byref(tm) if timing else None), "vuda_pipeline_run_host")
        return self._timing_out(tm, arr, nsteps) if timing else None

    def pipeline_capture(self, steps_per_graph: int, ring: Sequence[dict], stream=None):
        """Capture steps_per_graph pipelined steps into a CUDA graph that later
        pipeline_run calls with this ring replay."""
        frames = (Frame * 2)(self.frame_struct(ring[0]), self.frame_struct(ring[1 % len(ring)]))
        check(lib.vuda_pipeline_capture(self.h, steps_per_graph, frames, _stream(stream)), "vuda_pipeline_capture")

    def pipeline_release_graph(self):
        check(lib.vuda_pipeline_release_graph(self.h), "vuda_pipeline_release_graph")

    def autotune(self, ring: Sequence[dict], steps: int = 6, use_cache: bool = True) -> dict:
        """Measure candidate configurations and keep the fastest (see vuda.h)."""
        frames = (Frame * 2)(self.frame_struct(ring[0]), self.frame_struct(ring[1 % len(ring)]))
        r = TuneResult()
        check(lib.vuda_autotune(self.h, C.byref(TuneOpts(steps, int(use_cache))), frames, C.byref(r)),
              "vuda_autotune")
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def wait(self, phase: int):
        check(lib.vuda_wait(self.h, phase), "vuda_wait")

    # -- state ------------------------------------------------------------------------
    def get_state(self):
        B = self.B
        s = dict(pos=np.zeros((3, B), np.float32), quat=np.zeros((4, B), np.float32),
                 vel=np.zeros((3, B), np.float32), angvel=np.zeros((3, B), np.float32))
        st = State(_ptr(s["pos"]), _ptr(s["quat"]), _ptr(s["vel"]), _ptr(s["angvel"]))
        check(lib.vuda_env_get_state(self.h, C.byref(st)), "vuda_env_get_state")
        return s

    def set_state(self, s):
        arrs = {k: _np(s[k], np.float32) for k in ("pos", "quat", "vel", "angvel")}
        st = State(*[_ptr(arrs[k]) for k in ("pos", "quat", "vel", "angvel")])
        check(lib.vuda_env_set_state(self.h, C.byref(st)), "vuda_env_set_state")

    def get_pose(self, slot: int):
        pos = np.zeros((3, self.B), np.float32)
        quat = np.zeros((4, self.B), np.float32)
        check(lib.vuda_env_get_pose(self.h, slot, _ptr(pos), _ptr(quat)), "vuda_env_get_pose")
        return pos, quat

    def set_pose(self, slot: int, pos, quat):
        p = _np(pos, np.float32)
        q = _np(quat, np.float32)
        check(lib.vuda_env_set_pose(self.h, slot, _ptr(p), _ptr(q)), "vuda_env_set_pose")

    def status(self, clear: bool = False):
        f = np.zeros(max(self.E, 1), np.uint32)
        o = C.c_uint32()
        check(lib.vuda_env_status(self.h, _ptr(f), C.byref(o), int(clear)), "vuda_env_status")
        return f[:self.E], int(o.value)

    def contact_counts(self):
        c = np.zeros(max(self.E, 1), np.int32)
        check(lib.vuda_env_contact_counts(self.h, _ptr(c)), "vuda_env_contact_counts")
        return c[:self.E]


def rollout_run(g0: "Env", g1: "Env", nsteps: int, ring0: Sequence[dict], ring1: Sequence[dict], force0, force1,
                policy, stream=None, timing: bool = False):
    """vuda_rollout_run: two groups of trajectories (batches g0, g1), each
    step sim -> render -> policy, one group's sim beside the other's render
    and policy when g0 is co-scheduled (see vuda.h).  policy(group, step,
    slot, stream) enqueues the group's policy on `stream` (a torch stream):
    it reads ring_g[slot] and writes force_g (device tensors [3, B_g]).
    With timing=True returns the device time in ms (NaN if unavailable)."""
    import torch
    rings = (ring0, ring1)
    slots = [{int(f["depth"].data_ptr()): i for i, f in enumerate(r)} for r in rings]
    streams = {}
    err = []

    def cb(user, group, step, frame, force, strm):
        try:
            ptr = int(strm or 0)
            ts = streams.get(ptr)
            if ts is None:
                ts = torch.cuda.ExternalStream(ptr) if ptr else torch.cuda.default_stream()
                streams[ptr] = ts
            slot = slots[group][int(frame.contents.depth or 0)]
            policy(int(group), int(step), slot, ts)
            return 0
        except Exception as ex:  # reported after the call returns
            err.append(ex)
            return 1

    fn = PolicyFn(cb)
    fr0 = (Frame * 2)(Env.frame_struct(ring0[0]), Env.frame_struct(ring0[1 % len(ring0)]))
    fr1 = (Frame * 2)(Env.frame_struct(ring1[0]), Env.frame_struct(ring1[1 % len(ring1)]))
    tm = Timing(None, None, None, 0.0)
    st = lib.vuda_rollout_run(g0.h, g1.h, nsteps, fr0, fr1, _dptr(force0), _dptr(force1), fn, None,
                              _stream(stream), C.byref(tm) if timing else None)
    if err:
        raise err[0]
    check(st, "vuda_rollout_run")
    return float(tm.total_ms) if timing else None


def raster_screen_tris(xy, z, W: int, H: int, count: bool = False, stream=None):
    """Rasterise snapped 24.8 fixed-point triangles (torch int32 [n,3,2] and
    float32 [n,3] on the GPU).  Returns (triid, depth, count) device tensors."""
    import torch
    dev = xy.device
    tid = torch.empty((H, W), dtype=torch.int32, device=dev)
    dep = torch.empty((H, W), dtype=torch.float32, device=dev)
    cnt = torch.empty((H, W), dtype=torch.int32, device=dev) if count else None
    n = int(xy.shape[0])
    check(lib.vuda_raster_screen_tris(_dptr(xy.contiguous()) if n else None, _dptr(z.contiguous()) if n else None,
                                      n, W, H, _dptr(tid), _dptr(dep), _dptr(cnt), _stream(stream)),
          "vuda_raster_screen_tris")
    return tid, dep, cnt


def sim_step_noalloc(arrays: dict, params, nsteps: int, max_bodies: int, smem_per_env: int = 0, stream=None):
    """Physics step on caller-owned device tensors without any device
    allocation by the library (see vuda_sim_step_noalloc in vuda.h).
    arrays: body_off, pos, quat, vel, angvel, shape_type, shape_dims,
    inv_mass, inv_inertia, pose, flags, ncontacts (CUDA tensors) and an
    optional force."""
    E = int(arrays["body_off"].numel()) - 1
    B = int(arrays["inv_mass"].numel())
    prm = sim_params(params)
    g = lambda k: _dptr(arrays.get(k))
    check(lib.vuda_sim_step_noalloc(E, B, max_bodies, g("body_off"), g("pos"), g("quat"), g("vel"), g("angvel"),
                                    g("shape_type"), g("shape_dims"), g("inv_mass"), g("inv_inertia"), g("force"),
                                    C.byref(prm), nsteps, g("pose"), g("flags"), g("ncontacts"), smem_per_env,
                                    _stream(stream)), "vuda_sim_step_noalloc")


# ---------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------
class ServeOpts(C.Structure):
    _fields_ = [("device", C.c_int32), ("hbm_budget_bytes", C.c_int64), ("max_jobs", C.c_int32),
                ("max_inflight", C.c_int32), ("max_batch_jobs", C.c_int32), ("serialized", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("req_id", C.c_uint64), ("job_id", C.c_int64), ("status", C.c_int32), ("step", C.c_int64),
                ("t_submit_ms", C.c_double), ("t_start_ms", C.c_double), ("t_done_ms", C.c_double)]


class ServeStats(C.Structure):
    _fields_ = [("jobs", C.c_int32), ("admitted", C.c_int32), ("waiting", C.c_int32), ("inflight", C.c_int32),
                ("iterations", C.c_int64), ("requests_done", C.c_int64), ("mean_batch", C.c_double),
                ("max_batch", C.c_int32), ("used_bytes", C.c_int64), ("peak_bytes", C.c_int64)]


_sig("vuda_serve_create", [C.POINTER(ServeOpts), C.POINTER(vp)])
_sig("vuda_serve_destroy", [vp])
_sig("vuda_serve_add_job", [vp, C.POINTER(Scene), C.POINTER(SimParams), C.POINTER(C.c_int64)])
_sig("vuda_serve_submit", [vp, C.c_int64, C.POINTER(C.c_uint64)])
_sig("vuda_serve_poll", [vp, C.POINTER(Result), C.c_int32, C.POINTER(C.c_int32), C.c_int32])
_sig("vuda_serve_remove_job", [vp, C.c_int64])
_sig("vuda_serve_job_env", [vp, C.c_int64, C.POINTER(vp), C.POINTER(Frame)])
_sig("vuda_serve_stats_get", [vp, C.POINTER(ServeStats)])
_sig("vuda_serve_read_frame", [vp, C.c_int64, vp, vp, vp])


class Server:
    """Continuous-batching server for step+render requests of many jobs."""

    def __init__(self, hbm_budget_bytes: int = 0, max_jobs: int = 64, max_inflight: int = 2,
                 max_batch_jobs: int = 0, serialized: bool = False, device: int = 0):
        h = vp()
        check(lib.vuda_serve_create(C.byref(ServeOpts(device, hbm_budget_bytes, max_jobs, max_inflight,
                                                      max_batch_jobs, int(serialized))), C.byref(h)),
              "vuda_serve_create")
        self.h = h
        self.scenes = {}
        self._buf = (Result * 4096)()

    def close(self):
        if getattr(self, "h", None):
            lib.vuda_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_job(self, scene, params=None) -> int:
        sc, keep = scene_struct(scene)
        jid = C.c_int64()
        check(lib.vuda_serve_add_job(self.h, C.byref(sc), C.byref(sim_params(params or scene.params)),
                                     C.byref(jid)), "vuda_serve_add_job")
        self.scenes[jid.value] = scene
        return jid.value

    def submit(self, job: int) -> int:
        r = C.c_uint64()
        check(lib.vuda_serve_submit(self.h, job, C.byref(r)), "vuda_serve_submit")
        return r.value

    def poll(self, wait_ms: int = 0, max_results: int = 4096):
        n = C.c_int32()
        st = lib.vuda_serve_poll(self.h, self._buf, min(max_results, 4096), C.byref(n), wait_ms)
        if st == ERR_TIMEOUT:       # the bounded wait ran out with nothing completed
            return []
        check(st, "vuda_serve_poll")
        return [dict(req_id=r.req_id, job=r.job_id, status=r.status, step=r.step, t_submit_ms=r.t_submit_ms,
                     t_start_ms=r.t_start_ms, t_done_ms=r.t_done_ms) for r in self._buf[:n.value]]

    def remove_job(self, job: int):
        check(lib.vuda_serve_remove_job(self.h, job), "vuda_serve_remove_job")

    def stats(self) -> dict:
        st = ServeStats()
        check(lib.vuda_serve_stats_get(self.h, C.byref(st)), "vuda_serve_stats_get")
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def job_env(self, job: int) -> Env:
        """The job's resident batch (borrowed; read it while the job is idle)."""
        e = vp()
        check(lib.vuda_serve_job_env(self.h, job, C.byref(e), None), "vuda_serve_job_env")
        return Env(self.scenes[job], _handle=e)

    def read_frame(self, job: int):
        env = self.job_env(job)
        P = env.P
        rgb = np.zeros((P, 3), np.uint8)
        dep = np.zeros(P, np.float32)
        tid = np.zeros(P, np.uint32)
        check(lib.vuda_serve_read_frame(self.h, job, _ptr(rgb), _ptr(dep), _ptr(tid)), "vuda_serve_read_frame")
        return rgb, dep, tid

    def wait_all(self, n: int, timeout_s: float = 60.0):
        """Collect n results (blocking)."""
        import time
        out = []
        t0 = time.time()
        while len(out) < n:
            out += self.poll(wait_ms=50)
            if time.time() - t0 > timeout_s:
                raise TimeoutError("serving results did not arrive")
        return out
