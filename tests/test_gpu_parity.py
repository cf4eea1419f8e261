"""GPU path (through the C ABI) against the CPU oracle on identical seeded
inputs.

Bars: coverage / triangle ids bit-exact, depth within 1e-6 relative, colour
within 1 LSB; physics state within 1e-5 relative (absolute floor 1e-5 in
units of 1 m, 1 m/s, 1) after every step of a 10-step horizon, with
identical contact counts and status flags.
"""
import dataclasses

import numpy as np
import pytest

from paper_2605_01352_b300 import scene as S

pytestmark = pytest.mark.gpu

PHYS_RTOL = 1e-5
PHYS_ATOL = 1e-5
DEPTH_RTOL = 1e-6


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_01352_b300 import build
    build.build()
    from paper_2605_01352_b300 import vuda
    return vuda


def _cmp_state(g, o, where):
    for k in ("pos", "vel", "angvel", "quat"):
        np.testing.assert_allclose(g[k], o[k], rtol=PHYS_RTOL, atol=PHYS_ATOL, err_msg="%s %s" % (where, k))


def _physics_horizon(V, orc, sc, steps=10, force=None, **env_kw):
    import torch
    env = V.Env(sc, **env_kw)
    st_o = sc.state()
    ft = None if force is None else torch.from_numpy(np.ascontiguousarray(force, np.float32)).cuda()
    for s in range(steps):
        env.sim_step(1, force=ft)
        torch.cuda.synchronize()
        g = env.get_state()
        st_o, fl_o, cc_o = orc.sim_step(sc, 1, state=st_o, force=force)
        _cmp_state(g, st_o, "step %d" % s)
        np.testing.assert_array_equal(env.contact_counts(), cc_o)
        fl_g, _ = env.status()
        np.testing.assert_array_equal(fl_g & 1, fl_o & 1)
    # the pose slot of the last step is the state's pose
    pos, quat = env.get_pose((steps - 1) & 1)
    np.testing.assert_array_equal(pos, g["pos"])
    np.testing.assert_array_equal(quat, g["quat"])
    env.close()
    return g


PATHS = ["band", "tiled"]


def _path(V, name):
    return {"band": V.RENDER_BAND, "tiled": V.RENDER_TILED}[name]


def _render_cmp(V, orc, sc, pos=None, quat=None, env=None, path="tiled"):
    import torch
    own = env is None
    if own:
        env = V.Env(sc, render_path=_path(V, path))
        assert env.info().render_path == _path(V, path)
    pos = sc.pos if pos is None else pos
    quat = sc.quat if quat is None else quat
    env.set_pose(0, pos, quat)
    fr = env.alloc_frame()
    env.render(fr, pose_slot=0)
    torch.cuda.synchronize()
    rgb = fr["rgb"].cpu().numpy()
    dep = fr["depth"].cpu().numpy()
    tid = fr["triid"].cpu().numpy().view(np.uint32)
    o_rgb, o_dep, o_tid, o_fl = orc.render(sc, pos, quat)
    np.testing.assert_array_equal(tid, o_tid)
    np.testing.assert_allclose(dep, o_dep, rtol=DEPTH_RTOL, atol=0)
    assert np.abs(rgb.astype(int) - o_rgb.astype(int)).max() <= 1
    fl, _ = env.status()
    np.testing.assert_array_equal(fl & 6, o_fl & 6)
    if own:
        env.close()
    return tid


def test_physics_cfg1_horizon(V, orc):
    _physics_horizon(V, orc, S.cfg1())


def test_physics_cfg2_subset_horizon(V, orc):
    """Spheres and randomly oriented boxes (box-box, sphere-box contacts)."""
    sc = S.cfg2(24)
    st, _, _ = orc.sim_step(sc, 60)   # let them land and pile up first
    sc = dataclasses.replace(sc, **{k: st[k] for k in ("pos", "quat", "vel", "angvel")})
    _physics_horizon(V, orc, sc, steps=10)


@pytest.mark.parametrize("persistent", [False, True])
def test_physics_with_forces(V, orc, persistent):
    sc = S.cfg1(4)
    rng = np.random.default_rng(3)
    f = rng.normal(0, 0.5, (3, sc.num_bodies)).astype(np.float32)
    _physics_horizon(V, orc, sc, steps=5, force=f, persistent=persistent)


def test_physics_edge_contacts_and_gyroscopic_term(V, orc):
    """Box-box edge-edge contacts (crossed beams touching edge to edge, one
    in penetration) and the gyroscopic term (boxes spinning near their
    intermediate axis, in flight) through a 10-step horizon against the
    oracle, with identical contact counts."""
    from scipy.spatial.transform import Rotation

    def wxyz(r):
        x, y, z, w = r.as_quat()
        return (w, x, y, z)
    ra, rb = Rotation.from_euler("x", 45, degrees=True), Rotation.from_euler("zy", [20, 45], degrees=True)
    bodies = []
    for k, gap in enumerate((0.004, -0.002, 0.01)):
        x0 = 0.8 * k - 0.8
        zA = 0.05 + 0.03 * np.sqrt(2)
        bodies.append(dict(type="box", h=(0.3, 0.03, 0.03), pos=(x0, 0.0, zA), quat=wxyz(ra)))
        bodies.append(dict(type="box", h=(0.02, 0.3, 0.02), pos=(x0, 0.0, zA + 0.03 * np.sqrt(2) + gap + 0.02 * np.sqrt(2)),
                           quat=wxyz(rb)))
    for k in range(3):
        bodies.append(dict(type="box", h=(0.02, 0.05, 0.1), pos=(0.5 * k - 0.5, 1.5, 1.5),
                           angvel=(0.05, 12.0 - k, -0.05), quat=wxyz(Rotation.from_euler("xyz", [10 * k, 5, 0],
                                                                                            degrees=True))))
    p = dataclasses.replace(S.SimParams(), gyroscopic=1, edge_contacts=1)
    sc = S.custom(bodies, envs=3, params=p)
    c = orc.contacts(sc, 0)
    assert sum(1 for a, b in zip(c["a"], c["b"]) if b >= 0) >= 3    # the crossing edges
    _physics_horizon(V, orc, sc, steps=10)


def test_physics_piles_with_edge_contacts_and_gyroscopic_term(V, orc):
    """Settled piles of spheres and randomly oriented boxes with both
    options on: box pairs in crowded pair rounds (more passing pairs than
    the edge-test slots) and spinning boxes in contact."""
    sc = S.cfg2(24)
    sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, gyroscopic=1, edge_contacts=1))
    st, _, _ = orc.sim_step(sc, 60)
    sc = dataclasses.replace(sc, **{k: st[k] for k in ("pos", "quat", "vel", "angvel")})
    _physics_horizon(V, orc, sc, steps=10)


def test_physics_contact_overflow_matches(V, orc):
    """A capacity of 1 contact per body truncates identically on both sides."""
    sc = S.cfg2(8)
    st, _, _ = orc.sim_step(sc, 80)
    p = dataclasses.replace(sc.params, max_contacts_per_body=1)
    sc = dataclasses.replace(sc, params=p, **{k: st[k] for k in ("pos", "quat", "vel", "angvel")})
    _, fl, _ = orc.sim_step(sc, 1)
    assert fl.any()
    _physics_horizon(V, orc, sc, steps=3)


@pytest.mark.parametrize("persistent", [False, True])
def test_physics_uneven_and_empty_envs(V, orc, persistent):
    """Ragged batch: 0, 1, 3, 40, 70 and 130 bodies; more contacts than the
    shared memory holds spill to global memory.  Persistent: one work list
    per size class (up to 32, up to 64 bodies on 128-thread CTAs, more on
    512-thread CTAs)."""
    nb = np.array([0, 1, 3, 40, 70, 130], np.int32)
    sc = S.generate(6, nb, 1234, kinds="mixed", res=64, substeps=4)
    st, _, _ = orc.sim_step(sc, 40)
    sc = dataclasses.replace(sc, **{k: st[k] for k in ("pos", "quat", "vel", "angvel")})
    _physics_horizon(V, orc, sc, steps=4, persistent=persistent)


def test_physics_contact_spill_to_global(V, orc):
    """A shared-memory budget too small for any contact record: every contact
    lives in the global spill area, with the same results."""
    sc = S.cfg2(8)
    st, _, _ = orc.sim_step(sc, 80)
    sc = dataclasses.replace(sc, **{k: st[k] for k in ("pos", "quat", "vel", "angvel")})
    _physics_horizon(V, orc, sc, steps=3, phys_smem_bytes=1024)


@pytest.mark.parametrize("path", PATHS)
def test_render_cfg1(V, orc, path):
    sc = S.cfg1()
    st, _, _ = orc.sim_step(sc, 50)
    _render_cmp(V, orc, sc, st["pos"], st["quat"], path=path)


@pytest.mark.parametrize("path", PATHS)
def test_render_cfg2_subset(V, orc, path):
    sc = S.cfg2(16)
    st, _, _ = orc.sim_step(sc, 50)
    _render_cmp(V, orc, sc, st["pos"], st["quat"], path=path)


def test_render_mixed_resolutions_and_bands(V, orc):
    """Cameras of 64, 128 and 256 pixels in one batch, and non-default band
    heights (ragged last band)."""
    sc = S.generate(3, np.array([6, 10, 3]), 77, kinds="mixed", res=np.array([64, 256, 128]), substeps=4)
    st, _, _ = orc.sim_step(sc, 20)
    for rows in (0, 7, 13):
        env = V.Env(sc, band_rows=rows, render_path=V.RENDER_BAND)
        _render_cmp(V, orc, sc, st["pos"], st["quat"], env=env)
        env.close()
    _render_cmp(V, orc, sc, st["pos"], st["quat"], path="tiled")


@pytest.mark.parametrize("path", PATHS)
def test_render_ragged_tiles(V, orc, path):
    """Camera sizes that are not multiples of the 16-pixel tile or of the
    8-pixel runs (partial tiles, unaligned first pixels of later cameras),
    bodies close to the camera (large triangles) and far (small ones)."""
    sc = S.generate(4, np.array([7, 12, 5, 9]), 303, kinds="mixed", res=np.array([40, 71, 9, 100]), substeps=4)
    st, _, _ = orc.sim_step(sc, 30)
    _render_cmp(V, orc, sc, st["pos"], st["quat"], path=path)


TILINGS = [(8, 1), (8, 9), (16, 1), (16, 4), (16, 64), (32, 2), (32, 9)]


@pytest.mark.parametrize("tile,nlim", TILINGS)
def test_render_tilings_match_oracle(V, orc, tile, nlim):
    """Every tile size of the tiled path (8 x 8: two pixels a lane; 32 x 32:
    four 32 x 8 strips) with small and large bin limits (most triangles on
    the wide list, or none) gives the oracle's frames, on cameras that are
    not multiples of any tile size (partial tiles and strips, odd widths
    that leave runs unaligned)."""
    sc = S.generate(4, np.array([7, 12, 5, 9]), 303, kinds="mixed", res=np.array([40, 71, 9, 100]), substeps=4)
    st, _, _ = orc.sim_step(sc, 30)
    env = V.Env(sc, render_path=V.RENDER_TILED, tile_size=tile, tile_bin_limit=nlim)
    i = env.info()
    assert (i.render_path, i.tile_size, i.tile_bin_limit) == (V.RENDER_TILED, tile, nlim)
    _render_cmp(V, orc, sc, st["pos"], st["quat"], env=env)
    env.close()


def test_set_tiling_switches_without_changing_frames(V):
    """vuda_set_tiling moves one batch through every tile size and bin limit
    the autotuner tries; the frames stay bit-identical, and invalid choices
    are refused with the batch keeping its parameters."""
    import torch
    sc = S.cfg2(48)
    env = V.Env(sc, render_path=V.RENDER_TILED)
    assert (env.info().tile_size, env.info().tile_bin_limit) == (16, 9)
    bytes0 = env.info().device_bytes
    ring = [env.alloc_frame(), env.alloc_frame()]
    env.sim_step(40)
    ref = None
    for tile in (16, 8, 32):
        for nlim in (9, 4, 16):
            env.set_tiling(tile, nlim)
            assert (env.info().tile_size, env.info().tile_bin_limit) == (tile, nlim)
            for k in ring[0]:
                ring[0][k].zero_()
            env.render(ring[0], pose_slot=-1)
            torch.cuda.synchronize()
            got = {k: v.cpu().numpy().copy() for k, v in ring[0].items()}
            if ref is None:
                ref = got
            for k in ref:
                np.testing.assert_array_equal(got[k], ref[k], err_msg="%s tile %d limit %d" % (k, tile, nlim))
    for bad in ((12, 9), (16, 0), (16, 65)):
        with pytest.raises(V.VudaError):
            env.set_tiling(*bad)
        assert (env.info().tile_size, env.info().tile_bin_limit) == (32, 16)
    # the replaced tile lists were freed: back at the first parameters, the batch holds what it held
    env.set_tiling(16, 9)
    assert env.info().device_bytes == bytes0
    env.close()
    band = V.Env(S.cfg2(4), render_path=V.RENDER_BAND)
    with pytest.raises(V.VudaError):
        band.set_tiling(16, 9)
    assert band.info().tile_size == 0
    band.close()
    # 640 x 480 is 4800 tiles of 8 x 8, over the per-camera tile table
    big = S.generate(1, np.array([4]), 5, kinds="mixed", res=np.array([640]), height=np.array([480]), substeps=4)
    with pytest.raises(V.VudaError):
        V.Env(big, render_path=V.RENDER_TILED, tile_size=8)
    e = V.Env(big, render_path=V.RENDER_TILED, tile_size=32)
    with pytest.raises(V.VudaError):
        e.set_tiling(8, 9)
    assert e.info().tile_size == 32
    e.close()


@pytest.mark.parametrize("path", PATHS)
def test_render_non_square_cameras(V, orc, path):
    """A 640 x 480 data-generation camera (1200 tiles) beside non-square
    cameras narrower and taller than wide; the field of view is vertical."""
    sc = S.generate(3, np.array([10, 6, 8]), 505, kinds="mixed", res=np.array([640, 96, 33]),
                    height=np.array([480, 40, 70]), substeps=4)
    assert list(sc.cam_w) == [640, 96, 33] and list(sc.cam_h) == [480, 40, 70]
    st, _, _ = orc.sim_step(sc, 30)
    _render_cmp(V, orc, sc, st["pos"], st["quat"], path=path)


@pytest.mark.parametrize("path", PATHS)
def test_render_degenerate_camera_sizes(V, orc, path):
    """Cameras of one pixel, one row and one column, and a 2 x 3 camera:
    tiles and runs that are almost empty (most lanes own no pixel)."""
    sc = S.generate(4, np.array([5, 6, 4, 7]), 909, kinds="mixed", res=np.array([1, 37, 1, 2]),
                    height=np.array([1, 1, 29, 3]), substeps=4)
    st, _, _ = orc.sim_step(sc, 20)
    _render_cmp(V, orc, sc, st["pos"], st["quat"], path=path)


@pytest.mark.parametrize("tile", [8, 32])
def test_render_degenerate_camera_sizes_other_tiles(V, orc, tile):
    sc = S.generate(4, np.array([5, 6, 4, 7]), 909, kinds="mixed", res=np.array([1, 37, 1, 2]),
                    height=np.array([1, 1, 29, 3]), substeps=4)
    st, _, _ = orc.sim_step(sc, 20)
    env = V.Env(sc, render_path=V.RENDER_TILED, tile_size=tile)
    _render_cmp(V, orc, sc, st["pos"], st["quat"], env=env)
    env.close()


def _near_scenes():
    """Scenes with triangles crossing the near plane: a large box face
    2^-9 m below the eye (clipped to a triangle and to a quadrilateral), and
    spheres and boxes crowding the eye of a 96 x 72 camera (some wholly
    behind it, others cut by the plane at every angle)."""
    h = 2.0 ** -9
    face = S.custom([dict(type="box", h=(1.0, 1.0, 0.125), pos=(0.0, 0.5, 0.875))], res=128,
                    cams=[dict(eye=(0.0, 0.0, 1.0 + h), target=(0.0, 1.0, 1.0 + h), fov=60.0)])
    eye, tgt = np.array([0.0, -2.5, 1.5]), np.array([0.0, 0.0, 0.4])
    f = (tgt - eye) / np.linalg.norm(tgt - eye)
    r = np.cross(f, [0.0, 0.0, 1.0])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    out = [face]
    for seed in (0, 4):     # 22 and 62 triangles cross the plane
        rng = np.random.default_rng(seed)
        bodies = []
        for i in range(24):
            p = eye + f * rng.uniform(-0.1, 0.5) + r * rng.uniform(-0.15, 0.15) + u * rng.uniform(-0.15, 0.15)
            q = rng.normal(size=4)
            q /= np.linalg.norm(q)
            if i % 2:
                bodies.append(dict(type="box", h=tuple(rng.uniform(0.02, 0.08, 3)), pos=tuple(p), quat=tuple(q)))
            else:
                bodies.append(dict(type="sphere", r=float(rng.uniform(0.02, 0.08)), pos=tuple(p)))
        crowd = S.custom(bodies, res=96)
        crowd.cam_h[:] = 72
        out.append(crowd)
    return out


@pytest.mark.parametrize("path", PATHS)
def test_render_near_plane_clipping(V, orc, path):
    """Triangles crossing the near plane are clipped (Sutherland-Hodgman,
    one or two fan triangles with the original id) identically on both
    paths and in the oracle: ids bit-exact, depth 1e-6, colour 1 LSB."""
    for sc in _near_scenes():
        tid = _render_cmp(V, orc, sc, path=path)
        assert ((tid != 0xFFFFFFFF) & (tid >= 2)).any()


@pytest.mark.parametrize("tile,nlim", [(8, 1), (16, 9), (32, 64)])
def test_render_near_plane_clipping_tilings(V, orc, tile, nlim):
    for sc in _near_scenes():
        env = V.Env(sc, render_path=V.RENDER_TILED, tile_size=tile, tile_bin_limit=nlim)
        _render_cmp(V, orc, sc, env=env)
        assert env.status()[0][0] & V.FLAG_CLIP_CAPACITY == 0
        env.close()


def test_render_paths_identical_frames_full_size(V, orc):
    """The band and tiled paths give identical frames, bit for bit, on the
    1024-environment batch of 128 x 128 cameras (settled piles), and
    sampled environments' frames match the oracle's render of the pose
    slot they were rendered from."""
    import torch
    sc = S.cfg2()
    out = []
    for path in (V.RENDER_BAND, V.RENDER_TILED):
        env = V.Env(sc, render_path=path)
        assert env.info().render_path == path
        ring = [env.alloc_frame(), env.alloc_frame()]
        env.pipeline_run(40, ring)
        torch.cuda.synchronize()
        out.append({k: v.cpu().numpy() for k, v in ring[1].items()})
        out[-1]["flags"] = env.status()[0]
        _frames_of_gpu_poses(orc, sc, env, ring[1], 1, (0, 333, 1023))
        env.close()
    for k in out[0]:
        np.testing.assert_array_equal(out[0][k], out[1][k], err_msg=k)


def test_raster_screen_tris_matches_oracle(V, orc):
    import torch
    rng = np.random.default_rng(9)
    for W, H, n in ((16, 16, 40), (64, 48, 300), (200, 37, 800)):
        xy = rng.integers(-3 * 256, (max(W, H) + 3) * 256, (n, 3, 2)).astype(np.int32)
        xy[: n // 3] = (xy[: n // 3] // 128) * 128   # many ties on pixel centres
        z = rng.uniform(0.2, 5.0, (n, 3)).astype(np.float32)
        tid, dep, cnt = V.raster_screen_tris(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda(), W, H,
                                             count=True)
        o_tid, o_dep, o_cnt = orc.raster_screen_tris(xy, z, W, H, count=True)
        np.testing.assert_array_equal(tid.cpu().numpy().view(np.uint32), o_tid)
        np.testing.assert_allclose(dep.cpu().numpy(), o_dep, rtol=DEPTH_RTOL, atol=0)
        np.testing.assert_array_equal(cnt.cpu().numpy(), o_cnt)


def test_raster_screen_tris_guard_band_extremes(V, orc):
    """Triangles with vertices anywhere in the guard band (|x|, |y| up to
    2^22 in 1/256 px) give edge values up to about 2^46 at the pixel centres;
    their conversions to float must still be the correctly rounded ones.
    Vertices beyond the band discard the triangle on both sides."""
    import torch
    rng = np.random.default_rng(21)
    lim = 1 << 22
    for W, H, n in ((64, 64, 120), (130, 70, 200)):
        xy = rng.integers(-lim, lim + 1, (n, 3, 2)).astype(np.int64)
        xy[::7] = rng.choice([-lim, lim], (len(xy[::7]), 3, 2))          # on the band's edge
        xy[3::11, 1, 0] = lim + rng.integers(1, 1000, len(xy[3::11]))     # beyond it: discarded
        xy = xy.astype(np.int32)
        z = rng.uniform(0.05, 50.0, (n, 3)).astype(np.float32)
        tid, dep, cnt = V.raster_screen_tris(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda(), W, H,
                                             count=True)
        o_tid, o_dep, o_cnt = orc.raster_screen_tris(xy, z, W, H, count=True)
        assert (o_tid != 0xFFFFFFFF).mean() > 0.5          # the image is mostly covered
        np.testing.assert_array_equal(tid.cpu().numpy().view(np.uint32), o_tid)
        np.testing.assert_array_equal(dep.cpu().numpy(), o_dep)
        np.testing.assert_array_equal(cnt.cpu().numpy(), o_cnt)


def test_raster_screen_tris_empty(V):
    import torch
    tid, dep, cnt = V.raster_screen_tris(torch.zeros((0, 3, 2), dtype=torch.int32, device="cuda"),
                                         torch.zeros((0, 3), device="cuda"), 8, 8, count=True)
    assert (tid.cpu().numpy().view(np.uint32) == 0xFFFFFFFF).all()
    assert (dep.cpu().numpy() == 0).all() and (cnt.cpu().numpy() == 0).all()


def _run_loop(V, sc, steps, mode, **co):
    import torch
    env = V.Env(sc)
    ring = [env.alloc_frame(), env.alloc_frame()]
    if mode:
        env.coschedule(mode, **co)
    env.pipeline_run(steps, ring)
    torch.cuda.synchronize()
    st = env.get_state()
    out = [{k: v.cpu().numpy().copy() for k, v in f.items()} for f in ring]
    env.close()
    return st, out


@pytest.mark.parametrize("mode", ["streams", "green", "shared", "shared-1-1"])
def test_coscheduled_equals_serialized(V, mode):
    """Pipelined sim(t+1) || render(t) on two streams (shared SMs, disjoint
    green-context partitions, or per-SM CTA quotas with both phases resident
    on every SM) gives the same state and frames as the serialized loop, bit
    for bit."""
    sc = S.cfg2(64)
    m = {"streams": V.COSCHED_STREAMS, "green": V.COSCHED_GREEN}.get(mode, V.COSCHED_SHARED)
    co = dict(sim_ctas_per_sm=1, render_ctas_per_sm=1) if mode == "shared-1-1" else {}
    st0, fr0 = _run_loop(V, sc, 7, 0)
    st1, fr1 = _run_loop(V, sc, 7, m, **co)
    for k in st0:
        np.testing.assert_array_equal(st0[k], st1[k])
    for a, b in zip(fr0, fr1):
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])


def test_shared_quotas_reported_and_checked(V):
    """Per-SM quotas: the default pair fits one SM and is reported; a pair
    that cannot fit one SM together is refused before anything launches;
    reset returns the batch to serialized launches."""
    sc = S.cfg2(16)
    env = V.Env(sc)
    info = env.coschedule(V.COSCHED_SHARED)
    assert info["mode"] == V.COSCHED_SHARED
    assert info["sim_ctas_per_sm"] >= 1 and info["render_ctas_per_sm"] >= 1
    with pytest.raises(V.VudaError) as ex:
        env.coschedule(V.COSCHED_SHARED, sim_ctas_per_sm=32, render_ctas_per_sm=32)
    assert ex.value.status == V.ERR_INVALID
    with pytest.raises(V.VudaError):
        env.coschedule(V.COSCHED_SHARED, sim_ctas_per_sm=-1)
    env.coschedule_reset()
    env.close()


def test_pipeline_frames_match_oracle(V, orc):
    """The co-scheduled loop's final state matches the oracle, and its last
    two frames are the oracle's renders of the two pose slots they were
    rendered from (steps n-1 and n)."""
    import torch
    sc = S.cfg1(8)
    n = 6
    env = V.Env(sc)
    ring = [env.alloc_frame(), env.alloc_frame()]
    env.coschedule(V.COSCHED_STREAMS)
    env.pipeline_run(n, ring)
    torch.cuda.synchronize()
    s_last, _, _ = orc.sim_step(sc, n)
    _cmp_state(env.get_state(), s_last, "final")
    envs = range(sc.num_envs)
    for k in (n - 1, n - 2):
        _frames_of_gpu_poses(orc, sc, env, ring[k & 1], k & 1, envs)
    env.close()


@pytest.mark.parametrize("mode", ["serialized", "streams"])
def test_host_loop_forces_in_frames_out_match_oracle(V, orc, mode):
    """vuda_pipeline_run_host, the end-to-end loop: a different force per step
    is copied in from pinned host memory before each sim step, and the RGB
    and depth of every step are copied out into the pinned host ring (slot
    t & 1).  The last two frames in host memory and the final state match
    the oracle stepped with the same forces (an odd step count, so both ring
    slots and the wrap-around are checked)."""
    import torch
    sc = S.cfg2(8)
    st, _, _ = orc.sim_step(sc, 40)
    sc = dataclasses.replace(sc, **{k: st[k] for k in ("pos", "quat", "vel", "angvel")})
    n = 5
    f = np.random.default_rng(11).normal(0, 0.3, (n, 3, sc.num_bodies)).astype(np.float32)
    env = V.Env(sc)
    if mode == "streams":
        env.coschedule(V.COSCHED_STREAMS)
    ring = [env.alloc_frame(), env.alloc_frame()]
    hf = torch.from_numpy(f).pin_memory()
    hr = torch.zeros((2, env.P, 3), dtype=torch.uint8).pin_memory()
    hd = torch.zeros((2, env.P), dtype=torch.float32).pin_memory()
    env.pipeline_run_host(n, ring, hr, hd, h_force=hf, force_per_step=True)
    g = env.get_state()
    st_o = sc.state()
    for t in range(n):
        st_o, _, _ = orc.sim_step(sc, 1, state=st_o, force=f[t])
    _cmp_state(g, st_o, "final")
    for t in (n - 2, n - 1):
        pos, quat = env.get_pose(t & 1)     # the pose slot step t was rendered from
        o_rgb, o_dep, _, _ = orc.render(sc, pos, quat)
        np.testing.assert_allclose(hd[t & 1].numpy(), o_dep, rtol=DEPTH_RTOL, atol=0, err_msg="step %d" % t)
        assert np.abs(hr[t & 1].numpy().astype(int) - o_rgb.astype(int)).max() <= 1
    env.close()


def _frames_of_gpu_poses(orc, sc, env, frame, slot, envs):
    """Render parity on the GPU's own poses: the pose slot the GPU rendered
    from is read back and rendered by the oracle, environment by
    environment; triangle ids bit-exact, depth 1e-6, colour 1 LSB."""
    pos, quat = env.get_pose(slot)
    pix = env.cam_pix_off
    for e in envs:
        sub = sc.subset([e])
        b0, b1 = sc.body_off[e], sc.body_off[e + 1]
        o_rgb, o_dep, o_tid, _ = orc.render(sub, pos[:, b0:b1], quat[:, b0:b1])
        c0, c1 = sc.cam_off[e], sc.cam_off[e + 1]
        sl = slice(pix[c0], pix[c1])
        np.testing.assert_array_equal(frame["triid"][sl].cpu().numpy().view(np.uint32), o_tid,
                                      err_msg="env %d" % e)
        np.testing.assert_allclose(frame["depth"][sl].cpu().numpy(), o_dep, rtol=DEPTH_RTOL, atol=0,
                                   err_msg="env %d" % e)
        assert np.abs(frame["rgb"][sl].cpu().numpy().astype(int) - o_rgb.astype(int)).max() <= 1, e


def _sampled_physics(orc, sc, g, steps, envs, start=None):
    """Sampled environments of a batch stepped `steps` times from `start`
    (default: the scene's initial state) match the oracle run on each of
    them alone (environments are independent), within the physics
    tolerance."""
    for e in envs:
        sub = sc.subset([e])
        b0, b1 = sc.body_off[e], sc.body_off[e + 1]
        st0 = None if start is None else {k: start[k][:, b0:b1] for k in ("pos", "quat", "vel", "angvel")}
        so, _, _ = orc.sim_step(sub, steps, state=st0)
        for k in ("pos", "vel", "quat", "angvel"):
            np.testing.assert_allclose(g[k][:, b0:b1], so[k], rtol=PHYS_RTOL, atol=PHYS_ATOL,
                                       err_msg="env %d %s" % (e, k))


CFG2_SAMPLE = (0, 1, 511, 777, 1023)


@pytest.mark.parametrize("launch", ["green", "bench"])
def test_full_size_cfg2_sampled(V, orc, launch):
    """1024 envs x 32 bodies at 128x128: sampled environments' states match
    the oracle run on those environments alone, and their frames match the
    oracle's render of the pose slot the GPU rendered from.  Launch
    configurations: the paper's disjoint partitions (green contexts, 3
    steps), and the benchmark's headline one (two streams sharing all SMs,
    sim stream first, 8 pipelined steps replayed from a CUDA graph)."""
    import torch
    sc = S.cfg2()
    env = V.Env(sc)
    ring = [env.alloc_frame(), env.alloc_frame()]
    if launch == "green":
        env.coschedule(V.COSCHED_GREEN)
        steps = 3
    else:
        env.coschedule(V.COSCHED_STREAMS, priority=V.PRIORITY_SIM)
        steps = 8
        env.pipeline_capture(steps, ring)
    env.pipeline_run(steps, ring)
    torch.cuda.synchronize()
    g = env.get_state()
    assert env.status()[1] == 0
    _sampled_physics(orc, sc, g, steps, CFG2_SAMPLE)
    _frames_of_gpu_poses(orc, sc, env, ring[(steps - 1) & 1], (steps - 1) & 1, CFG2_SAMPLE)
    env.close()


@pytest.mark.parametrize("mode", ["streams-graph", "green"])
def test_full_size_cfg2_settled_piles(V, orc, mode):
    """The regime the benchmark times: the 1024-environment batch after 120
    settling steps (piles in contact, about 2.7 contacts per body; the most
    crowded environments spill contacts to global memory), then 8 pipelined
    steps in a co-scheduled launch configuration.  Sampled environments, stepped by the oracle from
    the GPU's settled state, match within the physics tolerance; their
    frames match the oracle's render of the GPU's last pose slot."""
    import torch
    sc = S.cfg2()
    env = V.Env(sc)
    ring = [env.alloc_frame(), env.alloc_frame()]
    env.pipeline_run(120, ring)
    torch.cuda.synchronize()
    settled = env.get_state()
    cc = env.contact_counts()
    assert cc.mean() > 2.0 * 32, cc.mean()          # settled piles, contact-rich
    if mode == "green":
        env.coschedule(V.COSCHED_GREEN)
    else:
        env.coschedule(V.COSCHED_STREAMS, priority=V.PRIORITY_SIM)
        env.pipeline_capture(8, ring)
    env.pipeline_run(8, ring)
    torch.cuda.synchronize()
    g = env.get_state()
    picks = CFG2_SAMPLE + (int(np.argmax(cc)),)
    _sampled_physics(orc, sc, g, 8, picks, start=settled)
    _frames_of_gpu_poses(orc, sc, env, ring[1], 1, picks)
    env.close()


def _sampled_env_check(orc, sc, env, ring, steps, envs, frame_slot):
    """Sampled environments of a batch stepped `steps` times match the oracle
    run on each of them alone (state), and every camera of the environment
    in frame ring[frame_slot] matches the oracle's render of the GPU's pose
    slot of that frame."""
    _sampled_physics(orc, sc, env.get_state(), steps, envs)
    _frames_of_gpu_poses(orc, sc, env, ring[frame_slot], frame_slot, envs)


def test_full_size_cfg3_graph_sampled(V, orc):
    """The RL-rollout shape at full size: 4096 envs x 64 convex hulls of
    500-2000 triangles, two 128 x 128 cameras each (about 330 M triangles per
    camera-step), two pipelined steps replayed from a CUDA graph on
    co-scheduled streams; sampled environments match the oracle."""
    import torch
    sc = S.cfg3()
    env = V.Env(sc)
    ring = [env.alloc_frame(), env.alloc_frame()]
    env.coschedule(V.COSCHED_STREAMS)
    env.pipeline_capture(2, ring)
    env.pipeline_run(2, ring)
    torch.cuda.synchronize()
    assert env.info().steps_enqueued == 2 and env.C == 8192
    _sampled_env_check(orc, sc, env, ring, 2, (0, 1, 2047, 4095), 1)
    env.close()


def test_full_size_cfg4_persistent_sampled(V, orc):
    """The uneven batch at full size: 2048 envs with 4-256 bodies and 64,
    128 or 256 pixel cameras through one persistent launch per phase;
    sampled environments (including the largest) match the oracle."""
    import torch
    sc = S.cfg4()
    env = V.Env(sc, persistent=True)
    ring = [env.alloc_frame(), env.alloc_frame()]
    env.pipeline_run(3, ring)
    torch.cuda.synchronize()
    sizes = np.diff(sc.body_off)
    picks = (0, 1023, 2047, int(np.argmax(sizes)), int(np.argmin(sizes)))
    _sampled_env_check(orc, sc, env, ring, 3, picks, 0)
    env.close()


def test_persistent_uneven_batch_matches(V, orc):
    """Uneven batch (body counts log-uniform in [4, 256], cameras of 64, 128
    and 256 pixels): the persistent work-list launches (largest items first,
    pulled from an atomic counter) give the same state and frames as one CTA
    per item, and sampled environments match the oracle."""
    import torch
    sc = S.cfg4(40)
    out = []
    for persistent in (False, True):
        env = V.Env(sc, persistent=persistent)
        ring = [env.alloc_frame(), env.alloc_frame()]
        env.pipeline_run(3, ring)
        torch.cuda.synchronize()
        out.append((env.get_state(), {k: v.cpu().numpy().copy() for k, v in ring[0].items()}, env.status()[0]))
        pose1 = env.get_pose(0)
        env.close()
    (s0, f0, fl0), (s1, f1, fl1) = out
    for k in s0:
        np.testing.assert_array_equal(s0[k], s1[k])
    for k in f0:
        np.testing.assert_array_equal(f0[k], f1[k])
    np.testing.assert_array_equal(fl0, fl1)
    pix = sc.cam_pix_off()
    for e in (0, 7, 21, 39):
        sub = sc.subset([e])
        so, _, _ = orc.sim_step(sub, 3)
        b0, b1 = sc.body_off[e], sc.body_off[e + 1]
        for k in ("pos", "vel", "quat", "angvel"):
            np.testing.assert_allclose(s1[k][:, b0:b1], so[k], rtol=PHYS_RTOL, atol=PHYS_ATOL)
    # frame 0 of the ring holds step 2 (the third step), rendered from pose
    # slot 0: the oracle renders that pose slot of the persistent run
    o_rgb, o_dep, o_tid, _ = orc.render(sc, *pose1)
    np.testing.assert_array_equal(f1["triid"].view(np.uint32), o_tid)
    np.testing.assert_allclose(f1["depth"], o_dep, rtol=DEPTH_RTOL)
    assert np.abs(f1["rgb"].astype(int) - o_rgb.astype(int)).max() <= 1


@pytest.mark.parametrize("mode", ["single", "streams", "green", "shared"])
def test_graph_replay_equals_launches(V, mode):
    """A captured CUDA graph of pipelined steps replays to the same state and
    frames as launching the steps one by one."""
    import torch
    sc = S.cfg2(32)
    m = {"single": 0, "streams": V.COSCHED_STREAMS, "green": V.COSCHED_GREEN, "shared": V.COSCHED_SHARED}[mode]
    out = []
    for use_graph in (False, True):
        env = V.Env(sc)
        ring = [env.alloc_frame(), env.alloc_frame()]
        stream = torch.cuda.Stream()
        if m:
            env.coschedule(m)
        if use_graph:
            try:
                env.pipeline_capture(4, ring, stream=stream)
            except V.VudaError as ex:
                assert mode == "green" and ex.status == V.ERR_UNSUPPORTED, ex
                pytest.skip("the driver refuses capture across green contexts: %s" % ex)
        env.pipeline_run(8, ring, stream=stream)
        torch.cuda.synchronize()
        assert env.info().steps_enqueued == 8
        out.append((env.get_state(), [{k: v.cpu().numpy().copy() for k, v in f.items()} for f in ring]))
        env.close()
    (s0, f0), (s1, f1) = out
    for k in s0:
        np.testing.assert_array_equal(s0[k], s1[k])
    for a, b in zip(f0, f1):
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])


def test_autotune_keeps_results_and_caches(V):
    """The autotuner leaves the batch's state untouched and its choice gives
    the same results as the default configuration; a second batch of the
    same shape reuses the cached choice."""
    import torch
    sc = S.cfg2(64)
    ref = V.Env(sc)
    ring_r = [ref.alloc_frame(), ref.alloc_frame()]
    ref.pipeline_run(4, ring_r)
    torch.cuda.synchronize()
    s_ref = ref.get_state()
    f_ref = ring_r[1]["triid"].cpu().numpy().copy()
    ref.close()
    env = V.Env(sc)
    ring = [env.alloc_frame(), env.alloc_frame()]
    res = env.autotune(ring, steps=3, use_cache=True)
    assert res["trials"] > 0
    assert env.info().render_path == V.RENDER_TILED
    assert res["tile_size"] in (8, 16, 32) and res["tile_bin_limit"] in (4, 9, 16)
    assert (env.info().tile_size, env.info().tile_bin_limit) == (res["tile_size"], res["tile_bin_limit"])
    assert res["cosched_mode"] in (0, V.COSCHED_STREAMS, V.COSCHED_GREEN, V.COSCHED_SHARED)
    if res["cosched_mode"] == V.COSCHED_SHARED:
        assert res["sim_ctas_per_sm"] >= 1 and res["render_ctas_per_sm"] >= 1
    assert env.info().steps_enqueued == 0
    env.pipeline_run(4, ring)
    torch.cuda.synchronize()
    s = env.get_state()
    for k in s:
        np.testing.assert_array_equal(s[k], s_ref[k])
    np.testing.assert_array_equal(ring[1]["triid"].cpu().numpy(), f_ref)
    env.close()
    env2 = V.Env(sc)
    ring2 = [env2.alloc_frame(), env2.alloc_frame()]
    res2 = env2.autotune(ring2, use_cache=True)
    assert res2["from_cache"] == 1 and res2["trials"] == 0
    assert (res2["tile_size"], res2["tile_bin_limit"], res2["cosched_mode"]) == \
        (res["tile_size"], res["tile_bin_limit"], res["cosched_mode"])
    assert (env2.info().tile_size, env2.info().tile_bin_limit) == (res["tile_size"], res["tile_bin_limit"])
    env2.close()
    # on the band path the raster parameter is the band height
    env3 = V.Env(S.cfg2(16), render_path=V.RENDER_BAND)
    ring3 = [env3.alloc_frame(), env3.alloc_frame()]
    res3 = env3.autotune(ring3, steps=2, use_cache=False)
    assert res3["band_rows"] in (16, 32, 64, 128) and res3["tile_size"] == 0
    # a second tuning pass (the persistent work lists now exist and are
    # rebuilt for every band height tried) frees the work items it replaces:
    # the batch ends up holding one set of them, which at 16 cameras of 128
    # rows is at most 16 x 8 bands x (4 + 4 + 2 x 16) bytes
    bytes3 = env3.info().device_bytes
    env3.autotune(ring3, steps=2, use_cache=False)
    grown = env3.info().device_bytes - bytes3
    assert abs(grown) <= 16 * 8 * (4 + 4 + 2 * 16), grown
    env3.close()


@pytest.mark.parametrize("path", PATHS)
def test_hull_meshes_two_cameras(V, orc, path):
    """Convex-hull bodies (500-2000 triangles each, sphere proxies in the
    physics) seen by two cameras per environment: physics and both cameras'
    frames match the oracle."""
    import torch
    sc = S.generate(3, 64, S.config_seed(3), kinds="hulls", res=128, cams_per_env=2, substeps=8,
                    n_hull_meshes=8)
    env = V.Env(sc, render_path=_path(V, path))
    ring = [env.alloc_frame(), env.alloc_frame()]
    env.pipeline_run(2, ring)
    torch.cuda.synchronize()
    g = env.get_state()
    so, _, _ = orc.sim_step(sc, 2)
    for k in ("pos", "vel", "quat", "angvel"):
        np.testing.assert_allclose(g[k], so[k], rtol=PHYS_RTOL, atol=PHYS_ATOL)
    _frames_of_gpu_poses(orc, sc, env, ring[1], 1, range(sc.num_envs))
    assert env.C == 6 and env.T > 3 * 64 * 500
    env.close()


@pytest.mark.parametrize("option", ["gyroscopic_edges", "hull_contacts"])
def test_full_size_physics_options_settled(V, orc, option):
    """The physics options at the size and in the regime the benchmark times
    them: 1024 environments of 32 bodies, settled for 120 steps, then 4
    plain steps -- the benchmark batch with the gyroscopic term and box-box
    edge contacts, and the batch of spheres, boxes and hulls of 8-48 faces
    with hull contacts.  Sampled environments (and the most contact-rich
    one), stepped by the oracle from the GPU's settled state, match within
    the physics tolerance."""
    import dataclasses
    import torch
    if option == "gyroscopic_edges":
        sc = S.cfg2()
        sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, gyroscopic=1, edge_contacts=1))
    else:
        sc = S.generate(1024, 32, S.config_seed(2) ^ 0x4855, kinds="mixed_hulls", res=128, substeps=8,
                        hull_tris=(8, 48), n_hull_meshes=16)
        sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, hull_contacts=1))
    env = V.Env(sc)
    env.sim_step(120)
    torch.cuda.synchronize()
    settled = env.get_state()
    cc = env.contact_counts()
    assert cc.mean() > 2.0 * 32, cc.mean()
    env.sim_step(4)
    torch.cuda.synchronize()
    assert env.status()[1] == 0
    picks = CFG2_SAMPLE + (int(np.argmax(cc)),)
    _sampled_physics(orc, sc, env.get_state(), 4, picks, start=settled)
    env.close()


def _fine_hull(n, seed):
    """Convex hull of n random points on the unit sphere (2 n - 4 triangles)."""
    rng = np.random.default_rng(seed)
    P = rng.normal(size=(n, 3))
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    return S.hull_from_points(P)


@pytest.mark.parametrize("path", PATHS)
def test_render_fine_meshes_sieved(V, orc, path):
    """Batches with more triangles per environment than pixels per camera
    take the sieved set-up on the tiled path: hulls of 400 and 900 triangles
    crowding the eye of a 32 x 24 camera (four of them cut by the near
    plane), and one body whose 2,792
    triangles (a 700-vertex hull listed twice: equal depths, the lower id
    wins) fill two sieve windows of one chunk.  Frames equal the oracle's on
    both paths."""
    m1, m2 = _fine_hull(202, 1), _fine_hull(452, 2)
    eye, tgt = np.array([0.0, -2.5, 1.5]), np.array([0.0, 0.0, 0.4])
    f = (tgt - eye) / np.linalg.norm(tgt - eye)
    r = np.cross(f, [0.0, 0.0, 1.0])
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    rng = np.random.default_rng(7)
    bodies = []
    for i in range(10):
        d = rng.uniform(-0.03, 0.03) if i < 4 else rng.uniform(0.1, 0.6)   # the first four straddle the eye
        p = eye + f * d + r * rng.uniform(-0.1, 0.1) + u * rng.uniform(-0.08, 0.08)
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        bodies.append(dict(type="hull", mesh=m1 if i % 2 else m2, r=float(rng.uniform(0.05, 0.12)), pos=tuple(p),
                           quat=tuple(q)))
    crowd = S.custom(bodies, res=32, envs=2)
    crowd.cam_h[:] = 24
    Vd, Td = _fine_hull(700, 3)
    twice = (Vd, np.concatenate([Td, Td]))   # every triangle twice
    dense = S.custom([dict(type="hull", mesh=twice, r=0.4, pos=(0.0, 0.0, 0.5))], res=32)
    assert len(twice[1]) == 2792
    for sc in (crowd, dense):
        P = int(sc.cam_pix_off()[-1])
        assert (np.diff(sc.mesh_tri_off)[sc.mesh_id].sum() / sc.num_envs) > P / sc.cam_off[-1]   # sieved
        tid = _render_cmp(V, orc, sc, path=path)
        assert ((tid != 0xFFFFFFFF) & (tid >= 2)).any()
