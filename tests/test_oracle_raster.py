"""Pins of the oracle's rasteriser and camera render (CPU only).

The rasteriser is checked against geometry it must reproduce exactly
(rectangle pixel counts, a tiling mesh covered exactly once), against an
independent exact-rational barycentric inside test with its own top/left
edge definition, and the render against closed forms for the ground plane.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2605_01352_b300 import scene as S

FX = 256


def _front(tri):
    """Reorder a triangle (3 x 2 fixed-point) so that it is counter-clockwise
    on screen as seen by the camera (clockwise in y-down coordinates)."""
    (x0, y0), (x1, y1), (x2, y2) = tri
    a = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0)
    return tri if a < 0 else [tri[0], tri[2], tri[1]]


def _rect(x0, y0, x1, y1):
    return [_front([(x0, y0), (x1, y0), (x1, y1)]), _front([(x0, y0), (x1, y1), (x0, y1)])]


@pytest.mark.parametrize("off", [0, 128])
def test_rectangle_pixel_counts(orc, off):
    """An axis-aligned rectangle [x0, x1) x [y0, y1) covers exactly
    (x1 - x0)(y1 - y0) pixels, whether its corners sit on pixel corners or
    on pixel centres (left/top edges in, right/bottom edges out)."""
    rng = np.random.default_rng(1)
    W, H = 40, 24
    for _ in range(20):
        x0, x1 = sorted(rng.choice(W + 1, 2, replace=False))
        y0, y1 = sorted(rng.choice(H + 1, 2, replace=False))
        tris = _rect(FX * x0 + off, FX * y0 + off, FX * x1 + off, FX * y1 + off)
        tid, dep, cnt = orc.raster_screen_tris(np.array(tris), np.ones((2, 3)), W, H, count=True)
        assert cnt.max() <= 1
        assert int((cnt == 1).sum()) == (x1 - x0) * (y1 - y0)
        covered = np.argwhere(cnt == 1)
        ys, xs = covered[:, 0], covered[:, 1]
        assert xs.min() == x0 and xs.max() == x1 - 1 and ys.min() == y0 and ys.max() == y1 - 1


def test_back_faces_and_degenerates_are_not_drawn(orc):
    tri = _front([(0, 0), (FX * 10, 0), (0, FX * 10)])
    back = [tri[0], tri[2], tri[1]]
    line = [(0, 0), (FX * 5, FX * 5), (FX * 10, FX * 10)]
    tid, _, cnt = orc.raster_screen_tris(np.array([back, line]), np.ones((2, 3)), 16, 16, count=True)
    assert cnt.sum() == 0 and (tid == 0xFFFFFFFF).all()
    tid, _, cnt = orc.raster_screen_tris(np.array([tri]), np.ones((1, 3)), 16, 16, count=True)
    assert cnt.sum() > 0


def test_jittered_grid_covers_every_pixel_once(orc):
    """A mesh of jittered quads (two triangles each) tiling a region larger
    than the image covers every pixel exactly once: no gaps at shared edges
    or vertices, no double coverage (watertightness of the tie rule)."""
    rng = np.random.default_rng(7)
    W, H = 48, 40
    n = 9
    gx = np.linspace(-2 * FX, (W + 2) * FX, n + 1)
    gy = np.linspace(-2 * FX, (H + 2) * FX, n + 1)
    P = np.zeros((n + 1, n + 1, 2), np.int64)
    for i in range(n + 1):
        for j in range(n + 1):
            jx = rng.integers(-300, 300) if 0 < i < n else 0
            jy = rng.integers(-300, 300) if 0 < j < n else 0
            P[i, j] = (int(gx[i]) + jx, int(gy[j]) + jy)
    # put a few vertices exactly on pixel centres and corners to force ties
    P[3, 3] = (FX * 10 + 128, FX * 12 + 128)
    P[5, 4] = (FX * 25, FX * 17)
    tris = []
    for i in range(n):
        for j in range(n):
            a, b, c, d = P[i, j], P[i + 1, j], P[i + 1, j + 1], P[i, j + 1]
            if (i + j) % 2:
                tris += [_front([a, b, c]), _front([a, c, d])]
            else:
                tris += [_front([a, b, d]), _front([b, c, d])]
    tid, _, cnt = orc.raster_screen_tris(np.array(tris), np.ones((len(tris), 3)), W, H, count=True)
    assert (cnt == 1).all()


def test_fan_is_watertight(orc):
    """A triangle fan around an interior point: no pixel is covered twice,
    and every pixel strictly inside the polygon (by an exact test) is
    covered."""
    rng = np.random.default_rng(11)
    W = H = 32
    c = (FX * 16 + 77, FX * 15 + 13)
    k = 13
    ang = np.sort(rng.uniform(0, 2 * np.pi, k))
    rad = rng.uniform(6, 15, k) * FX
    pts = [(int(c[0] + r * math.cos(a)), int(c[1] + r * math.sin(a))) for a, r in zip(ang, rad)]
    tris = [_front([c, pts[i], pts[(i + 1) % k]]) for i in range(k)]
    _, _, cnt = orc.raster_screen_tris(np.array(tris), np.ones((k, 3)), W, H, count=True)
    assert cnt.max() == 1
    # every pixel centre strictly inside one of the fan triangles is covered
    for y in range(H):
        for x in range(W):
            p = (FX * x + 128, FX * y + 128)
            for t in tris:
                if _strictly_inside(t, p):
                    assert cnt[y, x] == 1
                    break


def _bary(t, p):
    """Exact barycentric coordinates (Fractions) of p in triangle t."""
    (x0, y0), (x1, y1), (x2, y2) = [(Fraction(int(a)), Fraction(int(b))) for a, b in t]
    px, py = Fraction(int(p[0])), Fraction(int(p[1]))
    det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
    l1 = ((px - x0) * (y2 - y0) - (x2 - x0) * (py - y0)) / det
    l2 = ((x1 - x0) * (py - y0) - (px - x0) * (y1 - y0)) / det
    return (1 - l1 - l2, l1, l2)


def _strictly_inside(t, p):
    return all(l > 0 for l in _bary(t, p))


def _owns_edge(t, i):
    """Top-left ownership of the edge opposite vertex i, from geometry: a
    horizontal edge is owned iff the triangle lies below it (y down); any
    other edge is owned iff the triangle lies to its right."""
    P, Q, R = t[(i + 1) % 3], t[(i + 2) % 3], t[i]
    if P[1] == Q[1]:
        return R[1] > P[1]
    xl = Fraction(int(P[0])) + Fraction(int(R[1] - P[1]) * int(Q[0] - P[0]), int(Q[1] - P[1]))
    return R[0] > xl


def test_brute_force_barycentric(orc):
    """On small images, a pixel is covered iff its exact barycentric
    coordinates are all positive, or zero on an owned (top/left) edge; the
    depth is the perspective-correct interpolation 1 / sum(l_i / z_i)
    (computed in double) within 1e-6 relative."""
    rng = np.random.default_rng(5)
    for trial in range(60):
        W, H = int(rng.integers(8, 17)), int(rng.integers(8, 17))
        # vertices on a coarse sub-pixel grid so that edge ties occur often
        q = int(rng.choice([1, 64, 128]))
        v = rng.integers(-3 * FX // q, (W + 3) * FX // q, (3, 2)) * q
        t = _front([tuple(int(a) for a in r) for r in v])
        z = rng.uniform(0.5, 5.0, 3)
        tid, dep, cnt = orc.raster_screen_tris(np.array([t]), z[None, :], W, H, count=True)
        area = (t[1][0] - t[0][0]) * (t[2][1] - t[0][1]) - (t[1][1] - t[0][1]) * (t[2][0] - t[0][0])
        z32 = z.astype(np.float32).astype(np.float64)
        for y in range(H):
            for x in range(W):
                p = (FX * x + 128, FX * y + 128)
                if area == 0:
                    exp = False
                else:
                    lam = _bary(t, p)
                    exp = all(l > 0 or (l == 0 and _owns_edge(t, i)) for i, l in enumerate(lam))
                assert bool(cnt[y, x]) == exp, (trial, x, y)
                if exp:
                    zz = 1.0 / sum(float(l) / zi for l, zi in zip(lam, z32))
                    assert dep[y, x] == pytest.approx(zz, rel=1e-6)


def test_depth_order_and_ties(orc):
    """The nearer triangle wins; at equal depth the lower id wins."""
    a = _rect(0, 0, FX * 8, FX * 8)
    tris = np.array(a + a + a)
    z = np.array([[3.0] * 3, [3.0] * 3, [2.0] * 3, [2.0] * 3, [2.0] * 3, [2.0] * 3])
    tid, dep, _ = orc.raster_screen_tris(tris, z, 8, 8)
    assert set(np.unique(tid)) == {2, 3}
    assert (dep == np.float32(2.0)).all()


def _ground_only(res=64, fov=60.0, eye=(0.0, -2.5, 1.5), target=(0.0, 0.0, 0.4)):
    sc = S.custom([dict(type="sphere", r=0.05, pos=(0.0, 0.0, -5.0))], res=res,
                  cams=[dict(eye=eye, target=target, fov=fov)])
    return sc


def test_ground_depth_and_colour_closed_form(orc):
    """Ground pixels: the depth is the view depth of the ray/plane
    intersection, -eye_z / d_z for the pixel-centre ray d = f + a r - b u;
    the colour is the albedo times 0.2 + 0.8 max(0, n . L) with n = +z."""
    sc = _ground_only()
    rgb, dep, tid, flags = orc.render(sc)
    W = H = 64
    eye, r, u, f = (sc.cam_eye[0].astype(np.float64), sc.cam_right[0].astype(np.float64),
                    sc.cam_up[0].astype(np.float64), sc.cam_fwd[0].astype(np.float64))
    fpy = float(sc.cam_fpy[0])
    g = tid.reshape(H, W)
    d = dep.reshape(H, W)
    hit = 0
    for y in range(H):
        for x in range(W):
            a = (x + 0.5 - W / 2) / fpy
            b = (y + 0.5 - H / 2) / fpy
            ray = f + a * r - b * u
            if ray[2] >= 0:
                continue
            t = -eye[2] / ray[2]
            wpt = eye + t * ray
            if abs(wpt[0]) < 1.49 and abs(wpt[1]) < 1.49:
                assert g[y, x] in (0, 1)
                assert d[y, x] == pytest.approx(t, rel=2e-4)
                hit += 1
            elif abs(wpt[0]) > 1.51 or abs(wpt[1]) > 1.51:
                assert g[y, x] == 0xFFFFFFFF and d[y, x] == 0.0
    assert hit > 1000
    L = sc.light.astype(np.float64)
    I = 0.2 + 0.8 * max(0.0, L[2])
    exp = int(128 * I + 0.5)
    cols = rgb[(tid == 0) | (tid == 1)]
    assert np.abs(cols.astype(int) - exp).max() <= 1
    assert (rgb[tid == 0xFFFFFFFF] == 0).all()


def test_sphere_silhouette_area(orc):
    """A sphere straight ahead covers about the area of its projected disc:
    between the discs of the icosphere's inscribed and circumscribed radii
    (plus a one-pixel boundary band)."""
    r = 0.3
    D = 2.0
    sc = S.custom([dict(type="sphere", r=r, pos=(0.0, 0.0, 1.0))], res=64,
                  cams=[dict(eye=(0.0, -D, 1.0), target=(0.0, 0.0, 1.0), fov=60.0)])
    rgb, dep, tid, _ = orc.render(sc)
    fpy = float(sc.cam_fpy[0])
    body = int(((tid != 0xFFFFFFFF) & (tid >= 2)).sum())
    V, T = S.icosphere(1)
    c = V[T].mean(1)
    r_in = r * float(np.linalg.norm(c, axis=1).min())
    # sphere of radius r at distance D subtends a disc of angular radius asin(r/D)
    rad = lambda rr: fpy * math.tan(math.asin(rr / D))
    lo, hi = math.pi * (rad(r_in) - 1) ** 2, math.pi * (rad(r) + 1) ** 2
    assert lo <= body <= hi
    # the nearest visible depth is D - r at the centre (within the facet error)
    assert dep.reshape(64, 64)[32, 32] == pytest.approx(D - r, rel=0.02)


def test_body_behind_the_camera_draws_nothing(orc):
    """A body wholly behind the camera (every vertex before the near plane)
    leaves no fragment and raises no flag."""
    sc = S.custom([dict(type="sphere", r=0.1, pos=(0.0, -3.0, 1.5))], res=32)
    rgb, dep, tid, flags = orc.render(sc)
    assert flags[0] == 0
    assert not ((tid >= 2) & (tid != 0xFFFFFFFF)).any()


def _near_face_scene(res=128):
    """A camera 2^-9 m above the top face of a large box, looking straight
    along +y (the camera basis is exact: right = x, up = z, forward = y).
    The face (z = 1, |x| <= 1, -0.5 <= y <= 1.5) passes through the near
    plane: its two triangles cross it, one with one vertex behind the
    camera, the other with two."""
    h = 2.0 ** -9
    sc = S.custom([dict(type="box", h=(1.0, 1.0, 0.125), pos=(0.0, 0.5, 0.875))], res=res,
                  cams=[dict(eye=(0.0, 0.0, 1.0 + h), target=(0.0, 1.0, 1.0 + h), fov=60.0)])
    assert (sc.cam_right[0] == [1, 0, 0]).all() and (sc.cam_up[0] == [0, 0, 1]).all()
    assert (sc.cam_fwd[0] == [0, 1, 0]).all()
    return sc, h


def test_face_crossing_the_near_plane_is_clipped_not_dropped(orc):
    """Sutherland-Hodgman clipping at zc = near: the part of the face in
    front of the near plane is drawn.  A pixel-centre ray (a, 1, -b) meets
    the face at view depth t = h / b; it is covered iff t >= near (the
    clipped edge, projected to row H/2 + fpy h / near) and the hit lies on
    the face.  Every pixel of rows 64..85 is covered by the face (no gap
    along the fan diagonal or the triangles' shared edge), no other pixel
    is, and the depth is the ray's t (down to 1.007 near on the last row,
    next to the clipped edge)."""
    res = 128
    sc, h = _near_face_scene(res)
    rgb, dep, tid, flags = orc.render(sc)
    # the ground quad (z = 0, 1 m below) also crosses the near plane, but it
    # lies wholly below the frustum's bottom plane: culled, no flag (its
    # clipped corners would project beyond the guard band)
    assert flags[0] == 0
    assert not ((tid == 0) | (tid == 1)).any()
    fpy = float(sc.cam_fpy[0])
    near = float(np.float32(0.01))
    face = ((tid != 0xFFFFFFFF) & (tid >= 2)).reshape(res, res)
    exp = np.zeros((res, res), bool)
    tray = np.zeros((res, res))
    for py in range(res):
        b = (py + 0.5 - res / 2) / fpy
        if b <= 0:
            continue
        t = h / b
        for px in range(res):
            a = (px + 0.5 - res / 2) / fpy
            if near <= t <= 1.5 and abs(a * t) <= 1.0:
                exp[py, px] = True
                tray[py, px] = t
    # the clipped edge lies between pixel-centre rows (no tie to resolve)
    edge_row = res / 2 + fpy * h / near
    assert abs(edge_row - round(edge_row - 0.5) - 0.5) > 0.05
    rows = np.nonzero(exp.any(1))[0]
    assert rows[0] == 64 and rows[-1] == 85 and exp[64:86].all()
    np.testing.assert_array_equal(face, exp)
    # depth: the face is seen at a grazing angle (its far edge projects
    # 0.14 px below the horizon), so the 1/256 px snapping of its vertices
    # tilts the interpolated plane by up to a few 1e-4; the interpolation
    # itself is pinned to 1e-6 elsewhere
    d = dep.reshape(res, res)
    np.testing.assert_allclose(d[exp], tray[exp], rtol=1e-3)
    assert d[85].min() < 1.01 * near
    # both triangles of the face contribute (one clipped to a triangle, one to a quad)
    assert len(np.unique(tid.reshape(res, res)[exp])) == 2


def test_clipped_edge_shared_by_two_triangles_is_watertight(orc):
    """The same face split differently: with the box turned 90 degrees about
    z the face's diagonal runs the other way, so the near plane cuts the
    triangles' shared edge from the other side; coverage is still exactly
    the clipped face, with no pixel lost or drawn twice along the cut."""
    res = 96
    h = 2.0 ** -9
    s = math.sqrt(0.5)
    sc = S.custom([dict(type="box", h=(1.0, 1.0, 0.125), pos=(0.0, 0.5, 0.875), quat=(s, 0.0, 0.0, s))], res=res,
                  cams=[dict(eye=(0.0, 0.0, 1.0 + h), target=(0.0, 1.0, 1.0 + h), fov=60.0)])
    _, _, tid, flags = orc.render(sc)
    assert flags[0] == 0
    fpy = float(sc.cam_fpy[0])
    near = float(np.float32(0.01))
    face = ((tid != 0xFFFFFFFF) & (tid >= 2)).reshape(res, res)
    rows = [py for py in range(res) if (py + 0.5 - res / 2) > 0 and h * fpy / (py + 0.5 - res / 2) >= near]
    exp = np.zeros((res, res), bool)
    exp[rows] = True
    np.testing.assert_array_equal(face, exp)


def test_scene_meshes_are_closed_and_outward():
    """Input meshes (icosphere, cube, convex hulls): closed 2-manifolds with
    Euler characteristic 2 whose triangles all face away from the centre."""
    from paper_2605_01352_b300 import scene as S
    meshes = [S.icosphere(1), S.cube()]
    st = S.Streams(7, 1)
    meshes += [S.convex_hull_mesh(st, t) for t in (500, 512)]
    for V, T in meshes:
        edges = {}
        for a, b, c in T:
            for u, v in ((a, b), (b, c), (c, a)):
                edges[(u, v)] = edges.get((u, v), 0) + 1
        # every directed edge once and its reverse once: closed and consistently oriented
        assert all(n == 1 for n in edges.values())
        assert all((v, u) in edges for (u, v) in edges)
        nE = len(edges) // 2
        assert len(V) - nE + len(T) == 2
        Vd = V.astype(np.float64)
        n = np.cross(Vd[T[:, 1]] - Vd[T[:, 0]], Vd[T[:, 2]] - Vd[T[:, 0]])
        assert (np.einsum("ij,ij->i", n, Vd[T].mean(1)) > 0).all()
    assert S.icosphere(1)[1].shape == (80, 3) and S.icosphere(1)[0].shape == (42, 3)


def test_guard_band_vertex_discards_triangle(orc):
    """A vertex beyond the 2^14-pixel guard band (2^22 in 1/256 px) discards
    its triangle; one exactly on the band's edge is kept (hook rule, as the
    projection's guard-band discard in the renderer)."""
    lim = 1 << 22
    big = _front([(lim, lim), (-lim, lim), (lim, -lim)])   # covers x + y > 0: the whole image
    tid, _, _ = orc.raster_screen_tris(np.array([big]), np.ones((1, 3)), 8, 8)
    assert (tid == 0).all()
    over = _front([(lim + 1, lim), (-lim, lim), (lim, -lim)])
    tid, _, _ = orc.raster_screen_tris(np.array([over]), np.ones((1, 3)), 8, 8)
    assert (tid == 0xFFFFFFFF).all()


def test_box_with_unequal_half_extents_seen_face_on(orc):
    """A box of half extents (a, b, c), turned 90 degrees about the world y
    axis (its local x along world -z, local z along world x), straight ahead
    of a camera looking along +y.  The mesh is scaled before it is rotated,
    so the silhouette is the front face: a rectangle of 2c by 2a world units
    at view depth zf = D - b.  The sizes put its projected edges on pixel
    corners (fpy c / zf = 12, fpy a / zf = 20 pixels), so it covers exactly
    24 columns by 40 rows around the image centre, at depth zf, in the flat
    colour of a face whose normal is -y."""
    res = 128
    fpy = (res / 2) / math.tan(math.radians(30.0))
    zf = 2.0
    c, a, b = 12 * zf / fpy, 20 * zf / fpy, 0.1
    D = zf + b
    s = math.sqrt(0.5)
    sc = S.custom([dict(type="box", h=(a, b, c), pos=(0.0, 0.0, 1.0), quat=(s, 0.0, s, 0.0))], res=res,
                  cams=[dict(eye=(0.0, -D, 1.0), target=(0.0, 0.0, 1.0), fov=60.0)])
    rgb, dep, tid, flags = orc.render(sc)
    assert flags[0] == 0
    body = ((tid != 0xFFFFFFFF) & (tid >= 2)).reshape(res, res)
    exp = np.zeros((res, res), bool)
    exp[64 - 20:64 + 20, 64 - 12:64 + 12] = True
    np.testing.assert_array_equal(body, exp)
    np.testing.assert_allclose(dep.reshape(res, res)[exp], zf, rtol=1e-6)
    L = sc.light.astype(np.float64)
    I = 0.2 + 0.8 * max(0.0, -L[1])
    want = np.array([int(ch * I + 0.5) for ch in S.PALETTE[0]])
    assert np.abs(rgb.reshape(res, res, 3)[exp].astype(int) - want).max() <= 1


def test_guard_band_flag_only_for_triangles_that_reach_the_image(orc):
    """A vertex in front of the camera but beyond the 2^14 px guard band
    discards its triangle with the guard flag -- unless the triangle lies
    wholly beyond one side plane of the frustum, where it could not cover a
    pixel anyway (culled silently).  Camera at (0, 0, 1) looking along +y."""
    cam = [dict(eye=(0.0, 0.0, 1.0), target=(0.0, 1.0, 1.0), fov=60.0)]
    # a slab 3 cm ahead spanning x = -4 .. 4 m: its front corners project to
    # |sx| ~ 1.8e4 px, beyond the band, and it crosses the view: flagged
    wide = S.custom([dict(type="box", h=(4.0, 0.005, 0.05), pos=(0.0, 0.03, 1.0))], res=128, cams=cam)
    _, _, tid, flags = orc.render(wide)
    assert flags[0] == 4
    # the same slab moved 6 m to the right lies wholly right of the image
    # (fpy xc > W/2 zc at every vertex): culled without a flag
    right = S.custom([dict(type="box", h=(4.0, 0.005, 0.05), pos=(6.0, 0.03, 1.0))], res=128, cams=cam)
    _, _, tid, flags = orc.render(right)
    assert flags[0] == 0
    assert not ((tid >= 2) & (tid != 0xFFFFFFFF)).any()
