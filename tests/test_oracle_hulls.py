"""Pins of the oracle's hull contacts (the hull_contacts option) against
closed forms of the regular octahedron, an independent rotation (scipy) and
resting configurations (CPU only).

The octahedron with vertices +-x, +-y, +-z scaled by r has the faces
n . x = r / sqrt(3), n = (+-1, +-1, +-1) / sqrt(3): a point at distance L
from the centre along a face normal has depth L - r / sqrt(3) below that
face's plane, and an octahedron resting on a face has its centre r / sqrt(3)
above the support.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2605_01352_b300 import scene as S

S3 = math.sqrt(3.0)
N111 = np.array([1.0, 1.0, 1.0]) / S3


def _params(**kw):
    return dataclasses.replace(S.SimParams(), hull_contacts=1, **kw)


def _quat_taking(u, v):
    """(w, x, y, z) of the rotation taking unit vector u to unit vector v (scipy)."""
    from scipy.spatial.transform import Rotation
    u = np.asarray(u, float) / np.linalg.norm(u)
    v = np.asarray(v, float) / np.linalg.norm(v)
    ax = np.cross(u, v)
    s = np.linalg.norm(ax)
    ang = math.atan2(s, float(np.dot(u, v)))
    if s < 1e-12:   # parallel or opposite: any axis normal to u
        ax = np.cross(u, [1.0, 0.0, 0.0] if abs(u[0]) < 0.9 else [0.0, 1.0, 0.0])
        s = np.linalg.norm(ax)
    rv = ax / s * ang
    x, y, z, w = Rotation.from_rotvec(rv).as_quat()
    return (w, x, y, z)


def _rot(q):
    from scipy.spatial.transform import Rotation
    w, x, y, z = q
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def test_hull_plane_contacts_are_its_low_vertices(orc):
    """Plane contacts of a hull: the vertices below the margin, in mesh order,
    at positions from an independent rotation, distance their height."""
    V, T = S.hull_from_points(_sphere_points(14, 3))
    q = np.array([0.8, 0.3, -0.4, 0.2])
    q /= np.linalg.norm(q)
    r = 0.1
    sc = S.custom([dict(type="hull", r=r, mesh=(V, T), pos=(0.05, -0.02, 0.085), quat=tuple(q))], params=_params())
    c = orc.contacts(sc, 0)
    R = _rot(sc.quat[:, 0].astype(np.float64))
    w = (R @ (r * V.astype(np.float64)).T).T + sc.pos[:, 0]
    exp = w[w[:, 2] < sc.params.margin]
    assert c["count"] == len(exp) >= 2
    np.testing.assert_allclose(c["p"], exp, atol=2e-6)
    np.testing.assert_allclose(c["d"], exp[:, 2], atol=2e-6)
    assert (c["b"] == -1).all() and (c["n"] == [0, 0, 1]).all()


def _sphere_points(n, seed):
    rng = np.random.default_rng(seed)
    P = rng.normal(size=(n, 3))
    return P / np.linalg.norm(P, axis=1, keepdims=True)


def test_hull_high_above_the_plane_has_no_plane_contacts(orc):
    V, T = S.octahedron()
    sc = S.custom([dict(type="hull", r=0.1, mesh=(V, T), pos=(0, 0, 0.121))], params=_params())
    assert orc.contacts(sc, 0)["count"] == 0
    sc = S.custom([dict(type="hull", r=0.1, mesh=(V, T), pos=(0, 0, 0.119))], params=_params())
    c = orc.contacts(sc, 0)
    assert c["count"] == 1 and abs(c["d"][0] - (0.119 - 0.1)) < 1e-6


@pytest.mark.parametrize("L", [0.16, 0.1577, 0.15])
def test_hull_vertex_into_hull_face_closed_form(orc, L):
    """Octahedron A (r = 0.1) turned so that a vertex points at the centre of
    octahedron B's face (1, 1, 1) / sqrt(3): one contact, normal that face's
    normal (from B to A), depth (L - r) - r / sqrt(3), point the vertex.
    The pair is (B, A) when B comes first, so the normal flips."""
    V, T = S.octahedron()
    r = 0.1
    qa = _quat_taking((-1, 0, 0), -N111)   # A's vertex -x points back along the normal
    pa = L * N111
    for a_first in (True, False):
        A = dict(type="hull", r=r, mesh=(V, T), pos=tuple(pa), quat=qa)
        B = dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, 0.0))
        sc = S.custom([A, B] if a_first else [B, A], params=_params(plane=0))
        c = orc.contacts(sc, 0)
        assert c["count"] == 1
        D = (L - r) - r / S3
        np.testing.assert_allclose(c["d"][0], D, atol=2e-6)
        np.testing.assert_allclose(c["p"][0], (L - r) * N111, atol=2e-6)
        n = N111 if a_first else -N111   # from the pair's second body to its first
        np.testing.assert_allclose(c["n"][0], n, atol=2e-6)
        assert (c["a"][0], c["b"][0]) == (0, 1)


@pytest.mark.parametrize("sphere_first", [True, False])
def test_sphere_on_a_hull_face_closed_form(orc, sphere_first):
    """A sphere's centre on the normal of a face at distance L: distance
    L - r / sqrt(3) - r_s, point the foot on the face plane, normal the face
    normal (from the hull to the sphere, flipped for the pair order)."""
    V, T = S.octahedron()
    r, rs, L = 0.1, 0.04, 0.095
    H = dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, 0.0))
    Sp = dict(type="sphere", r=rs, pos=tuple(L * N111))
    sc = S.custom([Sp, H] if sphere_first else [H, Sp], params=_params(plane=0))
    c = orc.contacts(sc, 0)
    assert c["count"] == 1
    np.testing.assert_allclose(c["d"][0], (L - r / S3) - rs, atol=2e-6)
    np.testing.assert_allclose(c["p"][0], (r / S3) * N111, atol=2e-6)
    np.testing.assert_allclose(c["n"][0], N111 if sphere_first else -N111, atol=2e-6)


def test_hull_depth_ties_go_to_the_first_face(orc):
    """A sphere straight below an octahedron is equally deep under the four
    lower faces: the contact takes the first of them in mesh order."""
    V, T = S.octahedron()
    r, rs, L = 0.1, 0.05, 0.15
    sc = S.custom([dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, 0.0)),
                   dict(type="sphere", r=rs, pos=(0.0, 0.0, -L))], params=_params(plane=0))
    c = orc.contacts(sc, 0)
    assert c["count"] == 1
    Vd = V.astype(np.float64)
    nrm = np.cross(Vd[T[:, 1]] - Vd[T[:, 0]], Vd[T[:, 2]] - Vd[T[:, 0]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    depth = nrm @ np.array([0.0, 0.0, -L]) - r * np.einsum("ij,ij->i", nrm, Vd[T[:, 0]])
    ties = np.flatnonzero(np.isclose(depth, depth.max()))
    assert len(ties) == 4
    # the hull is the pair's first body: the normal points from the sphere to the hull
    np.testing.assert_allclose(-c["n"][0], nrm[ties[0]], atol=2e-6)
    np.testing.assert_allclose(c["d"][0], (L / S3 - r / S3) - rs, atol=2e-6)


def test_box_corner_into_hull_face(orc):
    """A cube turned so that its corner (+,+,+) points at the octahedron's
    face centre from outside: one contact from the box's corners (the hull's
    vertices stay outside the box's sphere), depth from the closed form."""
    V, T = S.octahedron()
    r, h, L = 0.1, 0.03, 0.07
    hd = h * S3                          # corner distance from the box centre
    qb = _quat_taking(N111, -N111)       # the box's (+,+,+) corner points back at the hull
    sc = S.custom([dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, 0.0)),
                   dict(type="box", h=(h, h, h), pos=tuple((L + hd) * N111), quat=qb)], params=_params(plane=0))
    c = orc.contacts(sc, 0)
    assert c["count"] == 1
    np.testing.assert_allclose(c["d"][0], L - r / S3, atol=2e-6)
    np.testing.assert_allclose(c["p"][0], L * N111, atol=2e-6)
    np.testing.assert_allclose(c["n"][0], -N111, atol=2e-6)   # from the box (j) to the hull (i)


def test_hull_vertex_into_box_face(orc):
    """An octahedron's vertex -z pushed into a box's top face: one contact,
    normal +z (from the box to the hull), distance the vertex's height above
    the face, point the vertex."""
    V, T = S.octahedron()
    r, h = 0.1, (0.2, 0.2, 0.05)
    z = 0.05 + 0.1 - 0.004
    sc = S.custom([dict(type="box", h=h, pos=(0.0, 0.0, 0.0)),
                   dict(type="hull", r=r, mesh=(V, T), pos=(0.01, -0.02, z))], params=_params(plane=0))
    c = orc.contacts(sc, 0)
    assert c["count"] == 1
    np.testing.assert_allclose(c["d"][0], -0.004, atol=2e-6)
    np.testing.assert_allclose(c["p"][0], (0.01, -0.02, z - r), atol=2e-6)
    np.testing.assert_allclose(c["n"][0], (0.0, 0.0, -1.0), atol=2e-6)   # from the hull (j) to the box (i)
    assert (c["a"][0], c["b"][0]) == (0, 1)


def test_hull_contacts_come_after_the_others_in_order(orc):
    """Canonical order with hull contacts: plane contacts of spheres and
    boxes, their pairs, then the hulls' plane contacts, then the pairs with
    a hull."""
    V, T = S.octahedron()
    r = 0.1
    bodies = [dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, 0.095)),
              dict(type="sphere", r=0.05, pos=(0.5, 0.0, 0.049)),
              dict(type="sphere", r=0.05, pos=(0.5, 0.0, 0.148)),
              dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, 0.095 + 2 * r - 0.003))]
    c = orc.contacts(S.custom(bodies, params=_params()), 0)
    pairs = list(zip(c["a"].tolist(), c["b"].tolist()))
    # sphere 1 on the plane, spheres 1-2, hull 0 on the plane, then hulls 0-3
    # (tip on tip: the clipped incident face gives several points)
    assert pairs[:3] == [(1, -1), (1, 2), (0, -1)]
    assert len(pairs) > 3 and all(p == (0, 3) for p in pairs[3:])
    # the reference face is one of hull 0's upper faces (the separations tie):
    # the normal points from hull 3 down to hull 0
    for k in range(3, len(pairs)):
        assert c["n"][k][2] < -0.5 and abs(np.linalg.norm(c["n"][k]) - 1.0) < 1e-6


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_octahedron_comes_to_rest_on_a_face(orc, prec):
    """Dropped face down, an octahedron settles with its centre r / sqrt(3)
    above the ground (less the allowed penetration) and stops."""
    V, T = S.octahedron()
    r = 0.1
    q = _quat_taking(N111, (0, 0, -1))
    sc = S.custom([dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, r / S3 + 0.03), quat=q)], params=_params())
    st, flags, cc = orc.sim_step(sc, 240, precision=prec)
    assert flags[0] == 0 and cc[0] == 3
    assert abs(st["pos"][2, 0] - r / S3) < 2e-3
    assert np.abs(st["vel"][:, 0]).max() < 1e-2 and np.abs(st["angvel"][:, 0]).max() < 1e-1


def test_octahedra_stack_face_to_face(orc):
    """One octahedron resting face down on another (face up): after a
    second the upper centre sits 2 r / sqrt(3) above the lower one and the
    stack stands still."""
    V, T = S.octahedron()
    r = 0.1
    down = _quat_taking(N111, (0, 0, -1))
    up = _quat_taking(N111, (0, 0, 1))
    z0 = r / S3
    sc = S.custom([dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, z0), quat=up),
                   dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, 3 * z0 + 0.01), quat=down)],
                  params=_params())
    st, flags, cc = orc.sim_step(sc, 240, precision="f64")
    assert flags[0] == 0
    dz = st["pos"][2, 1] - st["pos"][2, 0]
    assert abs(dz - 2 * r / S3) < 3e-3
    assert abs(st["pos"][0, 1]) < 5e-3 and abs(st["pos"][1, 1]) < 5e-3
    assert np.abs(st["vel"]).max() < 2e-2


def test_hulls_without_hull_contacts_are_spheres(orc):
    """With the option off a hull body moves exactly as a sphere of its radius."""
    V, T = S.octahedron()
    common = dict(pos=(0.0, 0.0, 0.3), vel=(0.5, 0.0, 0.0), angvel=(0.0, 3.0, 0.0))
    a = S.custom([dict(type="hull", r=0.1, mesh=(V, T), **common)])
    b = S.custom([dict(type="sphere", r=0.1, **common)])
    sa, _, ca = orc.sim_step(a, 120)
    sb, _, cb = orc.sim_step(b, 120)
    for k in ("pos", "quat", "vel", "angvel"):
        np.testing.assert_array_equal(sa[k], sb[k])
    assert ca[0] == cb[0] == 1


def _face_up_and_down(r, gap):
    """Octahedron 0 with its face (1,1,1) up, octahedron 1 above it with its
    face (1,1,1) down, the two faces parallel at distance gap and turned 60
    degrees against each other (a hexagram seen from above)."""
    V, T = S.octahedron()
    up = _quat_taking(N111, (0, 0, 1))
    down = _quat_taking(N111, (0, 0, -1))
    z0 = r / S3
    return V, T, [dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, z0), quat=up),
                  dict(type="hull", r=r, mesh=(V, T), pos=(0.0, 0.0, 3 * z0 + gap), quat=down)]


@pytest.mark.parametrize("lower_first", [True, False])
def test_parallel_faces_turned_60_degrees_clip_to_a_hexagon(orc, lower_first):
    """Two parallel triangular faces turned against each other: the incident
    triangle clipped by the reference triangle's sides is the regular
    hexagon of circumradius 2 r_in / sqrt(3) (r_in = r / sqrt(6), the face's
    inradius); every corner is a contact at the gap's distance, normal +z
    (from the upper body to the lower)."""
    r, gap = 0.1, 0.01
    V, T, bodies = _face_up_and_down(r, gap)
    if not lower_first:
        bodies = bodies[::-1]
    c = orc.contacts(S.custom(bodies, params=_params(plane=0)), 0)
    assert c["count"] == 6
    np.testing.assert_allclose(c["d"], gap, atol=2e-6)
    rad = np.hypot(c["p"][:, 0], c["p"][:, 1])
    np.testing.assert_allclose(rad, 2.0 * (r / math.sqrt(6.0)) / S3, atol=2e-6)
    ang = np.sort(np.degrees(np.arctan2(c["p"][:, 1], c["p"][:, 0])) % 360.0)
    np.testing.assert_allclose(np.diff(ang), 60.0, atol=1e-3)
    # normal from the pair's second body to its first
    np.testing.assert_allclose(c["n"], np.tile([0.0, 0.0, -1.0 if lower_first else 1.0], (6, 1)), atol=2e-6)
    # the separations tie (up to rounding), so the reference face is the
    # first body's and the points lie on the second body's (incident) face
    np.testing.assert_allclose(c["p"][:, 2], 2 * r / S3 + (gap if lower_first else 0.0), atol=2e-6)


def test_octahedron_face_down_on_a_box_gives_its_three_corners(orc):
    """An octahedron face down on a wide box: the incident face (its lower
    face) lies inside the box's top face, so its three corners are the
    contacts, at the gap's distance, normal -z (from the hull to the box)."""
    V, T = S.octahedron()
    r, gap = 0.1, 0.004
    down = _quat_taking(N111, (0, 0, -1))
    sc = S.custom([dict(type="box", h=(0.3, 0.3, 0.05), pos=(0.0, 0.0, 0.0)),
                   dict(type="hull", r=r, mesh=(V, T), pos=(0.02, 0.01, 0.05 + r / S3 + gap), quat=down)],
                  params=_params(plane=0))
    c = orc.contacts(sc, 0)
    assert c["count"] == 3
    np.testing.assert_allclose(c["d"], gap, atol=2e-6)
    R = _rot(sc.quat[:, 1].astype(np.float64))
    w = (R @ (r * V.astype(np.float64)).T).T + sc.pos[:, 1]
    low = w[np.argsort(w[:, 2])[:3]]
    for p in c["p"]:
        assert np.min(np.linalg.norm(low - p, axis=1)) < 2e-6
    np.testing.assert_allclose(c["n"], np.tile([0.0, 0.0, -1.0], (3, 1)), atol=2e-6)


def test_separated_polytopes_have_no_contacts(orc):
    """Beyond the margin along a face normal the pair has no contacts."""
    r = 0.1
    V, T, bodies = _face_up_and_down(r, 0.021)
    assert orc.contacts(S.custom(bodies, params=_params(plane=0)), 0)["count"] == 0
