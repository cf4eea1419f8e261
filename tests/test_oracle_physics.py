"""Pins of the oracle's physics step against closed forms, textbook results
and conservation laws (CPU only).

Each test targets a mistake that would survive a self-comparison: a wrong
sign or index in the quaternion/rotation formulas, a dropped r x P term in
the impulse, a wrong effective mass, a mis-ordered integrator.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2605_01352_b300 import scene as S


def _one(body, **pk):
    p = dataclasses.replace(S.SimParams(), **pk)
    return S.custom([body], params=p)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 3e-5)])
def test_ballistic_closed_form(orc, prec, tol):
    """Semi-implicit Euler with constant g: v_n = v0 + n h g and
    x_n = x0 + n h v0 + h^2 g n(n+1)/2 (exact discrete solution)."""
    sc = _one(dict(type="sphere", r=0.05, pos=(0.1, -0.2, 50.0), vel=(1.0, 2.0, 3.0)), substeps=4)
    steps = 25
    st, _, cc = orc.sim_step(sc, steps, precision=prec)
    h = sc.params.dt / sc.params.substeps
    n = steps * sc.params.substeps
    g = np.array(sc.params.gravity)
    v0 = np.array([1.0, 2.0, 3.0])
    x0 = np.array([0.1, -0.2, 50.0], dtype=np.float32).astype(np.float64)
    v = v0 + n * h * g
    x = x0 + n * h * v0 + h * h * g * n * (n + 1) / 2.0
    assert cc[0] == 0
    np.testing.assert_allclose(st["vel"][:, 0], v, rtol=tol, atol=tol)
    np.testing.assert_allclose(st["pos"][:, 0], x, rtol=tol, atol=tol * 50)


def test_free_flight_energy_drift(orc):
    """Semi-implicit Euler loses exactly m g^2 h^2 / 2 of energy per substep
    in free flight: E_n - E_0 = -m |g|^2 h^2 n / 2."""
    sc = _one(dict(type="box", h=(0.05, 0.07, 0.09), pos=(0.0, 0.0, 80.0), vel=(0.5, -1.0, 2.0)))
    m = 1.0 / float(sc.inv_mass[0])
    g = np.array(sc.params.gravity)
    h = sc.params.dt / sc.params.substeps

    def energy(st):
        v = st["vel"][:, 0]
        return 0.5 * m * float(v @ v) - m * float(g @ st["pos"][:, 0])

    s0 = {k: v.astype(np.float64) for k, v in sc.state().items()}
    st, _, _ = orc.sim_step(sc, 30, state=s0, precision="f64")
    n = 30 * sc.params.substeps
    assert energy(st) - energy(s0) == pytest.approx(-0.5 * m * float(g @ g) * h * h * n, rel=1e-7)


@pytest.mark.parametrize("body", [
    dict(type="sphere", r=0.08, pos=(0.0, 0.0, 10.0), angvel=(0.0, 0.0, 7.0)),
    dict(type="box", h=(0.03, 0.06, 0.1), pos=(0.0, 0.0, 10.0), angvel=(0.0, 0.0, -5.0)),
])
def test_rotation_angle_closed_form(orc, body):
    """With omega along z and no torque, each substep rotates the quaternion
    by exactly 2 atan(h w / 2) (first-order update then renormalise)."""
    sc = _one(body, gravity=(0.0, 0.0, 0.0))
    steps = 40
    st, _, _ = orc.sim_step(sc, steps, precision="f64")
    w = body["angvel"][2]
    h = sc.params.dt / sc.params.substeps
    ang = 2 * steps * sc.params.substeps * math.atan(h * w / 2)
    q = st["quat"][:, 0]
    np.testing.assert_allclose(q, [math.cos(ang / 2), 0, 0, math.sin(ang / 2)], atol=1e-12)
    np.testing.assert_allclose(st["angvel"][:, 0], body["angvel"], atol=0)


def test_resting_sphere_stays(orc):
    """A sphere touching the plane at rest: the normal impulse cancels
    gravity every substep, no friction acts, and it stays put."""
    r = 0.07
    sc = _one(dict(type="sphere", r=r, pos=(0.2, 0.1, r)))
    st, _, cc = orc.sim_step(sc, 1000)
    assert cc[0] == 1
    assert abs(float(st["pos"][2, 0]) - r) < 1e-5
    assert np.abs(st["vel"][:, 0]).max() < 1e-5
    assert np.abs(st["pos"][:2, 0] - [0.2, 0.1]).max() < 1e-7
    assert np.abs(st["angvel"][:, 0]).max() == 0.0


def test_resting_cube_symmetry(orc):
    """A cube face-down on the plane: the four corner contacts are symmetric
    and their torques cancel exactly.  With mass splitting each corner sees
    k_n = 4 (1/m + 3/m) = 16/m, so every Jacobi iteration removes a quarter
    of the remaining approach speed: after one substep of K iterations
    v_z = -(3/4)^K h g."""
    a = 0.05
    sc = _one(dict(type="box", h=(a, a, a), pos=(0.0, 0.0, a)), substeps=1)
    st, _, cc = orc.sim_step(sc, 1, precision="f64")
    assert cc[0] == 4
    assert np.abs(st["angvel"][:, 0]).max() == 0.0
    h = sc.params.dt
    K = sc.params.iterations
    assert st["vel"][2, 0] == pytest.approx(-(0.75 ** K) * h * 9.81, rel=1e-6)
    assert st["vel"][0, 0] == 0.0 and st["vel"][1, 0] == 0.0
    sc = _one(dict(type="box", h=(a, a, a), pos=(0.0, 0.0, a)))
    # the remaining approach speed lets it sink until the position bias,
    # which acts only beyond the allowed penetration (slop), holds it
    st, _, _ = orc.sim_step(sc, 1000)
    assert float(st["pos"][2, 0]) == pytest.approx(a - sc.params.slop, abs=5e-5)
    assert abs(float(st["vel"][2, 0])) < 1e-5
    assert np.abs(st["angvel"][:, 0]).max() == 0.0


def test_sliding_sphere_rolls_at_five_sevenths(orc):
    """Textbook: a solid sphere launched sliding without spin on a rough
    plane ends up rolling at 5/7 of its initial speed, with w r = v."""
    r = 0.08
    v0 = 2.0
    sc = _one(dict(type="sphere", r=r, pos=(0.0, 0.0, r), vel=(v0, 0.0, 0.0)))
    st, _, _ = orc.sim_step(sc, 240, precision="f64")
    vx = st["vel"][0, 0]
    wy = st["angvel"][1, 0]
    assert vx == pytest.approx(5.0 / 7.0 * v0, rel=2e-3)
    assert wy * r == pytest.approx(vx, rel=2e-3)


def test_sliding_box_stopping_distance(orc):
    """A cube sliding face-down decelerates at mu g: it stops after
    v0^2 / (2 mu g)."""
    a = 0.05
    v0 = 1.0
    sc = _one(dict(type="box", h=(a, a, a), pos=(0.0, 0.0, a), vel=(v0, 0.0, 0.0)))
    st, _, _ = orc.sim_step(sc, 240, precision="f64")
    mu, g = sc.params.friction, 9.81
    assert abs(st["vel"][0, 0]) < 2e-3  # stopped (from 1 m/s)
    assert st["pos"][0, 0] == pytest.approx(v0 * v0 / (2 * mu * g), rel=0.03)


@pytest.mark.parametrize("deg", [20.0, 35.0])
def test_box_on_an_incline_sticks_or_slides(orc, deg):
    """A flat box on the ground under gravity tilted by theta (the same as a
    slope of angle theta): its four corner contacts hold it when tan theta
    < mu (Coulomb static friction), and below the cone's edge it slides with
    acceleration g (sin theta - mu cos theta)."""
    th = math.radians(deg)
    g = 9.81
    sc = _one(dict(type="box", h=(0.1, 0.1, 0.02), pos=(0.0, 0.0, 0.02)),
              gravity=(g * math.sin(th), 0.0, -g * math.cos(th)))
    mu = sc.params.friction
    st, _, cc = orc.sim_step(sc, 60, precision="f64")            # settle onto the corners
    assert cc[0] == 4
    st2, _, _ = orc.sim_step(sc, 120, state=st, precision="f64")  # 0.5 s more
    t = 120 * sc.params.dt
    if math.tan(th) < mu:
        assert abs(st2["vel"][0, 0]) < 1e-3 and abs(st2["pos"][0, 0] - st["pos"][0, 0]) < 1e-3
    else:
        acc = g * (math.sin(th) - mu * math.cos(th))
        assert (st2["vel"][0, 0] - st["vel"][0, 0]) / t == pytest.approx(acc, rel=0.02)
    assert np.abs(st2["angvel"][:, 0]).max() < 1e-2          # it neither tips nor spins


def _sphere_cloud(n, seed, spread=0.25, speed=1.0):
    rng = np.random.default_rng(seed)
    bodies = []
    for i in range(n):
        bodies.append(dict(type="sphere", r=float(rng.uniform(0.05, 0.1)),
                           pos=tuple(rng.uniform(-spread, spread, 3) + [0, 0, 5.0]),
                           vel=tuple(rng.uniform(-speed, speed, 3)),
                           angvel=tuple(rng.uniform(-3, 3, 3))))
    return bodies


def test_momentum_conservation_pairs(orc):
    """No gravity, no plane: pair impulses are equal and opposite at a common
    point, so linear momentum and (for spheres, whose world inertia does not
    rotate) angular momentum about the origin are conserved."""
    p = dataclasses.replace(S.SimParams(), gravity=(0.0, 0.0, 0.0), plane=0)
    sc = S.custom(_sphere_cloud(12, 3), params=p)
    m = 1.0 / sc.inv_mass.astype(np.float64)
    I = 1.0 / sc.inv_inertia.astype(np.float64)

    def moments(st):
        P = (m * st["vel"]).sum(1)
        L = (I * st["angvel"]).sum(1) + (m * np.cross(st["pos"].T, st["vel"].T).T).sum(1)
        return P, L

    s0 = {k: v.astype(np.float64) for k, v in sc.state().items()}
    P0, L0 = moments(s0)
    st, _, _ = orc.sim_step(sc, 30, state=s0, precision="f64")
    st1, _, cc = orc.sim_step(sc, 1, state=s0, precision="f64")
    assert cc[0] > 0  # the cloud is in contact
    P1, L1 = moments(st)
    np.testing.assert_allclose(P1, P0, atol=1e-12)
    np.testing.assert_allclose(L1, L0, atol=1e-12)
    # and something did happen
    assert np.abs(st["vel"] - s0["vel"]).max() > 1e-3


def test_head_on_inelastic(orc):
    """Equal spheres meeting head on with e = 0 stop along the normal."""
    p = dataclasses.replace(S.SimParams(), gravity=(0.0, 0.0, 0.0), plane=0)
    sc = S.custom([dict(type="sphere", r=0.05, pos=(-0.06, 0, 1), vel=(1, 0, 0)),
                   dict(type="sphere", r=0.05, pos=(0.06, 0, 1), vel=(-1, 0, 0))], params=p)
    st, _, _ = orc.sim_step(sc, 20, precision="f64")
    np.testing.assert_allclose(st["vel"], 0.0, atol=1e-9)
    assert st["pos"][0, 1] - st["pos"][0, 0] == pytest.approx(0.1, abs=2e-3)


def test_mirror_symmetry(orc):
    """A scene mirrored in x stays mirrored (f64)."""
    p = dataclasses.replace(S.SimParams(), gravity=(0.0, 0.0, -9.81))
    sc = S.custom([dict(type="sphere", r=0.06, pos=(-0.1, 0.0, 0.3), vel=(0.5, 0, 0)),
                   dict(type="sphere", r=0.06, pos=(0.1, 0.0, 0.3), vel=(-0.5, 0, 0)),
                   dict(type="sphere", r=0.05, pos=(0.0, 0.0, 0.06))], params=p)
    st, _, _ = orc.sim_step(sc, 60, precision="f64")
    np.testing.assert_allclose(st["pos"][0, 0], -st["pos"][0, 1], atol=1e-12)
    np.testing.assert_allclose(st["pos"][2, 0], st["pos"][2, 1], atol=1e-12)
    assert abs(st["pos"][0, 2]) < 1e-12


def _rotmat(q):
    from scipy.spatial.transform import Rotation
    w, x, y, z = q
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def test_box_plane_corners_match_scipy_rotation(orc):
    """Box-plane contacts are the corners below the margin, in sign order,
    at positions given by an independent rotation (scipy)."""
    q = np.array([0.9, 0.2, -0.3, 0.25])
    q /= np.linalg.norm(q)
    h = np.array([0.04, 0.06, 0.08])
    sc = S.custom([dict(type="box", h=tuple(h), pos=(0.1, 0.2, 0.075), quat=tuple(q))])
    c = orc.contacts(sc, 0)
    R = _rotmat(sc.quat[:, 0].astype(np.float64))
    exp = []
    for k in range(8):
        s = np.array([1 if k & 1 else -1, 1 if k & 2 else -1, 1 if k & 4 else -1])
        w = R @ (s * h) + sc.pos[:, 0]
        if w[2] < sc.params.margin:
            exp.append(w)
    assert c["count"] == len(exp) > 0
    np.testing.assert_allclose(c["p"], np.array(exp), atol=2e-6)
    np.testing.assert_allclose(c["d"], np.array(exp)[:, 2], atol=2e-6)
    assert (c["b"] == -1).all() and (c["n"] == [0, 0, 1]).all()


def test_sphere_box_contact_distance(orc):
    """Sphere outside a rotated box: the signed distance is the distance from
    the sphere centre to the box (found by dense sampling of the box) minus r;
    the normal points from the box to the sphere."""
    q = np.array([0.8, 0.1, 0.5, -0.3])
    q /= np.linalg.norm(q)
    h = np.array([0.05, 0.03, 0.07])
    pb = np.array([0.0, 0.0, 1.0])
    ps = np.array([0.09, 0.02, 1.05])
    r = 0.04
    p = dataclasses.replace(S.SimParams(), plane=0, margin=0.05)
    sc = S.custom([dict(type="sphere", r=r, pos=tuple(ps)),
                   dict(type="box", h=tuple(h), pos=tuple(pb), quat=tuple(q))], params=p)
    c = orc.contacts(sc, 0)
    assert c["count"] == 1 and c["a"][0] == 0 and c["b"][0] == 1
    R = _rotmat(sc.quat[:, 1].astype(np.float64))
    g = np.linspace(-1, 1, 81)
    X, Y, Z = np.meshgrid(g * h[0], g * h[1], g * h[2], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) @ R.T + sc.pos[:, 1]
    dist = np.sqrt(((pts - sc.pos[:, 0]) ** 2).sum(1))
    k = dist.argmin()
    assert c["d"][0] == pytest.approx(dist[k] - r, abs=3e-4)
    nexp = (sc.pos[:, 0] - pts[k]) / dist[k]
    assert float(c["n"][0] @ nexp) > 0.99


def test_box_on_box_face_contacts(orc):
    """An axis-aligned box resting on a larger one: the four bottom corners
    of the top box lie within the lower box's top face, with n = +z (from
    the lower body B to the upper body A... here A = 0 is the upper box)."""
    p = dataclasses.replace(S.SimParams(), plane=0)
    gap = 0.004
    sc = S.custom([dict(type="box", h=(0.03, 0.03, 0.03), pos=(0.01, -0.02, 1.0 + 0.05 + 0.03 + gap)),
                   dict(type="box", h=(0.1, 0.1, 0.05), pos=(0.0, 0.0, 1.0))], params=p)
    c = orc.contacts(sc, 0)
    assert c["count"] == 4
    assert (c["a"] == 0).all() and (c["b"] == 1).all()
    np.testing.assert_allclose(c["n"], np.tile([0, 0, 1.0], (4, 1)), atol=1e-6)
    np.testing.assert_allclose(c["d"], gap, atol=1e-6)
    # sign order: corners (-,-,-), (+,-,-), (-,+,-), (+,+,-)
    np.testing.assert_allclose(c["p"][:, 0], [-0.02, 0.04, -0.02, 0.04], atol=1e-6)
    np.testing.assert_allclose(c["p"][:, 1], [-0.05, -0.05, 0.01, 0.01], atol=1e-6)


def test_canonical_order_and_overflow(orc):
    """Plane contacts come first by body, then pairs (i, j) in order; with a
    capacity of one contact per body the list is truncated and flagged."""
    bodies = [dict(type="sphere", r=0.05, pos=(0.0, 0.0, 0.05)),
              dict(type="sphere", r=0.05, pos=(0.095, 0.0, 0.05)),
              dict(type="sphere", r=0.05, pos=(0.19, 0.0, 0.05))]
    sc = S.custom(bodies)
    c = orc.contacts(sc, 0)
    assert list(zip(c["a"], c["b"])) == [(0, -1), (1, -1), (2, -1), (0, 1), (1, 2)]
    p = dataclasses.replace(S.SimParams(), max_contacts_per_body=1)
    sc2 = S.custom(bodies, params=p)
    _, flags, cc = orc.sim_step(sc2, 1)
    assert flags[0] & 1 and cc[0] == 3


def test_f32_tracks_f64_on_cfg1(orc):
    """The float step stays within float rounding of the double step over a
    short horizon of a contact-rich batch (no discrete contact decision
    flips in this window)."""
    sc = S.cfg1(4)
    s32, _, _ = orc.sim_step(sc, 5, precision="f32")
    s64, _, _ = orc.sim_step(sc, 5, precision="f64")
    for k in ("pos", "vel", "quat"):
        np.testing.assert_allclose(s32[k], s64[k], rtol=1e-4, atol=1e-5)


def test_box_corners_of_b_inside_a_flip_the_normal(orc):
    """Box-box, the second half of the test (B's corners inside A): a small
    box B (body 1), turned 30 degrees about A's up axis, sits sunk by `sink`
    into the top face of a tilted larger box A (body 0).  A's corners are all
    far outside B, so every contact is one of B's four bottom corners, in
    sign-bit order, with d = -sink and the normal pointing from B to A
    (minus A's up axis).  Geometry from an independent rotation (scipy)."""
    from scipy.spatial.transform import Rotation
    RA = Rotation.from_euler("xyz", [20.0, -10.0, 35.0], degrees=True)
    RB = RA * Rotation.from_euler("z", 30.0, degrees=True)
    hA = np.array([0.1, 0.12, 0.05])
    hB = np.array([0.03, 0.04, 0.035])
    sink = 0.004
    pA = np.array([0.0, 0.0, 1.0])
    pB = pA + RA.apply([0.01, -0.015, hA[2] + hB[2] - sink])

    def wxyz(r):
        x, y, z, w = r.as_quat()
        return (w, x, y, z)

    p = dataclasses.replace(S.SimParams(), plane=0)
    sc = S.custom([dict(type="box", h=tuple(hA), pos=tuple(pA), quat=wxyz(RA)),
                   dict(type="box", h=tuple(hB), pos=tuple(pB), quat=wxyz(RB))], params=p)
    c = orc.contacts(sc, 0)
    RBm = _rotmat(sc.quat[:, 1].astype(np.float64))
    RAm = _rotmat(sc.quat[:, 0].astype(np.float64))
    exp = []
    for k in range(4):   # bottom corners: sign bit 2 clear
        s = np.array([1 if k & 1 else -1, 1 if k & 2 else -1, -1])
        exp.append(RBm @ (s * hB) + sc.pos[:, 1].astype(np.float64))
    assert c["count"] == 4
    assert (c["a"] == 0).all() and (c["b"] == 1).all()
    np.testing.assert_allclose(c["p"], np.array(exp), atol=2e-6)
    np.testing.assert_allclose(c["d"], -sink, atol=2e-6)
    np.testing.assert_allclose(c["n"], np.tile(-RAm[:, 2], (4, 1)), atol=2e-6)
    # the same pair listed the other way round (the small box first) puts
    # the corners in the first half of the test, with the normal from the
    # large box to the small one: +A's up axis
    sc2 = S.custom([dict(type="box", h=tuple(hB), pos=tuple(pB), quat=wxyz(RB)),
                    dict(type="box", h=tuple(hA), pos=tuple(pA), quat=wxyz(RA))], params=p)
    c2 = orc.contacts(sc2, 0)
    assert c2["count"] == 4 and (c2["a"] == 0).all() and (c2["b"] == 1).all()
    np.testing.assert_allclose(c2["p"], c["p"], atol=0)
    np.testing.assert_allclose(c2["n"], -c["n"], atol=0)


@pytest.mark.parametrize("sphere_first", [True, False])
def test_sphere_centre_inside_box(orc, sphere_first):
    """A sphere whose centre lies inside a box: the contact uses the box face
    of least penetration, d = -(h_m - |l_m|) - r, the point on that face
    straight out from the centre, and the normal pointing from the box to
    the sphere (or its negative when the box is listed first).  Rotated box;
    geometry from an independent rotation (scipy)."""
    from scipy.spatial.transform import Rotation
    R = Rotation.from_euler("xyz", [15.0, 40.0, -25.0], degrees=True)
    x, y, z, w = R.as_quat()
    h = np.array([0.08, 0.05, 0.1])
    pb = np.array([0.2, -0.1, 1.0])
    l = np.array([0.02, -0.035, 0.03])   # penetrations h - |l| = 0.06, 0.015, 0.07: axis y, side -
    r = 0.02
    ps = pb + R.apply(l)
    p = dataclasses.replace(S.SimParams(), plane=0)
    sph = dict(type="sphere", r=r, pos=tuple(ps))
    box = dict(type="box", h=tuple(h), pos=tuple(pb), quat=(w, x, y, z))
    sc = S.custom([sph, box] if sphere_first else [box, sph], params=p)
    c = orc.contacts(sc, 0)
    assert c["count"] == 1 and c["a"][0] == 0 and c["b"][0] == 1
    Rm = _rotmat(sc.quat[:, 1 if sphere_first else 0].astype(np.float64))
    n_box_to_sphere = -Rm[:, 1]
    face_pt = Rm @ np.array([l[0], -h[1], l[2]]) + sc.pos[:, 1 if sphere_first else 0]
    assert c["d"][0] == pytest.approx(-(h[1] - abs(l[1])) - r, abs=2e-6)
    np.testing.assert_allclose(c["p"][0], face_pt, atol=2e-6)
    np.testing.assert_allclose(c["n"][0], n_box_to_sphere if sphere_first else -n_box_to_sphere, atol=2e-6)


def test_sphere_centre_inside_box_ties_go_to_the_lowest_axis(orc):
    """Equal penetrations along x and y (exact in float: an axis-aligned box
    and dyadic offsets): the lower axis, x, is chosen; a centre at the box
    centre ties all three axes and takes +x (the sign of a zero coordinate
    is +)."""
    p = dataclasses.replace(S.SimParams(), plane=0)
    for l, nexp, dexp in (((0.25, -0.25, 0.125), (1.0, 0.0, 0.0), -0.25 - 0.0625),
                          ((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), -0.5 - 0.0625)):
        sc = S.custom([dict(type="sphere", r=0.0625, pos=(l[0], l[1], 2.0 + l[2])),
                       dict(type="box", h=(0.5, 0.5, 0.5), pos=(0.0, 0.0, 2.0))], params=p)
        c = orc.contacts(sc, 0)
        assert c["count"] == 1
        np.testing.assert_array_equal(c["n"][0], nexp)
        assert c["d"][0] == dexp
        np.testing.assert_array_equal(c["p"][0], (0.5, l[1], 2.0 + l[2]))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 3e-5)])
def test_constant_force_closed_form(orc, prec, tol):
    """A constant force F held on a free body adds F / m to the acceleration:
    v_n = v0 + n h (g + F/m), x_n = x0 + n h v0 + h^2 (g + F/m) n (n+1) / 2.
    One sphere and one box (different masses) in the same environment, far
    apart."""
    sc = S.custom([dict(type="sphere", r=0.06, pos=(-5.0, 0.0, 50.0), vel=(0.5, 0.0, 1.0)),
                   dict(type="box", h=(0.03, 0.05, 0.08), pos=(5.0, 0.0, 50.0), vel=(0.0, -1.0, 2.0))])
    F = np.array([[0.3, -1.5], [-0.2, 0.7], [4.0, 0.25]])
    steps = 20
    st, _, cc = orc.sim_step(sc, steps, precision=prec, force=F)
    assert cc[0] == 0
    h = sc.params.dt / sc.params.substeps
    n = steps * sc.params.substeps
    g = np.array(sc.params.gravity)
    for b in range(2):
        m = 1.0 / float(np.float32(sc.inv_mass[b]))
        acc = g + F[:, b] / m if prec == "f64" else g + F[:, b].astype(np.float32) / m
        v0 = sc.vel[:, b].astype(np.float64)
        x0 = sc.pos[:, b].astype(np.float64)
        np.testing.assert_allclose(st["vel"][:, b], v0 + n * h * acc, rtol=tol, atol=tol)
        np.testing.assert_allclose(st["pos"][:, b], x0 + n * h * v0 + h * h * acc * n * (n + 1) / 2.0,
                                   rtol=tol, atol=tol * 50)


@pytest.mark.parametrize("speed,bounces", [(3.0, True), (0.4, False)])
def test_head_on_restitution(orc, speed, bounces):
    """Equal spheres overlapping by less than the slop, approaching head on
    along x with e = 0.5 (no gravity, no plane).  Faster than the 1 m/s
    threshold, the textbook outcome: they separate at e times the approach
    speed after one substep, momentum conserved, no spin.  Slower, the
    restitution target does not apply and they stop along the normal."""
    e = 0.5
    p = dataclasses.replace(S.SimParams(), gravity=(0.0, 0.0, 0.0), plane=0, restitution=e, substeps=1)
    r = 0.0625
    ov = 0.000244140625   # overlap 2^-12 < slop: no position bias
    x = r - ov / 2
    sc = S.custom([dict(type="sphere", r=r, pos=(-x, 0.0, 1.0), vel=(speed / 2, 0.0, 0.0)),
                   dict(type="sphere", r=r, pos=(x, 0.0, 1.0), vel=(-speed / 2, 0.0, 0.0))], params=p)
    s0 = {k: v.astype(np.float64) for k, v in sc.state().items()}
    st, _, cc = orc.sim_step(sc, 1, state=s0, precision="f64")
    assert cc[0] == 1
    v_rel = st["vel"][0, 1] - st["vel"][0, 0]   # separation speed along x
    assert v_rel == pytest.approx(e * speed if bounces else 0.0, abs=1e-12)
    assert st["vel"][0, 0] + st["vel"][0, 1] == pytest.approx(0.0, abs=1e-12)
    np.testing.assert_array_equal(st["angvel"], 0.0)
    np.testing.assert_array_equal(st["vel"][1:], 0.0)


def _body_omega(st, i=0):
    """Body-frame angular velocity R^T w (independent rotation: scipy)."""
    R = _rotmat(st["quat"][:, i].astype(np.float64))
    return R.T @ st["angvel"][:, i].astype(np.float64)


def _world_momentum(sc, st, i=0):
    """World angular momentum R I R^T w of body i (I from the scene's inverse inertia)."""
    R = _rotmat(st["quat"][:, i].astype(np.float64))
    I = np.diag(1.0 / sc.inv_inertia[:, i].astype(np.float64))
    return R @ I @ R.T @ st["angvel"][:, i].astype(np.float64)


def _spinning_box(w_body, gyro=1):
    p = dataclasses.replace(S.SimParams(), gravity=(0.0, 0.0, 0.0), plane=0, gyroscopic=gyro)
    # half extents 0.02, 0.05, 0.1: principal moments I0 > I1 > I2 (y intermediate)
    return S.custom([dict(type="box", h=(0.02, 0.05, 0.1), pos=(0.0, 0.0, 1.0), angvel=tuple(w_body))], params=p)


def test_gyroscopic_intermediate_axis_flips(orc):
    """Torque-free spin about the intermediate principal axis is unstable
    (the tennis-racket theorem): with the gyroscopic term the body-frame spin
    about y reverses within a few seconds while the world angular momentum
    stays nearly constant (implicit Euler dissipates slowly); without the
    term the angular velocity never changes."""
    sc = _spinning_box((0.01, 10.0, 0.01))
    I = 1.0 / sc.inv_inertia[:, 0].astype(np.float64)
    assert I[0] > I[1] > I[2]
    s0 = {k: v.astype(np.float64) for k, v in sc.state().items()}
    L0 = _world_momentum(sc, s0)
    st, seen_flip = s0, False
    for _ in range(60):                       # 60 x 10 steps = 2.5 s
        st, _, _ = orc.sim_step(sc, 10, state=st, precision="f64")
        wb = _body_omega(st)
        seen_flip |= wb[1] < -5.0
        L = _world_momentum(sc, st)
        assert np.linalg.norm(L - L0) < 0.02 * np.linalg.norm(L0)
    assert seen_flip
    off = _spinning_box((0.01, 10.0, 0.01), gyro=0)
    st_off, _, _ = orc.sim_step(off, 600, state={k: v.astype(np.float64) for k, v in off.state().items()},
                                precision="f64")
    np.testing.assert_allclose(st_off["angvel"][:, 0], (0.01, 10.0, 0.01), atol=1e-12)


@pytest.mark.parametrize("axis", [0, 2])
def test_gyroscopic_major_and_minor_axes_are_stable(orc, axis):
    """Spin about the axis of the largest or the smallest moment stays close
    to that axis in the body frame (both are stable)."""
    w = [0.01, 0.01, 0.01]
    w[axis] = 10.0
    sc = _spinning_box(w)
    st = {k: v.astype(np.float64) for k, v in sc.state().items()}
    for _ in range(30):
        st, _, _ = orc.sim_step(sc, 20, state=st, precision="f64")
        wb = _body_omega(st)
        assert wb[axis] > 9.8
        assert np.abs(np.delete(wb, axis)).max() < 0.5


def test_gyroscopic_step_is_first_order_euler_equations(orc):
    """One substep changes the body-frame angular velocity by
    -h I^-1 (w x I w) to first order in h (the implicit step and the explicit
    one differ by O(h^2 |w|^2))."""
    w = np.array([3.0, -2.0, 5.0])
    sc = _spinning_box(tuple(w))
    sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, substeps=1, dt=1e-4))
    st, _, _ = orc.sim_step(sc, 1, state={k: v.astype(np.float64) for k, v in sc.state().items()},
                            precision="f64")
    I = 1.0 / sc.inv_inertia[:, 0].astype(np.float64)
    h = 1e-4
    explicit = -h * np.cross(w, I * w) / I
    got = st["angvel"][:, 0] - w        # identity orientation at the start: body = world
    np.testing.assert_allclose(got, explicit, rtol=5e-3, atol=1e-12)
    assert np.abs(explicit).max() > 1e-3


def test_gyroscopic_step_is_one_newton_step_of_implicit_euler(orc):
    """A large step (h |w| ~ 0.1), where the implicit and explicit updates
    differ clearly: the change of the body-frame angular velocity is the
    Newton step D = -J^-1 f of f(x) = I (x - w) + h x x I x at x = w, with
    J = I + h (skew(w) I - skew(I w)) assembled from skew matrices and
    solved by numpy."""
    w = np.array([4.0, -6.0, 9.0])
    sc = _spinning_box(tuple(w))
    h = 0.01
    sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, substeps=1, dt=h))
    st, _, _ = orc.sim_step(sc, 1, state={k: v.astype(np.float64) for k, v in sc.state().items()},
                            precision="f64")
    I = np.diag(1.0 / sc.inv_inertia[:, 0].astype(np.float64))

    def skew(a):
        return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])

    f = h * np.cross(w, I @ w)
    J = I + h * (skew(w) @ I - skew(I @ w))
    D = -np.linalg.solve(J, f)
    np.testing.assert_allclose(st["angvel"][:, 0], w + D, rtol=1e-12, atol=1e-12)
    explicit = -h * np.linalg.solve(I, np.cross(w, I @ w))
    assert np.abs(D - explicit).max() > 0.05 * np.abs(explicit).max()


def _crossed_beams(gap, lower_first=True, yaw=0.0):
    """Two square beams turned 45 degrees about their long axes (diamond
    cross-sections): A along x with its top edge at z = 1 + hA sqrt 2,
    B along y (turned `yaw` about z) with its bottom edge `gap` above it.
    The two edges cross; no corner of either beam is near the other."""
    from scipy.spatial.transform import Rotation
    hA, hB = 0.03, 0.02
    RA = Rotation.from_euler("x", 45.0, degrees=True)
    RB = Rotation.from_euler("z", yaw, degrees=True) * Rotation.from_euler("y", 45.0, degrees=True)

    def wxyz(r):
        x, y, z, w = r.as_quat()
        return (w, x, y, z)

    zA = 1.0
    zB = zA + hA * math.sqrt(2) + gap + hB * math.sqrt(2)
    A = dict(type="box", h=(0.3, hA, hA), pos=(0.0, 0.0, zA), quat=wxyz(RA))
    B = dict(type="box", h=(hB, 0.3, hB), pos=(0.0, 0.0, zB), quat=wxyz(RB))
    p = dataclasses.replace(S.SimParams(), plane=0, edge_contacts=1)
    return S.custom([A, B] if lower_first else [B, A], params=p), zA + hA * math.sqrt(2), zB - hB * math.sqrt(2)


@pytest.mark.parametrize("gap", [0.005, -0.003])
def test_box_edges_crossing_give_one_edge_contact(orc, gap):
    """Crossed diamond beams touch edge to edge: the only contact is the
    edge-edge one, with the normal along a_x x b_y = z pointing from B to A
    (down when A is the lower beam), the distance equal to the gap between
    the edges (speculative when positive, penetration when negative) and
    the point midway between them."""
    sc, top, bottom = _crossed_beams(gap)
    c = orc.contacts(sc, 0)
    assert c["count"] == 1 and c["a"][0] == 0 and c["b"][0] == 1
    np.testing.assert_allclose(c["n"][0], (0.0, 0.0, -1.0), atol=1e-6)
    assert c["d"][0] == pytest.approx(gap, abs=2e-6)
    np.testing.assert_allclose(c["p"][0], (0.0, 0.0, 0.5 * (top + bottom)), atol=2e-6)
    # listed the other way round the normal flips (still from B to A)
    sc2, _, _ = _crossed_beams(gap, lower_first=False)
    c2 = orc.contacts(sc2, 0)
    assert c2["count"] == 1
    np.testing.assert_allclose(c2["n"][0], (0.0, 0.0, 1.0), atol=1e-6)
    np.testing.assert_allclose(c2["p"][0], c["p"][0], atol=2e-6)
    # beyond the margin: no contact
    sc3, _, _ = _crossed_beams(sc.params.margin + 0.004)
    assert orc.contacts(sc3, 0)["count"] == 0
    # without edge contacts the corner tests alone miss the crossing
    sc4 = dataclasses.replace(sc, params=dataclasses.replace(sc.params, edge_contacts=0))
    assert orc.contacts(sc4, 0)["count"] == 0


def test_box_edge_contact_geometry_at_an_angle(orc):
    """Beams crossing at 60 degrees (B turned 30 degrees about z): the normal
    is perpendicular to both edge directions, the contact distance is the
    distance between the two edge lines (independent closed form: the
    projection of the offset of two points on the lines onto their common
    normal), and the point is the midpoint of the common perpendicular."""
    from scipy.spatial.transform import Rotation
    sc, _, _ = _crossed_beams(0.004, yaw=30.0)
    c = orc.contacts(sc, 0)
    assert c["count"] == 1
    RA = _rotmat(sc.quat[:, 0].astype(np.float64))
    RB = _rotmat(sc.quat[:, 1].astype(np.float64))
    ea, eb = RA[:, 0], RB[:, 1]
    n = c["n"][0].astype(np.float64)
    assert abs(n @ ea) < 1e-6 and abs(n @ eb) < 1e-6
    # points on the two supporting edges (A's top edge, B's bottom edge)
    hA, hB = sc.shape_dims[:, 0].astype(np.float64), sc.shape_dims[:, 1].astype(np.float64)
    pA, pB = sc.pos[:, 0].astype(np.float64), sc.pos[:, 1].astype(np.float64)
    cand_a = [pA + RA @ np.array([0.0, sy * hA[1], sz * hA[2]]) for sy in (-1, 1) for sz in (-1, 1)]
    cand_b = [pB + RB @ np.array([sx * hB[0], 0.0, sz * hB[2]]) for sx in (-1, 1) for sz in (-1, 1)]
    qa = max(cand_a, key=lambda v: v[2])
    qb = min(cand_b, key=lambda v: v[2])
    m = np.cross(ea, eb)
    m /= np.linalg.norm(m)
    dist = abs((qb - qa) @ m)
    assert c["d"][0] == pytest.approx(dist, abs=2e-6)
    # the common perpendicular's midpoint
    A_ = np.array([[ea @ ea, -(ea @ eb)], [ea @ eb, -(eb @ eb)]])
    s, t = np.linalg.solve(A_, [(qb - qa) @ ea, (qb - qa) @ eb])
    mid = 0.5 * ((qa + s * ea) + (qb + t * eb))
    np.testing.assert_allclose(c["p"][0], mid, atol=2e-6)


def test_box_edge_contact_clamped_to_the_edge_end(orc):
    """B's edge passes 1 mm beyond the end of A's edge: A's end corner is
    within the margin of B (the corner test's contact, first) and the edges
    still give the greatest separation, so an edge contact follows whose
    point on A's edge is clamped to its end (x = 0.3) while B's stays where
    the lines cross (x = 0.301): the contact is midway between the two."""
    sc, top, bottom = _crossed_beams(0.004)
    sc.pos[0, 1] = 0.301
    c = orc.contacts(sc, 0)
    assert c["count"] == 2
    np.testing.assert_allclose(c["p"][0], (0.3, 0.0, top), atol=2e-6)          # A's corner in B
    np.testing.assert_allclose(c["p"][1], (0.5 * (0.3 + 0.301), 0.0, 0.5 * (top + bottom)), atol=2e-6)
    np.testing.assert_allclose(c["n"][1], (0.0, 0.0, -1.0), atol=1e-6)
    assert c["d"][1] == pytest.approx(0.004, abs=2e-6)
