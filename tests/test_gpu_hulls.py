"""Hull contacts (the hull_contacts option) on the GPU against the oracle:
the same 1e-5 physics bar as the other parity tests, through a horizon of
steps, with identical contact counts."""
import dataclasses
import math

import numpy as np
import pytest

from paper_2605_01352_b300 import scene as S
from test_gpu_parity import _physics_horizon

pytestmark = pytest.mark.gpu

N111 = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_01352_b300 import build
    build.build()
    from paper_2605_01352_b300 import vuda
    return vuda


def _wxyz_taking(u, v):
    from scipy.spatial.transform import Rotation
    u = np.asarray(u, float) / np.linalg.norm(u)
    v = np.asarray(v, float) / np.linalg.norm(v)
    ax = np.cross(u, v)
    s = np.linalg.norm(ax)
    if s < 1e-12:
        ax = np.cross(u, [1.0, 0.0, 0.0] if abs(u[0]) < 0.9 else [0.0, 1.0, 0.0])
        s = np.linalg.norm(ax)
    x, y, z, w = Rotation.from_rotvec(ax / s * math.atan2(np.linalg.norm(np.cross(u, v)), float(np.dot(u, v)))).as_quat()
    return (w, x, y, z)


def _hull_scene(envs=3):
    """Octahedra face down on the ground and stacked with their faces turned
    60 degrees, a sphere on a hull face, a box on a hull, a hull face down on
    a box, and a random 14-vertex hull tumbling onto another."""
    V8, T8 = S.octahedron()
    rng = np.random.default_rng(5)
    P = rng.normal(size=(14, 3))
    Vr, Tr = S.hull_from_points(P / np.linalg.norm(P, axis=1, keepdims=True))
    r = 0.1
    z0 = r / math.sqrt(3.0)
    up, down = _wxyz_taking(N111, (0, 0, 1)), _wxyz_taking(N111, (0, 0, -1))
    oct8 = (V8, T8)
    B = []
    B.append(dict(type="hull", r=r, mesh=oct8, pos=(-1.0, 0.0, z0 + 0.01), quat=down))
    B.append(dict(type="hull", r=r, mesh=oct8, pos=(-0.5, 0.0, z0), quat=up))
    B.append(dict(type="hull", r=r, mesh=oct8, pos=(-0.5, 0.0, 3 * z0 + 0.008), quat=down))
    B.append(dict(type="hull", r=r, mesh=oct8, pos=(0.0, 0.0, z0), quat=up))
    B.append(dict(type="sphere", r=0.04, pos=(0.0, 0.0, 2 * z0 + 0.045)))
    B.append(dict(type="hull", r=r, mesh=oct8, pos=(0.5, 0.0, z0), quat=up))
    B.append(dict(type="box", h=(0.03, 0.03, 0.02), pos=(0.5, 0.0, 2 * z0 + 0.025), quat=(0.96, 0.0, 0.0, 0.28)))
    B.append(dict(type="box", h=(0.15, 0.15, 0.03), pos=(1.0, 0.0, 0.03)))
    B.append(dict(type="hull", r=r, mesh=oct8, pos=(1.0, 0.02, 0.06 + z0 + 0.005), quat=down))
    B.append(dict(type="hull", r=0.08, mesh=(Vr, Tr), pos=(0.0, 0.6, 0.08)))
    B.append(dict(type="hull", r=0.07, mesh=(Vr, Tr), pos=(0.03, 0.62, 0.26), angvel=(2.0, -1.0, 0.5)))
    p = dataclasses.replace(S.SimParams(), hull_contacts=1)
    return S.custom(B, envs=envs, params=p)


@pytest.mark.parametrize("persistent", [False, True])
def test_hull_scenes_match_oracle(V, orc, persistent):
    sc = _hull_scene()
    c = orc.contacts(sc, 0)
    pairs = set(zip(c["a"].tolist(), c["b"].tolist()))
    assert {(1, 2), (3, 4), (5, 6), (7, 8)} <= pairs   # stacked hulls, sphere on hull, box on hull, hull on box
    _physics_horizon(V, orc, sc, steps=10, persistent=persistent)


def _settled(orc, sc, steps):
    st, _, _ = orc.sim_step(sc, steps)
    return dataclasses.replace(sc, **{k: st[k] for k in ("pos", "quat", "vel", "angvel")})


@pytest.mark.parametrize("persistent", [False, True])
def test_hull_piles_match_oracle(V, orc, persistent):
    """Piles of spheres, boxes and small hulls (8-48 faces) after settling."""
    sc = S.generate(12, 18, S.config_seed(3) ^ 0x77, kinds="mixed_hulls", hull_tris=(8, 48), n_hull_meshes=8)
    sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, hull_contacts=1))
    sc = _settled(orc, sc, 120)
    assert orc.contacts(sc, 0)["count"] > 0
    _physics_horizon(V, orc, sc, steps=10, persistent=persistent)


def test_hulls_with_many_faces_per_lane(V, orc):
    """Hulls of 80-160 faces and 42-82 vertices: a warp's lanes take several
    faces and vertices each, and the face searches reduce across them."""
    sc = S.generate(4, 8, S.config_seed(3) ^ 0x99, kinds="hulls", hull_tris=(80, 160), n_hull_meshes=4)
    sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, hull_contacts=1))
    sc = _settled(orc, sc, 120)
    _physics_horizon(V, orc, sc, steps=6)


def test_hull_contacts_off_keep_the_sphere_proxies(V, orc):
    """The same hull scene with the option off is the sphere-proxy physics."""
    sc = _hull_scene(envs=2)
    sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, hull_contacts=0))
    _physics_horizon(V, orc, sc, steps=5)


@pytest.mark.parametrize("persistent", [False, True])
def test_hull_and_edge_contacts_together(V, orc, persistent):
    """Both optional contact tests (and the gyroscopic term) in one batch:
    the kernel variant compiled with the edge and the hull paths."""
    sc = S.generate(8, 15, S.config_seed(3) ^ 0x55, kinds="mixed_hulls", hull_tris=(8, 40), n_hull_meshes=6)
    sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, hull_contacts=1, edge_contacts=1,
                                                            gyroscopic=1))
    sc = _settled(orc, sc, 120)
    _physics_horizon(V, orc, sc, steps=8, persistent=persistent)


@pytest.mark.parametrize("persistent", [False, True])
def test_hulls_in_large_environments(V, orc, persistent):
    """Environments of 80 and 100 bodies beside one of 12 (the persistent
    launch runs the large ones on the 512-thread size class): the hull pass
    with sixteen warps and several candidate rounds per substep."""
    sc = S.generate(3, np.array([80, 12, 100]), S.config_seed(3) ^ 0x33, kinds="mixed_hulls", hull_tris=(8, 40),
                    n_hull_meshes=6)
    sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, hull_contacts=1))
    sc = _settled(orc, sc, 120)
    assert orc.contacts(sc, 2)["count"] > 300
    _physics_horizon(V, orc, sc, steps=6, persistent=persistent)
