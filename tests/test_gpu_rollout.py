"""RL rollout with the inter-trajectory schedule (vuda_rollout_run): two
groups of trajectories, each looping sim -> render -> policy (a randomly
initialised torch MLP reading the group's frame), with one group's sim
beside the other group's render and policy.  The schedule does not change
the results, and the physics and frames match the oracle stepped with the
same forces."""
import numpy as np
import pytest

from paper_2605_01352_b300 import scene as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_01352_b300 import build
    build.build()
    from paper_2605_01352_b300 import vuda
    return vuda


def _groups(make, n):
    return make(n, 0), make(n, n)


def _run(V, scenes, steps, mode, hidden=256, record=False, graph=False):
    import torch
    from paper_2605_01352_b300.policy import MLPPolicy
    envs = [V.Env(sc) for sc in scenes]
    rings = [[e.alloc_frame(), e.alloc_frame()] for e in envs]
    forces = [torch.zeros((3, e.B), dtype=torch.float32, device="cuda") for e in envs]
    pols = [MLPPolicy(envs[g], sc, hidden, seed=7 + g) for g, sc in enumerate(scenes)]
    if graph:
        for g in range(2):
            pols[g].capture(rings[g], forces[g], torch.cuda.Stream())
            forces[g].zero_()                 # the capture's warm-up wrote forces
    hist = [[f.clone()] for f in forces]
    order = []

    def policy(group, step, slot, stream):
        if graph:
            pols[group].act_captured(slot, stream)
        with torch.cuda.stream(stream):
            if not graph:
                pols[group].act(rings[group][slot], forces[group])
            if record:
                hist[group].append(forces[group].clone())
        order.append((group, step, slot))

    if mode == "streams":
        envs[0].coschedule(V.COSCHED_STREAMS)
    elif mode == "green":
        envs[0].coschedule(V.COSCHED_GREEN)
    V.rollout_run(envs[0], envs[1], steps, rings[0], rings[1], forces[0], forces[1], policy,
                  stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    out = dict(state=[e.get_state() for e in envs],
               frames=[[{k: v.cpu().numpy().copy() for k, v in f.items()} for f in r] for r in rings],
               forces=[f.cpu().numpy() for f in forces], order=order,
               hist=[[h.cpu().numpy() for h in hh] for hh in hist],
               pose=[e.get_pose((steps - 1) & 1) for e in envs])
    for e in envs:
        e.close()
    return out


@pytest.mark.parametrize("mode,graph", [("streams", False), ("green", False), ("streams", True), ("green", True)])
def test_rollout_schedule_does_not_change_results(V, mode, graph):
    """Co-scheduled rollouts (shared SMs, or disjoint green partitions with
    the policy on a stream of its own) equal the time-sliced rollout bit for
    bit: states, both frames of both groups, and the forces -- also with the
    policy replayed from CUDA graphs captured per frame slot."""
    scenes = _groups(lambda n, b: S.cfg2(n, env_base=b), 24)
    ref = _run(V, scenes, 5, "serialized")
    got = _run(V, scenes, 5, mode, graph=graph)
    assert ref["order"] == got["order"] == [(g, k, k & 1) for k in range(5) for g in (0, 1)]
    for g in range(2):
        for k in ref["state"][g]:
            np.testing.assert_array_equal(got["state"][g][k], ref["state"][g][k], err_msg="group %d %s" % (g, k))
        for a, b in zip(got["frames"][g], ref["frames"][g]):
            for k in a:
                np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(got["forces"][g], ref["forces"][g])
    assert np.abs(ref["forces"][0]).max() > 0.01          # the policy acts


@pytest.mark.parametrize("hidden", [256, 4096])
def test_rollout_matches_oracle_with_the_policy_forces(V, orc, hidden):
    """Each group stepped by the oracle with the forces the policy wrote
    (step k uses the forces written after step k - 1; zeros first) matches
    the GPU state within the physics tolerance, and the last frames are the
    oracle's render of the GPU's last pose slot."""
    scenes = _groups(lambda n, b: S.generate(n, 8, S.config_seed(1), kinds="mixed", res=64, substeps=4,
                                             env_base=b), 3)
    steps = 6
    got = _run(V, scenes, steps, "streams", hidden=hidden, record=True)
    for g, sc in enumerate(scenes):
        st = sc.state()
        for k in range(steps):
            st, _, _ = orc.sim_step(sc, 1, state=st, force=got["hist"][g][k])
        for key in ("pos", "vel", "quat", "angvel"):
            np.testing.assert_allclose(got["state"][g][key], st[key], rtol=1e-5, atol=1e-5,
                                       err_msg="group %d %s" % (g, key))
        pos, quat = got["pose"][g]
        o_rgb, o_dep, o_tid, _ = orc.render(sc, pos, quat)
        f = got["frames"][g][(steps - 1) & 1]
        np.testing.assert_array_equal(f["triid"].view(np.uint32), o_tid)
        np.testing.assert_allclose(f["depth"], o_dep, rtol=1e-6, atol=0)
        assert np.abs(f["rgb"].astype(int) - o_rgb.astype(int)).max() <= 1


def test_rollout_rejects_bad_arguments(V):
    import torch
    a, b = V.Env(S.cfg2(4)), V.Env(S.cfg2(4, env_base=4))
    ra, rb = [a.alloc_frame(), a.alloc_frame()], [b.alloc_frame(), b.alloc_frame()]
    fa = torch.zeros((3, a.B), device="cuda")
    fb = torch.zeros((3, b.B), device="cuda")
    noop = lambda g, k, s, st: None
    with pytest.raises(V.VudaError):
        V.rollout_run(a, a, 2, ra, ra, fa, fa, noop)            # one batch for both groups
    b.coschedule(V.COSCHED_STREAMS)
    with pytest.raises(V.VudaError):
        V.rollout_run(a, b, 2, ra, rb, fa, fb, noop)            # group 1 co-scheduled itself
    b.coschedule_reset()
    a.coschedule(V.COSCHED_SHARED)
    with pytest.raises(V.VudaError) as ex:
        V.rollout_run(a, b, 2, ra, rb, fa, fb, noop)
    assert ex.value.status == V.ERR_UNSUPPORTED
    a.coschedule_reset()

    def boom(g, k, s, st):
        raise RuntimeError("policy failed")
    with pytest.raises(RuntimeError):
        V.rollout_run(a, b, 2, ra, rb, fa, fb, boom)
    a.close()
    b.close()


def test_observe_pools_the_frame(V, orc):
    """vuda_observe: per camera and 16 x 16 cell, the mean depth times the
    scale and the mean luminance, against the oracle's pooling of the frame
    read back (square and non-square cameras); bad arguments are refused."""
    import torch
    for res, height in ((64, None), (64, 32)):
        sc = S.generate(3, 6, 41, kinds="mixed", res=res, height=height, cams_per_env=2)
        env = V.Env(sc)
        fr = env.alloc_frame()
        env.render(fr, pose_slot=-1)
        out = torch.zeros((3, 2 * 2 * 16 * 16), dtype=torch.float32, device="cuda")
        env.observe(fr, 16, 0.25, out)
        torch.cuda.synchronize()
        want = orc.observe(sc, fr["rgb"].cpu().numpy(), fr["depth"].cpu().numpy(), 16, 0.25)
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-5, atol=1e-6)
        assert np.abs(want[:, 512:]).max() > 0.05        # the frame is not blank
        with pytest.raises(V.VudaError):
            env.observe(fr, 48, 0.25, out)      # 64 is not divisible by 48
        with pytest.raises(V.VudaError):
            env.observe(fr, 0, 0.25, out)
        env.close()
