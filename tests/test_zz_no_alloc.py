"""The allocation-free physics entry point (vuda_sim_step_noalloc) against
the regular one, for callers that cannot allocate device memory.

Runs last (file name) so that a failure here stops a -x run only after every
other test.  Both paths are forced to keep every contact in the spill area
(a shared-memory budget too small for any contact record), so the fixed
scratch array is exercised on every substep."""
import dataclasses

import numpy as np
import pytest

from paper_2605_01352_b300 import scene as S

pytestmark = pytest.mark.gpu


def _dev_arrays(torch, sc):
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dict(body_off=f(sc.body_off.astype(np.int32)), pos=f(sc.pos.astype(np.float32)),
                quat=f(sc.quat.astype(np.float32)), vel=f(sc.vel.astype(np.float32)),
                angvel=f(sc.angvel.astype(np.float32)), shape_type=f(sc.shape_type.astype(np.uint8)),
                shape_dims=f(sc.shape_dims.astype(np.float32)), inv_mass=f(sc.inv_mass.astype(np.float32)),
                inv_inertia=f(sc.inv_inertia.astype(np.float32)),
                pose=torch.zeros((7, sc.num_bodies), dtype=torch.float32, device="cuda"),
                flags=torch.zeros(sc.num_envs, dtype=torch.int32, device="cuda"),
                ncontacts=torch.zeros(sc.num_envs, dtype=torch.int32, device="cuda"))


def test_noalloc_step_matches_regular_step(orc):
    import torch
    assert torch.cuda.is_available()
    from paper_2605_01352_b300 import build
    build.build()
    from paper_2605_01352_b300 import vuda as V
    sc = S.cfg2(16)
    st, _, _ = orc.sim_step(sc, 60)   # settled piles: plenty of contacts
    sc = dataclasses.replace(sc, **{k: st[k] for k in ("pos", "quat", "vel", "angvel")})
    env = V.Env(sc, phys_smem_bytes=1024)
    arr = _dev_arrays(torch, sc)
    nmax = int(np.diff(sc.body_off).max())
    for call in range(2):   # two calls in a row: the second reuses the scratch as left by the first
        env.sim_step(3)
        V.sim_step_noalloc(arr, sc.params, 3, nmax, smem_per_env=1024)
        torch.cuda.synchronize()
        g = env.get_state()
        for k in ("pos", "quat", "vel", "angvel"):
            np.testing.assert_allclose(arr[k].cpu().numpy(), g[k], rtol=1e-5, atol=1e-5, err_msg="call %d %s" % (call, k))
        pos, quat = env.get_pose((env.info().steps_enqueued - 1) & 1)
        np.testing.assert_allclose(arr["pose"][:3].cpu().numpy(), pos, rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(arr["pose"][3:].cpu().numpy(), quat, rtol=1e-5, atol=1e-5)
        np.testing.assert_array_equal(arr["ncontacts"].cpu().numpy(), env.contact_counts())
        assert env.contact_counts().min() > 0
    env.close()


def test_noalloc_rejects_batches_beyond_the_scratch():
    """Batches whose scratch would not fit the fixed array are refused on the
    host before anything launches: through the spill records (many bodies)
    and through the per-environment offsets alone (many environments of a
    few bodies each)."""
    import torch
    assert torch.cuda.is_available()
    from paper_2605_01352_b300 import build
    build.build()
    from paper_2605_01352_b300 import vuda as V
    sc = S.cfg1(2)
    arr = _dev_arrays(torch, sc)
    # claim far more bodies than the fixed scratch can hold
    arr_big = dict(arr)
    arr_big["inv_mass"] = torch.zeros(4_000_000, device="cuda")
    with pytest.raises(V.VudaError) as ex:
        V.sim_step_noalloc(arr_big, sc.params, 1, 8)
    assert ex.value.status == V.ERR_INVALID
    assert "scratch" in str(ex.value)
    # 2.2 M environments of no bodies over 8 bodies in all: the records need
    # 16 x 8 x 36 words, the offsets 2 (E + 1) > 4 M words on their own
    E = 2_200_000
    arr_many = dict(arr)
    arr_many["body_off"] = torch.full((E + 1,), 0, dtype=torch.int32, device="cuda")
    arr_many["body_off"][-1] = 8
    with pytest.raises(V.VudaError) as ex:
        V.sim_step_noalloc(arr_many, sc.params, 1, 8)
    assert ex.value.status == V.ERR_INVALID
    assert "scratch" in str(ex.value)
    # the same batch shape below the limit (1.5 M environments) is accepted
    E = 1_500_000
    arr_ok = dict(arr)
    arr_ok["body_off"] = torch.full((E + 1,), 0, dtype=torch.int32, device="cuda")
    arr_ok["body_off"][-1] = 8
    arr_ok["flags"] = torch.zeros(E, dtype=torch.int32, device="cuda")
    arr_ok["ncontacts"] = torch.zeros(E, dtype=torch.int32, device="cuda")
    V.sim_step_noalloc(arr_ok, sc.params, 1, 8)
    torch.cuda.synchronize()
    assert int(arr_ok["flags"].abs().sum()) == 0
