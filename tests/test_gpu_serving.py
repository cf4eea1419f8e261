"""Serving loop: continuous batching of step+render requests from several
jobs, admission by HBM budget, cancellation.  A job's results are the same
alone and in a mix (bit for bit), and match the oracle."""
import random
import time

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


def _jobs():
    # E's 800 x 660 camera has more tiles than the tiled path holds: it
    # renders through the band work list beside the others' tiled work lists
    return {"A": S.cfg2(8), "B": S.cfg1(6), "C": S.cfg4(5), "D": S.cfg2(4, env_base=100),
            "E": S.generate(2, np.array([5, 7]), 77, kinds="mixed", res=np.array([800, 64]),
                            height=np.array([660, 48]), substeps=4)}


def _alone(V, sc, n):
    srv = V.Server()
    j = srv.add_job(sc)
    for _ in range(n):
        srv.submit(j)
    res = srv.wait_all(n)
    assert all(r["status"] == 0 for r in res)
    st = srv.job_env(j).get_state()
    fr = srv.read_frame(j)
    srv.close()
    return st, fr


def test_job_results_are_the_same_alone_and_in_a_mix(V, orc):
    jobs = _jobs()
    counts = {"A": 5, "B": 7, "C": 4, "D": 6, "E": 3}
    srv = V.Server(max_inflight=2)
    ids = {k: srv.add_job(sc) for k, sc in jobs.items()}
    order = [k for k, n in counts.items() for _ in range(n)]
    random.Random(4).shuffle(order)
    # two waves submitted back to back: requests arriving while a launch is on
    # the GPU are batched into the next one
    for k in order[: len(order) // 2]:
        srv.submit(ids[k])
    time.sleep(0.003)
    for k in order[len(order) // 2:]:
        srv.submit(ids[k])
    res = srv.wait_all(sum(counts.values()))
    assert all(r["status"] == 0 for r in res)
    # requests of a job complete in order, with consecutive step indices
    for k, jid in ids.items():
        steps = [r["step"] for r in res if r["job"] == jid]
        assert steps == list(range(counts[k]))
    st = srv.stats()
    assert st["requests_done"] == sum(counts.values())
    assert st["max_batch"] >= 2          # requests of several jobs shared a launch
    mixed = {k: (srv.job_env(ids[k]).get_state(), srv.read_frame(ids[k])) for k in jobs}
    # the pose slot each job's last frame was rendered from
    poses = {k: srv.job_env(ids[k]).get_pose((counts[k] - 1) & 1) for k in jobs}
    paths = {k: srv.job_env(ids[k]).info().render_path for k in jobs}
    assert paths == {"A": V.RENDER_TILED, "B": V.RENDER_TILED, "C": V.RENDER_TILED, "D": V.RENDER_TILED,
                     "E": V.RENDER_BAND}
    srv.close()
    for k in ("A", "C", "E"):
        st_a, fr_a = _alone(V, jobs[k], counts[k])
        st_m, fr_m = mixed[k]
        for f in st_a:
            np.testing.assert_array_equal(st_a[f], st_m[f])
        for x, y in zip(fr_a, fr_m):
            np.testing.assert_array_equal(x, y)
    # and the jobs of both render paths match the oracle: the state within
    # the physics tolerance, the frame against the oracle's render of the
    # pose slot it was rendered from
    for k in ("A", "E"):
        sc = jobs[k]
        so, _, _ = orc.sim_step(sc, counts[k])
        for f in ("pos", "vel", "quat", "angvel"):
            np.testing.assert_allclose(mixed[k][0][f], so[f], rtol=1e-5, atol=1e-5)
        o_rgb, o_dep, o_tid, _ = orc.render(sc, *poses[k])
        np.testing.assert_array_equal(mixed[k][1][2], o_tid)
        np.testing.assert_allclose(mixed[k][1][1], o_dep, rtol=1e-6)
        assert np.abs(mixed[k][1][0].astype(int) - o_rgb.astype(int)).max() <= 1


def test_admission_waits_for_budget(V):
    """With room for one job at a time, the second job is admitted only after
    the first is removed; its requests then complete."""
    a, b = S.cfg1(4), S.cfg1(4, )
    est = V.estimate_bytes(a)
    srv = V.Server(hbm_budget_bytes=int(est * 1.5))
    ja = srv.add_job(a)
    jb = srv.add_job(b)
    for _ in range(2):
        srv.submit(ja)
        srv.submit(jb)
    got = srv.wait_all(2)
    assert {r["job"] for r in got} == {ja}
    st = srv.stats()
    assert st["admitted"] == 1 and st["waiting"] == 1
    time.sleep(0.05)
    assert srv.poll() == []                # b's requests are still waiting for admission
    srv.remove_job(ja)
    got = srv.wait_all(2)
    assert {r["job"] for r in got} == {jb} and all(r["status"] == 0 for r in got)
    srv.close()


def test_errors_and_cancellation(V):
    sc = S.cfg1(2)
    srv = V.Server(hbm_budget_bytes=1024)
    with pytest.raises(V.VudaError) as ex:
        srv.add_job(sc)                     # larger than the whole budget
    assert ex.value.status == V.ERR_OOM
    with pytest.raises(V.VudaError) as ex:
        srv.submit(12345)
    assert ex.value.status == V.ERR_INVALID
    srv.close()
    srv = V.Server(hbm_budget_bytes=int(V.estimate_bytes(sc) * 1.5))
    j1 = srv.add_job(sc)
    j2 = srv.add_job(sc)                    # waits for admission
    r = [srv.submit(j2) for _ in range(3)]
    srv.remove_job(j2)                      # its queued requests are cancelled
    got = srv.wait_all(3)
    assert sorted(x["req_id"] for x in got) == sorted(r)
    assert all(x["status"] == V.ERR_BUSY for x in got)
    srv.submit(j1)
    assert srv.wait_all(1)[0]["status"] == 0
    srv.close()


def _faulted_run(V, monkeypatch, env, jobs, counts, cancel=None):
    """Jobs run together under an injected host-side fault (environment
    variables read when the server is created); returns each job's
    (statuses, state, frame) and the server's job ids."""
    for k, v in env.items():
        monkeypatch.setenv(k, str(v))
    srv = V.Server(max_inflight=2)
    for k in env:
        monkeypatch.delenv(k)
    ids = {k: srv.add_job(sc) for k, sc in jobs.items()}
    assert sorted(ids.values()) == list(range(1, len(jobs) + 1))
    order = [k for k, n in counts.items() for _ in range(n)]
    random.Random(8).shuffle(order)
    reqs = {k: [] for k in jobs}
    refused = {k: 0 for k in jobs}
    for k in order:
        try:
            reqs[k].append(srv.submit(ids[k]))
        except V.VudaError as ex:         # the job already failed its admission
            assert ex.status == V.ERR_INVALID
            refused[k] += 1
    if cancel:
        srv.remove_job(ids[cancel])       # launched requests finish, queued ones are cancelled
    total = sum(len(r) for r in reqs.values())
    res = srv.wait_all(total)
    by_job = {k: sorted((r for r in res if r["job"] == ids[k]), key=lambda r: r["req_id"]) for k in jobs}
    out = {}
    for k in jobs:
        st = [r["status"] for r in by_job[k]] + ["refused"] * refused[k]
        if st and all(x == 0 for x in st):
            out[k] = (st, srv.job_env(ids[k]).get_state(), srv.read_frame(ids[k]))
        else:
            out[k] = (st, None, None)
    srv.close()
    return out


def _same_as_alone(V, sc, n, got):
    st_a, fr_a = _alone(V, sc, n)
    for f in st_a:
        np.testing.assert_array_equal(got[1][f], st_a[f])
    for x, y in zip(got[2], fr_a):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("fault,status", [("VUDA_FAULT_REJECT_JOB", 1), ("VUDA_FAULT_OOM_JOB", 2)])
def test_fault_at_admission_leaves_the_other_jobs_unchanged(V, monkeypatch, fault, status):
    """The second job's admission is refused (or fails as out of memory):
    its requests complete with that status (or, once the job has failed, are
    refused at submission), and the other jobs' states and frames are
    bit-identical to running alone."""
    jobs = {"A": S.cfg2(6), "B": S.cfg1(4), "C": S.cfg4(4)}
    counts = {"A": 4, "B": 3, "C": 5}
    got = _faulted_run(V, monkeypatch, {fault: 2}, jobs, counts)
    # submitted before the admission failed: that status; after: refused at submit
    assert len(got["B"][0]) == 3 and set(got["B"][0]) <= {status, "refused"}
    for k in ("A", "C"):
        assert got[k][0] == [0] * counts[k]
        _same_as_alone(V, jobs[k], counts[k], got[k])


def test_fault_stalled_producer_leaves_results_unchanged(V, monkeypatch):
    """The batching worker stalls 4 ms before every second launch: requests
    pile up and are batched differently, every job's results are still
    bit-identical to running alone."""
    jobs = {"A": S.cfg2(6), "B": S.cfg1(4)}
    counts = {"A": 6, "B": 5}
    got = _faulted_run(V, monkeypatch, {"VUDA_FAULT_STALL_MS": 4, "VUDA_FAULT_STALL_EVERY": 2}, jobs, counts)
    for k in jobs:
        assert got[k][0] == [0] * counts[k]
        _same_as_alone(V, jobs[k], counts[k], got[k])


def test_cancelled_job_mid_batch_leaves_the_other_jobs_unchanged(V, monkeypatch):
    """A job removed while some of its requests are on the GPU: its queued
    requests are cancelled (VUDA_ERR_BUSY), the ones already launched
    complete, and the other jobs' results are bit-identical to running
    alone."""
    jobs = {"A": S.cfg2(6), "B": S.cfg2(5, env_base=50), "C": S.cfg1(4)}
    counts = {"A": 5, "B": 8, "C": 6}
    got = _faulted_run(V, monkeypatch, {}, jobs, counts, cancel="B")
    st_b = got["B"][0]
    assert len(st_b) == counts["B"] and set(st_b) <= {0, 6}
    assert st_b == sorted(st_b)                 # launched (in order) before cancelled
    assert 6 in st_b                            # some were still queued
    for k in ("A", "C"):
        assert got[k][0] == [0] * counts[k]
        _same_as_alone(V, jobs[k], counts[k], got[k])


def test_hull_contact_job_in_a_mix_matches_the_oracle(V, orc):
    """A job with hull contacts served in one launch with a job without them
    (the work lists run the physics variant with hull contacts for both):
    both match the oracle."""
    import dataclasses
    H = S.generate(6, 12, 91, kinds="mixed_hulls", hull_tris=(8, 24), n_hull_meshes=4, substeps=4)
    H = dataclasses.replace(H, params=dataclasses.replace(H.params, hull_contacts=1))
    st0, _, _ = orc.sim_step(H, 60)
    H = dataclasses.replace(H, **{k: st0[k] for k in ("pos", "quat", "vel", "angvel")})
    P = S.cfg1(4)
    srv = V.Server(max_inflight=2)
    jh, jp = srv.add_job(H), srv.add_job(P)
    for _ in range(3):
        srv.submit(jh)
        srv.submit(jp)
    res = srv.wait_all(6)
    assert all(r["status"] == 0 for r in res)
    for sc, j in ((H, jh), (P, jp)):
        got = srv.job_env(j).get_state()
        so, _, _ = orc.sim_step(sc, 3)
        for f in ("pos", "vel", "quat", "angvel"):
            np.testing.assert_allclose(got[f], so[f], rtol=1e-5, atol=1e-5)
    srv.close()
