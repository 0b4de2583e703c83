"""Serving: continuous batching on the GPU.

Jobs of different shapes (SQA and PT, ME and LHZ, several N, L and replica
counts) are submitted while others are running, under a memory budget that
holds only some of them at once.  Every job's final state and energies must
equal the same job run alone through sqa_run, bit for bit, and agree with the
oracle on a sampled job.
"""
import time

import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu


def _jobs():
    out = []
    specs = [("sqa", "lhz", 8, 32, 64, 400), ("sqa", "me", 12, 16, 40, 300), ("pt", "me", 8, 0, 64, 250),
             ("sqa", "lhz", 10, 8, 200, 500), ("pt", "lhz", 7, 0, 33, 300), ("sqa", "me", 5, 4, 7, 900),
             ("sqa", "lhz", 14, 16, 96, 120), ("pt", "me", 16, 0, 32, 150)]
    for k, (kind, emb, N, L, R, S) in enumerate(specs):
        kw = dict(embedding=emb, N=N, J=W.random_instances(N, 2, 300 + k), penalty=6 if emb == "me" else 9,
                  sweeps=S, R=R, seed=300 + k, kind=kind)
        if kind == "sqa":
            kw.update(L=L, beta=10 / 3)
        else:
            kw.update(betas=W.geometric_ladder(8, 5.0, 0.2), swap_every=2)
        out.append(kw)
    return out


def test_served_results_equal_alone_runs():
    jobs = _jobs()
    budgets = [pkg.plan_device_bytes(**kw) for kw in jobs]
    srv = pkg.Server(mem_budget_bytes=int(2.5 * max(budgets)), unit_attempts_per_chunk=2_000_000)
    ids = []
    for k, kw in enumerate(jobs):
        ids.append(srv.submit(**kw))
        if k == 3:
            time.sleep(0.05)      # later jobs arrive while the first ones run
    for jid in ids:
        srv.wait(jid, timeout=600)
    stats = srv.stats()
    assert stats["jobs_done"] == len(jobs) and stats["jobs_failed"] == 0
    assert stats["max_resident"] >= 2           # jobs shared launches
    assert stats["max_bytes"] <= int(2.5 * max(budgets))
    for jid, kw, est in zip(ids, jobs, budgets):
        info = srv.poll(jid)
        assert info["state"] == "done"
        # admission estimate: exact for a handle of its own but for the
        # work-unit list, which it sizes for one unit per 32-replica word (an
        # upper bound); a served job packed into multi-job launches holds
        # less (no tie queue of its own)
        slack = kw["J"].shape[0] * ((kw["R"] + 31) // 32) * 16
        assert info["device_bytes"] <= est
        assert info["t_submit"] <= info["t_start"] <= info["t_done"]
        st, en = srv.result(jid)
        h = pkg.Handle(**kw)
        assert h.info["device_bytes"] <= est <= h.info["device_bytes"] + slack
        h.run(stream=0)
        assert np.array_equal(st, h.state(stream=0)), kw
        assert np.array_equal(en, h.energies(stream=0)), kw
        h.close()
    # one sampled job against the oracle
    kw = jobs[5]
    st, _ = srv.result(ids[5])
    pb = O.Problem(kw["embedding"], kw["N"], kw["J"][1], kw["penalty"])
    A, B = O.linear_schedule(kw["sweeps"])
    q = O.SQA(pb, kw["L"], kw["R"], kw["beta"], A, B, kw["seed"], 1)
    q.run(0, kw["sweeps"])
    assert np.array_equal(pkg.unpack_words(st[1], kw["R"]), q.s)
    for jid in ids:
        srv.release(jid)
    srv.close()


def test_job_larger_than_budget_fails_cleanly():
    kw = _jobs()[0]
    srv = pkg.Server(mem_budget_bytes=1024)
    jid = srv.submit(**kw)
    srv.wait(jid, timeout=60)
    info = srv.poll(jid)
    assert info["state"] == "failed" and info["status"] == pkg.SQA_ERR_NOMEM
    with pytest.raises(pkg.SQAError):
        srv.result(jid)
    srv.close()


def test_a_failing_job_fails_alone():
    """Jobs that cannot be planned (odd L; a cluster-move ring longer than
    128 slices) fail with their own status while the jobs around them
    finish with the same bits as alone; the worker keeps serving."""
    good = _jobs()[:3]
    bad_odd = dict(good[0], L=31)
    bad_ring = dict(good[0], L=130, move="wolff")
    srv = pkg.Server(mem_budget_bytes=1 << 32)
    ids = [srv.submit(**kw) for kw in (good[0], bad_odd, good[1], bad_ring, good[2])]
    for jid in ids:
        srv.wait(jid, timeout=600)
    states = [srv.poll(jid) for jid in ids]
    assert [s["state"] for s in states] == ["done", "failed", "done", "failed", "done"]
    assert states[1]["status"] == pkg.SQA_ERR_INVALID
    assert states[3]["status"] == pkg.SQA_ERR_UNSUPPORTED
    st = srv.stats()
    assert st["jobs_done"] == 3 and st["jobs_failed"] == 2 and st["worker_status"] == 0
    for jid, kw in zip([ids[0], ids[2], ids[4]], good):
        got, _ = srv.result(jid)
        h = pkg.Handle(**kw)
        h.run(stream=0)
        assert np.array_equal(got, h.state(stream=0))
        h.close()
    srv.close()


def test_cluster_job_beside_packed_jobs():
    """A job whose 32-replica word does not fit one block (LHZ K_40, L = 128),
    so that it runs clusters of its own sweep kernel on a high-priority
    stream, served beside small jobs packed into multi-job launches: every
    result equals the job alone."""
    J40 = W.random_instances(40, 1, 410)
    big = dict(embedding="lhz", N=40, J=J40, penalty=9, sweeps=16_000, R=32, seed=410, kind="sqa", L=128,
               beta=10 / 3)
    small = _jobs()[:3]
    srv = pkg.Server(mem_budget_bytes=1 << 33)
    ids = [srv.submit(**kw) for kw in [big] + small]
    for jid in ids:
        srv.wait(jid, timeout=600)
    assert all(srv.poll(jid)["state"] == "done" for jid in ids)
    for jid, kw in zip(ids, [big] + small):
        got, en = srv.result(jid)
        h = pkg.Handle(**kw)
        h.run(stream=0)
        assert np.array_equal(got, h.state(stream=0)), kw["N"]
        assert np.array_equal(en, h.energies(stream=0)), kw["N"]
        h.close()
    srv.close()
