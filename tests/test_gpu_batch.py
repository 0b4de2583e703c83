"""Reusable batches replayed from a CUDA graph, and the launch-shape autotuner.

Launch shapes and graph replays change speed only: every random number is
keyed by sweep, site, slice, replica and instance, so the bits must equal the
same jobs run alone through sqa_run (which the parity tests pin to the
oracle), and one sampled job is checked against the oracle directly.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu


def _specs():
    # ragged: LHZ and ME, several N, L, replica counts with ragged tails, PT
    return [dict(kind="sqa", embedding="lhz", N=8, L=32, R=96, sweeps=40, seed=11),
            dict(kind="sqa", embedding="me", N=12, L=16, R=40, sweeps=60, seed=12),
            dict(kind="pt", embedding="me", N=8, R=64, sweeps=30, seed=13),
            dict(kind="sqa", embedding="me", N=5, L=8, R=7, sweeps=90, seed=14),
            dict(kind="pt", embedding="lhz", N=7, R=33, sweeps=25, seed=15),
            dict(kind="sqa", embedding="lhz", N=10, L=64, R=256, sweeps=20, seed=16)]


def _make(spec, I=3):
    kw = dict(spec)
    kw["J"] = W.random_instances(kw["N"], I, kw["seed"])
    kw["penalty"] = 6 if kw["embedding"] == "me" else 9
    if kw["kind"] == "sqa":
        kw["beta"] = 10 / 3
    else:
        kw.update(betas=W.geometric_ladder(8, 5.0, 0.2), swap_every=2)
    return kw


def _alone(kw):
    h = pkg.Handle(**kw)
    h.run(stream=0)
    st, en = h.state(stream=0), h.energies(stream=0)
    h.close()
    return st, en


def test_graph_replay_equals_alone_runs_and_oracle():
    kws = [_make(s) for s in _specs()]
    hs = [pkg.Handle(**kw) for kw in kws]
    b = pkg.Batch(hs)
    ref = [_alone(kw) for kw in kws]
    for rep in range(2):                      # the second launch replays the graph
        b.launch(stream=0)
        for h, (st, en) in zip(hs, ref):
            assert np.array_equal(h.state(stream=0), st)
            assert np.array_equal(h.energies(stream=0), en)
    # one job against the oracle
    kw = kws[3]
    pb = O.Problem(kw["embedding"], kw["N"], kw["J"][2], kw["penalty"])
    A, B = O.linear_schedule(kw["sweeps"])
    q = O.SQA(pb, kw["L"], kw["R"], kw["beta"], A, B, kw["seed"], 2)
    q.run(0, kw["sweeps"])
    assert np.array_equal(pkg.unpack_words(hs[3].state(stream=0), kw["R"])[2], q.s)
    b.close()
    for h in hs:
        h.close()


def test_batch_autotune_keeps_the_bits():
    kws = [_make(s, I=2) for s in _specs()]
    hs = [pkg.Handle(**kw) for kw in kws]
    b = pkg.Batch(hs)
    got = b.autotune(n_trial=5, stream=0)
    assert got["words_per_unit"] in (0, 1, 2, 4, 8)
    assert got["trial_attempts_per_s"] > 0
    b.launch(stream=0)
    for h, kw in zip(hs, kws):
        st, en = _alone(kw)
        assert np.array_equal(h.state(stream=0), st)
        assert np.array_equal(h.energies(stream=0), en)
    b.close()
    for h in hs:
        h.close()


@pytest.mark.parametrize("spec", [dict(kind="sqa", embedding="me", N=8, L=16, R=200, sweeps=30, seed=21),
                                  dict(kind="pt", embedding="lhz", N=8, R=64, sweeps=20, seed=22)])
def test_autotune_keeps_state_and_bits(spec):
    """Autotune between two halves of a run (checkpoint/resume): the spins
    are saved and restored, and the finished run equals an untuned one."""
    kw = _make(spec, I=4)
    ref_st, ref_en = _alone(kw)
    h = pkg.Handle(**kw)
    S = kw["sweeps"]
    h.run_sweeps(0, S // 2, stream=0)
    mid = h.state(stream=0)
    got = h.autotune(n_trial=4, stream=0)
    assert got["trial_attempts_per_s"] > 0
    assert h.launch()["words_per_unit"] == got["words_per_unit"]
    assert np.array_equal(h.state(stream=0), mid)
    h.run_sweeps(S // 2, S, stream=0)
    assert np.array_equal(h.state(stream=0), ref_st)
    assert np.array_equal(h.energies(stream=0), ref_en)
    h.close()
