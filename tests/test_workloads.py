"""Checks of the seeded input generators and the paper's temperature ladder.

P9: the PT temperatures the paper quotes (1.05, 2.1 and 4.0 in Figs. 5-7 and
App. C; beta_1 = 20 in Fig. 7) are members of its ladder
beta_i = beta_1 (0.1/20)^((i-1)/63), at i = 36, 28, 20 and 1.  This pins the
ladder formula and its 1-based index.
"""
import numpy as np

import workloads as W


def test_paper_ladder_contains_quoted_temperatures():
    b = W.paper_beta_ladder()
    assert len(b) == 64
    assert b[0] == 20.0 and abs(b[-1] - 0.1) < 1e-12
    assert np.all(np.diff(b) < 0)
    assert round(b[36 - 1], 2) == 1.05
    assert round(b[28 - 1], 1) == 2.1
    assert round(b[20 - 1], 1) == 4.0


def test_couplings_values_and_determinism():
    J = W.random_instances(8, 50, 0)
    assert J.shape == (50, 28) and J.dtype == np.int32
    assert set(np.unique(J).tolist()) == {-3, -2, -1, 1, 2, 3}
    assert np.array_equal(J, W.random_instances(8, 50, 0))
    assert not np.array_equal(J[0], J[1])
    counts = np.bincount(J.ravel() + 3, minlength=7)
    assert counts[3] == 0 and counts.min(initial=10**9, where=np.arange(7) != 3) > 150


def test_splitmix64_stream():
    g = W.SplitMix64(0)
    a = [g.next() for _ in range(3)]
    assert len(set(a)) == 3 and all(0 <= x < 2**64 for x in a)
    assert a == [W.SplitMix64(0).next() for _ in range(1)] + a[1:]


def test_workload_shapes():
    c1 = W.lhz_n6_config()
    assert c1["N"] == 6 and c1["L"] == 32 and c1["R"] == 64 and c1["sweeps"] == 1000
    assert c1["penalty"] == 3 * W.max_abs(c1["J"])
    c2 = W.me_n8_batch_config(n_inst=4)
    assert c2["J"].shape == (4, 28) and c2["penalty"] == 6
    mix = W.ragged_mix_config(n_inst=20, sweeps=10)
    assert {j["embedding"] for j in mix} == {"me", "lhz"}
    assert {j["L"] for j in mix} == {32, 64}
    pt = W.pt_config("me", n_inst=2, sweeps=10)
    assert pt["N"] == 32 and len(pt["betas"]) == 32
    assert abs(pt["betas"][0] - 10.0) < 1e-12 and abs(pt["betas"][-1] - 0.1) < 1e-12
    jobs = W.serving_stream(30)
    assert all(6 <= j["N"] <= 40 and 1 <= j["R"] <= 256 for j in jobs)
    assert all(1000 <= j["sweeps"] <= 100000 for j in jobs)
