"""Pins of the oracle's time-like cluster (Wolff) move.

The move must leave the same Trotterised path distribution invariant as the
single-spin sweep: at a frozen (A, B) it samples
exp(-alpha sum_tau E_P(sigma^tau) + Jperp sum sigma^tau sigma^{tau+1}),
enumerated over every path (chi-square), and at large L it approaches the
quantum single-spin closed form.  The bond probability is pinned to its
closed form 1 - e^(-2 Jperp) = 1 - tanh(beta A / L); at L = 4 and 8 on a
4-spin problem it matches the exact finite-L transfer-matrix value; the
three random streams are pinned as uniform; resume and replica subsets give
the same bits.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W
from test_oracle_statistics import (_all_states, _chisq_p, _energy_np, _path_index, _thermal_expectation,
                                    _trotter_expectation, _trotter_weights)


def _sample_paths(pb, L, beta, A0, B0, seed, R=128, S=3000, burn=40, every=3):
    A = np.full(S, A0)
    B = np.full(S, B0)
    q = O.SQA(pb, L, R, beta, A, B, seed=seed, move="wolff")
    q.run(0, burn)
    used = np.flatnonzero(pb.used)
    counts = None
    t = burn
    while t + every <= S:
        q.run(t, t + every)
        t += every
        idx = _path_index(q.s, used, L)
        if counts is None:
            counts = np.zeros(2 ** (len(used) * L), np.int64)
        np.add.at(counts, idx, 1)
    return counts


@pytest.mark.parametrize("L,A0,R,S,every", [(2, 0.8, 128, 3000, 3), (4, 0.8, 128, 3000, 4),
                                             (4, 0.15, 256, 6000, 12)])
def test_wolff_samples_the_exact_trotter_distribution(L, A0, R, S, every):
    """LHZ K_3 (3 spins, one 3-body constraint) at a frozen schedule point;
    A0 = 0.15 makes Jperp large, so most bonds join and clusters are long
    (samples thinned further there: successive states are more alike)."""
    pb = O.Problem("lhz", 3, np.array([1, -2, 3], np.int32), 2)
    beta, B0 = 1.5, 0.6
    counts = _sample_paths(pb, L, beta, A0, B0, seed=31, R=R, S=S, every=every)
    probs, _ = _trotter_weights(pb, L, beta, A0, B0)
    assert _chisq_p(counts, probs) > 1e-3
    wrong, _ = _trotter_weights(pb, L, beta, A0, B0, jperp_sign=-1.0)
    assert _chisq_p(counts, wrong) < 1e-6


def test_wolff_single_spin_ring_distribution():
    """One spin (LHZ K_2, field J) on a ring of L = 8 slices: all 256 paths."""
    pb = O.Problem("lhz", 2, np.array([2], np.int32), 1)
    L, beta, A0, B0 = 8, 2.0, 0.6, 0.4
    counts = _sample_paths(pb, L, beta, A0, B0, seed=8, R=256, S=2500, every=2)
    probs, _ = _trotter_weights(pb, L, beta, A0, B0)
    assert _chisq_p(counts, probs) > 1e-3
    # a bond probability of e^(-2 Jperp) instead of 1 - e^(-2 Jperp) would
    # sample another ring coupling: a different Jperp must be rejected
    alt, _ = _trotter_weights(pb, L, beta, A0 * 1.6, B0)
    assert _chisq_p(counts, alt) < 1e-6


def test_wolff_single_spin_quantum_limit():
    """<sigma^z> = -(B J / w) tanh(beta w), w = sqrt(A^2 + B^2 J^2), at L = 64."""
    J = np.array([2], np.int32)
    pb = O.Problem("lhz", 2, J, 1)
    beta, A0, B0, L = 2.0, 1.0, 0.5, 64
    S = 600
    q = O.SQA(pb, L, 256, beta, np.full(S, A0), np.full(S, B0), seed=5, move="wolff")
    q.run(0, 50)
    acc = []
    for t in range(50, S, 5):
        q.run(t, t + 5)
        acc.append(q.s[:, 0, :].astype(np.float64).mean())
    est = float(np.mean(acc))
    w = math.sqrt(A0 ** 2 + (B0 * J[0]) ** 2)
    exact = -(B0 * J[0] / w) * math.tanh(beta * w)
    assert abs(est - exact) < 0.02, (est, exact)


def test_wolff_finite_trotter_number_transfer_matrix():
    """ME of K_2 (4 spins; 32 path bits at L = 8, beyond enumeration) at a
    frozen (A, B) with a large Trotter error: the cluster move's <H_P> at
    L = 4 and 8 equals the exact finite-L value from the transfer matrix
    (exp((beta A / L) sigma^x) per spin), not the other L's nor the limit."""
    pb = O.Problem("me", 2, np.array([2], np.int32), 1)
    states, used = _all_states(pb)
    diagE = _energy_np(pb, states).astype(np.float64)
    m = len(used)
    beta, A0, B0 = 3.0, 1.0, 0.6
    exact = {L: _trotter_expectation(diagE, m, beta, A0, B0, L) for L in (4, 8, 16)}
    limit = _thermal_expectation(diagE, m, beta, A0, B0)
    for L in (4, 8):
        S = 1600
        q = O.SQA(pb, L, 256, beta, np.full(S, A0), np.full(S, B0), seed=60 + L, move="wolff")
        q.run(0, 100)
        acc = []
        for t in range(100, S, 6):
            q.run(t, t + 6)
            acc.append(q.slice_energies().mean())
        est = float(np.mean(acc))
        assert abs(est - exact[L]) < 0.03, (L, est, exact[L])
        others = [exact[k] for k in (4, 8, 16) if k != L] + [limit]
        assert min(abs(est - o) for o in others) > 0.12, (L, est, others)


@pytest.mark.parametrize("beta,A,L", [(10 / 3, 0.9, 64), (10 / 3, 0.01, 64), (1.0, 0.5, 8), (20.0, 1e-4, 128)])
def test_bond_threshold_closed_form(beta, A, L):
    a = beta * A / L
    mpmath.mp.dps = 50
    p = 1 - mpmath.tanh(mpmath.mpf(a))
    want = min(int(mpmath.floor(p * 2 ** 32)), 2 ** 32 - 2)
    got = O.bond_threshold(beta, A, L)
    assert abs(got - want) <= 1          # double rounding of tanh at the last bit
    # the same probability written through Jperp: 1 - e^(-2 Jperp)
    jp = O.jperp(beta, A, L)
    assert abs(got / 2 ** 32 - (1 - math.exp(-2 * jp))) < 2.0 ** -31  # floor to 2^-32 steps
    assert O.bond_threshold(beta, 0.0, L) == 0xFFFFFFFF


def test_wolff_streams_are_uniform():
    L = 48
    starts = np.array([O.wolff_start(7, t, s, r, 3, L) for t in range(4) for s in range(5) for r in range(100)])
    assert starts.min() >= 0 and starts.max() < L
    assert stats.chisquare(np.bincount(starts, minlength=L)).pvalue > 1e-3
    bonds = np.array([O.wolff_bond_uniform(7, t, s, L, tau, r, 3)
                      for t in range(2) for s in range(3) for tau in (0, 17, 47) for r in range(0, 200, 3)])
    assert stats.kstest(bonds / 2 ** 32, "uniform").pvalue > 1e-3
    acc = np.array([O.wolff_accept_uniform(7, t, s, r, 3) for t in range(5) for s in range(6) for r in range(90)])
    assert stats.kstest(acc / 2 ** 32, "uniform").pvalue > 1e-3
    # the streams differ from each other and from the single-spin sweep's
    assert O.wolff_accept_uniform(7, 0, 0, 0, 3) != O.sweep_uniform(7, 0, 0, 0, 3)


def test_wolff_resume_and_replica_subsets():
    pb = O.Problem("me", 8, W.random_couplings(8, 4), 6)
    A, B = O.linear_schedule(60)
    a = O.SQA(pb, 16, 40, 10 / 3, A, B, seed=4, inst=2, move="wolff")
    a.run(0, 60)
    b = O.SQA(pb, 16, 40, 10 / 3, A, B, seed=4, inst=2, move="wolff")
    b.run(0, 23)
    b.run(23, 60)
    assert np.array_equal(a.s, b.s)
    c = O.SQA(pb, 16, 40, 10 / 3, A, B, seed=4, inst=2, move="wolff")
    c.run(0, 60, 0, 17)
    c.run(0, 60, 17, 40)
    assert np.array_equal(a.s, c.s)
    d = O.SQA(pb, 16, 40, 10 / 3, A, B, seed=4, inst=2)  # single-spin sweep: another chain
    d.run(0, 60)
    assert not np.array_equal(a.s, d.s)
