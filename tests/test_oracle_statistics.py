"""Statistical pins of the oracle's Markov chains against exact results.

P4  Zero-field Metropolis (PT with one slot) samples the Boltzmann
    distribution of the physical problem (chi-square over all states); a 15%
    error in beta or one flipped coupling sign is rejected.
P5  SQA at a frozen (A, B) samples the exact Trotterised path distribution
    exp(-alpha sum_tau E_P(sigma^tau) + Jperp sum sigma^tau sigma^{tau+1}),
    enumerated over every path (chi-square); a wrong sign of Jperp is rejected.
P6  SQA at large L approaches the quantum thermal state: the single-spin
    closed form <sigma^z> = -(B J / w) tanh(beta w), w = sqrt(A^2 + B^2 J^2),
    and an exact diagonalisation (numpy) of a 4-spin transverse-field problem;
    at small L it matches the exact finite-L Trotter value from the transfer
    matrix (whose error against the limit falls as (beta / L)^2).
P8  PT with two slots and swaps samples the product of the two Boltzmann
    distributions (chi-square over the joint histogram).
P3  PT on the paper's ladder down to beta = 20 finds the logical ground state.
P10 Same seed -> same bits; resuming at any sweep and simulating a subset of
    replicas give the same bits as one uninterrupted run.

The exact distributions here are computed from the term lists with numpy,
independently of the oracle's energy and flip routines.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W


def _energy_np(pb, states):
    """E(sigma) = sum_terms w prod sigma over members, for states [M][n]."""
    e = np.zeros(len(states), np.int64)
    for mem, w in pb.terms():
        e += w * np.prod(states[:, mem].astype(np.int64), axis=1)
    return e


def _all_states(pb):
    used = np.flatnonzero(pb.used)
    m = len(used)
    idx = np.arange(2 ** m)
    states = np.ones((2 ** m, pb.n), np.int8)
    for b, site in enumerate(used):
        states[:, site] = np.where((idx >> b) & 1, -1, 1)
    return states, used


def _state_index(s, used):
    """s [n][R] -> index per replica (bit b = site used[b] is down)."""
    bits = (s[used, :] < 0).astype(np.int64)
    return (bits << np.arange(len(used))[:, None]).sum(axis=0)


def _chisq_p(counts, probs, min_expected=5.0):
    n = counts.sum()
    exp = probs * n
    big = exp >= min_expected
    c = np.append(counts[big], counts[~big].sum())
    e = np.append(exp[big], exp[~big].sum())
    if e[-1] == 0:
        c, e = c[:-1], e[:-1]
    e = e * c.sum() / e.sum()
    return stats.chisquare(c, e).pvalue


def _boltzmann(E, beta):
    w = np.exp(-beta * (E - E.min()))
    return w / w.sum()


def _sample_pt(pb, betas, R, swap_every, seed, burn, n_samples, thin):
    pt = O.PT(pb, betas, R, swap_every, seed)
    pt.run(0, burn)
    t = burn
    out = []
    for _ in range(n_samples):
        pt.run(t, t + thin)
        t += thin
        out.append(pt.s.copy())
    return out


@pytest.mark.parametrize("emb,N,beta", [("me", 4, 0.35), ("lhz", 4, 0.45)])
def test_p4_metropolis_boltzmann(emb, N, beta):
    J = W.random_couplings(N, 21)
    pb = O.Problem(emb, N, J, 2)
    states, used = _all_states(pb)
    E = _energy_np(pb, states)
    samples = _sample_pt(pb, [beta], 128, 10**9, seed=2024, burn=50, n_samples=300, thin=8)
    counts = np.zeros(len(states), np.int64)
    for s in samples:
        np.add.at(counts, _state_index(s[0], used), 1)
    assert _chisq_p(counts, _boltzmann(E, beta)) > 1e-3
    # power: a 15% error in beta, or one coupling with the wrong sign, is rejected
    assert _chisq_p(counts, _boltzmann(E, 1.15 * beta)) < 1e-6
    J2 = J.copy()
    J2[0] = -J2[0]
    pb2 = O.Problem(emb, N, J2, 2)
    assert _chisq_p(counts, _boltzmann(_energy_np(pb2, states), beta)) < 1e-6


def _trotter_weights(pb, L, beta, A, B, jperp_sign=1.0):
    used = np.flatnonzero(pb.used)
    m = len(used)
    M = 2 ** (m * L)
    idx = np.arange(M)
    # path[k][tau][b]: bit (tau*m + b) of k
    path = np.where((idx[:, None, None] >> (np.arange(L)[None, :, None] * m
                                            + np.arange(m)[None, None, :])) & 1, -1, 1)
    Etot = np.zeros(M, np.float64)
    for tau in range(L):
        st = np.ones((M, pb.n), np.int8)
        st[:, used] = path[:, tau, :]
        Etot += _energy_np(pb, st)
    bond = np.zeros(M, np.float64)
    for tau in range(L):
        bond += (path[:, tau, :] * path[:, (tau + 1) % L, :]).sum(axis=1)
    alpha = beta * B / L
    jp = 0.5 * math.log(1.0 / math.tanh(beta * A / L)) * jperp_sign
    logw = -alpha * Etot + jp * bond
    w = np.exp(logw - logw.max())
    return w / w.sum(), used


def _path_index(s, used, L):
    m = len(used)
    idx = np.zeros(s.shape[-1], np.int64)
    for tau in range(L):
        bits = (s[tau][used, :] < 0).astype(np.int64)
        idx |= (bits << (tau * m + np.arange(m))[:, None]).sum(axis=0)
    return idx


@pytest.mark.parametrize("L", [2, 4])
def test_p5_exact_trotter_distribution(L):
    N = 3
    J = np.array([1, -2, 3], np.int32)
    pb = O.Problem("lhz", N, J, 2)
    beta, A0, B0 = 1.5, 0.8, 0.6
    S = 4000
    A = np.full(S, A0)
    B = np.full(S, B0)
    q = O.SQA(pb, L, 128, beta, A, B, seed=99)
    q.run(0, 40)
    t = 40
    probs, used = _trotter_weights(pb, L, beta, A0, B0)
    counts = np.zeros(len(probs), np.int64)
    while t + 4 <= S:
        q.run(t, t + 4)
        t += 4
        np.add.at(counts, _path_index(q.s, used, L), 1)
    assert _chisq_p(counts, probs) > 1e-3
    wrong, _ = _trotter_weights(pb, L, beta, A0, B0, jperp_sign=-1.0)
    assert _chisq_p(counts, wrong) < 1e-6


def test_p6_single_spin_closed_form():
    """LHZ K_2 is one spin with local field J: H = -A sigma^x + B J sigma^z."""
    J = np.array([2], np.int32)
    pb = O.Problem("lhz", 2, J, 1)
    beta, A0, B0, L = 2.0, 1.0, 0.5, 64
    S = 1200
    q = O.SQA(pb, L, 256, beta, np.full(S, A0), np.full(S, B0), seed=5)
    q.run(0, 100)
    acc = []
    for t in range(100, S, 10):
        q.run(t, t + 10)
        acc.append(q.s[:, 0, :].astype(np.float64).mean())
    est = float(np.mean(acc))
    w = math.sqrt(A0 ** 2 + (B0 * J[0]) ** 2)
    exact = -(B0 * J[0] / w) * math.tanh(beta * w)
    classical = -math.tanh(beta * B0 * J[0])
    assert abs(est - exact) < 0.02, (est, exact)
    assert abs(est - classical) > 0.2


def test_p6_exact_diagonalisation_me_k2():
    """ME of K_2: two chains of two spins (4 spins); <H_P> from PIMC at L = 64
    against the thermal expectation from exact diagonalisation."""
    N = 2
    J = np.array([2], np.int32)
    P = 1
    pb = O.Problem("me", N, J, P)
    used = np.flatnonzero(pb.used)
    m = len(used)
    assert m == 4
    dim = 2 ** m
    states = np.ones((dim, pb.n), np.int8)
    for b, site in enumerate(used):
        states[:, site] = np.where((np.arange(dim) >> b) & 1, -1, 1)
    diagE = _energy_np(pb, states).astype(np.float64)
    beta, A0, B0, L = 1.5, 0.7, 0.8, 64
    H = np.diag(B0 * diagE)
    for b in range(m):                             # -A sigma^x on each used spin
        for k in range(dim):
            H[k ^ (1 << b), k] -= A0
    ev, V = np.linalg.eigh(H)
    rho = V @ np.diag(np.exp(-beta * (ev - ev.min()))) @ V.T
    exact = float(np.trace(np.diag(diagE) @ rho) / np.trace(rho))
    S = 900
    q = O.SQA(pb, L, 128, beta, np.full(S, A0), np.full(S, B0), seed=17)
    q.run(0, 100)
    acc = []
    for t in range(100, S, 8):
        q.run(t, t + 8)
        acc.append(q.slice_energies().mean())
    est = float(np.mean(acc))
    classical = float((_boltzmann(diagE, beta * B0) * diagE).sum())
    assert abs(est - exact) < 0.05 * abs(exact) + 0.05, (est, exact)
    assert abs(classical - exact) > 3 * abs(est - exact)


def _trotter_expectation(diagE, m, beta, A0, B0, L, obs=None):
    """<E_P> (or <obs>, diagonal) of the L-slice Trotter decomposition of exp(-beta H),
    H = B0 diag(E) - A0 sum_i sigma^x_i, as the trace of the transfer matrix
    sqrt(D) K sqrt(D) to the power L: D = diag(exp(-beta B0 E / L)) and
    K = exp((beta A0 / L) sigma^x) on every spin (cosh / sinh entries), built
    from the matrix exponential, not from a coupling along imaginary time."""
    a = beta * A0 / L
    k1 = np.array([[math.cosh(a), math.sinh(a)], [math.sinh(a), math.cosh(a)]])
    K = np.ones((1, 1))
    for _ in range(m):
        K = np.kron(K, k1)
    d = np.exp(-beta * B0 * (diagE - diagE.min()) / (2 * L))
    ML = np.linalg.matrix_power(d[:, None] * K * d[None, :], L)
    o = diagE if obs is None else obs
    return float(np.trace(np.diag(o) @ ML) / np.trace(ML))


def _thermal_expectation(diagE, m, beta, A0, B0):
    dim = 2 ** m
    H = np.diag(B0 * diagE)
    for b in range(m):
        for k in range(dim):
            H[k ^ (1 << b), k] -= A0
    ev, V = np.linalg.eigh(H)
    rho = V @ np.diag(np.exp(-beta * (ev - ev.min()))) @ V.T
    return float(np.trace(np.diag(diagE) @ rho) / np.trace(rho))


def test_p6_finite_trotter_number_transfer_matrix():
    """ME of K_2 (4 spins, 4 L path bits: too many to enumerate at L = 8) at a
    frozen (A, B) where the Trotter error is large: the oracle's <H_P> at
    L = 4 and 8 equals the transfer-matrix value of that L, which differs from
    the other L and from the quantum limit by far more than the tolerance, and
    at L = 8 so does <sigma^z_a sigma^z_b> for every pair of spins.  The
    transfer matrices themselves approach exact diagonalisation with an error
    falling as (beta / L)^2."""
    pb = O.Problem("me", 2, np.array([2], np.int32), 1)
    states, used = _all_states(pb)
    diagE = _energy_np(pb, states).astype(np.float64)
    m = len(used)
    beta, A0, B0 = 3.0, 1.0, 0.6
    exact = {L: _trotter_expectation(diagE, m, beta, A0, B0, L) for L in (4, 8, 16, 32, 512)}
    limit = _thermal_expectation(diagE, m, beta, A0, B0)
    assert abs(exact[512] - limit) < 1e-3
    r = (exact[16] - limit) / (exact[32] - limit)
    assert 3.6 < r < 4.4, r                       # Trotter error ~ (beta / L)^2
    pairs = [(a, b) for a in range(m) for b in range(a + 1, m)]
    corr = {(a, b): states[:, used[a]].astype(np.float64) * states[:, used[b]] for a, b in pairs}
    for L in (4, 8):
        S = 1600
        q = O.SQA(pb, L, 256, beta, np.full(S, A0), np.full(S, B0), seed=40 + L)
        q.run(0, 100)
        acc, cacc = [], []
        for t in range(100, S, 6):
            q.run(t, t + 6)
            acc.append(q.slice_energies().mean())
            sz = q.s.astype(np.float64)
            cacc.append([(sz[:, used[a], :] * sz[:, used[b], :]).mean() for a, b in pairs])
        est = float(np.mean(acc))
        assert abs(est - exact[L]) < 0.03, (L, est, exact[L])
        others = [exact[k] for k in (4, 8, 16) if k != L] + [limit]
        assert min(abs(est - o) for o in others) > 0.12, (L, est, others)
        if L == 8:
            got = np.mean(cacc, axis=0)
            want = np.array([_trotter_expectation(diagE, m, beta, A0, B0, 8, corr[p]) for p in pairs])
            far = np.array([_trotter_expectation(diagE, m, beta, A0, B0, 512, corr[p]) for p in pairs])
            assert np.abs(got - want).max() < 0.03, (got, want)
            assert np.abs(got - far).max() > 0.06, (got, far)


def test_p8_pt_two_slot_joint_distribution():
    N = 4
    pb = O.Problem("lhz", N, W.random_couplings(N, 8), 1)
    states, used = _all_states(pb)
    E = _energy_np(pb, states)
    betas = [0.6, 0.3]
    samples = _sample_pt(pb, betas, 128, 1, seed=31, burn=50, n_samples=600, thin=4)
    ns = len(states)
    counts = np.zeros(ns * ns, np.int64)
    for s in samples:
        i0 = _state_index(s[0], used)
        i1 = _state_index(s[1], used)
        np.add.at(counts, i0 * ns + i1, 1)
    p0 = _boltzmann(E, betas[0])
    p1 = _boltzmann(E, betas[1])
    assert _chisq_p(counts, np.outer(p0, p1).ravel()) > 1e-3
    # swapping the two marginals is rejected
    assert _chisq_p(counts, np.outer(p1, p0).ravel()) < 1e-6


@pytest.mark.parametrize("emb,N", [("me", 4), ("lhz", 4), ("me", 6), ("lhz", 5)])
def test_p3_pt_finds_ground_state(emb, N):
    J = W.random_couplings(N, 500 + N)
    e_gs, _ = O.ground_energy(N, J)
    pb = O.Problem(emb, N, J, 12)                  # penalty well above critical
    betas = W.paper_beta_ladder(16, 20.0, 0.1)
    pt = O.PT(pb, betas, 32, 10, seed=3)
    pt.run(0, 400)
    ok = 0
    for r in range(32):
        phys = pt.s[0, :, r]
        if emb == "me":
            s = O.me_decode(pb, phys)
        else:
            s = O.lhz_tree_decode(N, O.star_tree(N), phys)
        ok += O.logical_energy(N, J, s) == e_gs
    assert ok >= 31


def test_p10_determinism_resume_and_replica_subsets():
    N = 6
    pb = O.Problem("lhz", N, W.random_couplings(N, 0), 9)
    A, B = O.linear_schedule(60)
    a = O.SQA(pb, 8, 40, 10 / 3, A, B, seed=7)
    a.run(0, 60)
    b = O.SQA(pb, 8, 40, 10 / 3, A, B, seed=7)
    b.run(0, 25)
    b.run(25, 60)
    assert np.array_equal(a.s, b.s)
    c = O.SQA(pb, 8, 40, 10 / 3, A, B, seed=7)
    c.run(0, 60, 8, 19)                            # replicas 8..18 only
    assert np.array_equal(a.s[:, :, 8:19], c.s[:, :, 8:19])
    d = O.SQA(pb, 8, 40, 10 / 3, A, B, seed=8)
    d.run(0, 60)
    assert not np.array_equal(a.s, d.s)
    # PT, with swaps, resumed across a swap boundary and on a replica subset
    pme = O.Problem("me", 5, W.random_couplings(5, 1), 6)
    betas = W.geometric_ladder(6, 3.0, 0.2)
    p = O.PT(pme, betas, 33, 3, seed=5)
    p.run(0, 31)
    q = O.PT(pme, betas, 33, 3, seed=5)
    q.run(0, 10)
    q.run(10, 31)
    assert np.array_equal(p.s, q.s) and np.array_equal(p.E, q.E)
    r = O.PT(pme, betas, 33, 3, seed=5)
    r.run(0, 31, 32, 33)
    assert np.array_equal(p.s[:, :, 32], r.s[:, :, 32])
    for z in range(6):
        assert np.array_equal(p.E[z], pme.energies(p.s[z]))
