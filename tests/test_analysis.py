"""Pins of the host-side analyses (App. D distance, App. E error rates).

Each function is checked against cases its definition fixes: distances of
identical, disjoint and hand-worked sets; the embedded ground states against
the oracle's own embedding and brute-force enumeration; error rates of
ground states, single flips and a brute-force minimum; the corner distance
against a breadth-first search over the LHZ constraint graph; error profiles
of planted and uniform noise; exact polynomial interpolation.
"""
import itertools
from collections import deque

import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_1603_03755_gb300 import analysis as A


def test_energy_distance_fixed_cases():
    assert A.energy_distance([1, 2, 2, 5], [5, 2, 1, 2]) == 0.0
    assert A.energy_distance([1, 2], [1, 1, 2, 2]) == 0.0            # same proportions
    assert A.energy_distance([1, 1], [2, 3]) == 1.0                  # disjoint
    assert A.energy_distance([1, 1, 2], [2, 2, 3]) == pytest.approx(2 / 3)  # 1/2 (2/3 + 1/3 + 1/3)
    rng = np.random.default_rng(0)
    a, b, c = (rng.integers(-5, 5, 200) for _ in range(3))
    dab, dba = A.energy_distance(a, b), A.energy_distance(b, a)
    assert dab == dba and 0.0 <= dab <= 1.0
    assert A.energy_distance(a, c) <= dab + A.energy_distance(b, c) + 1e-12
    with pytest.raises(ValueError):
        A.energy_distance([], [1])


@pytest.mark.parametrize("emb,N", [("me", 5), ("me", 8), ("me", 9), ("me", 12), ("lhz", 5), ("lhz", 8)])
def test_embedding_matches_the_oracle(emb, N):
    pb = O.Problem(emb, N, W.random_couplings(N, N), 6)
    rng = np.random.default_rng(N)
    for _ in range(5):
        q = rng.choice(np.array([-1, 1], np.int8), N)
        mine = A.embed_logical(emb, N, q)
        assert mine.shape == (pb.n,)
        assert np.array_equal(mine[pb.used.astype(bool)], pb.embed(q)[pb.used.astype(bool)])
        assert np.all(mine[~pb.used.astype(bool)] == 0)
    if emb == "me":
        ch = A.me_chains(N)
        for i in range(N):
            assert sorted(ch[i]) == sorted(pb.chain_sites[i * (pb.Lc + 1):(i + 1) * (pb.Lc + 1)])


@pytest.mark.parametrize("N,seed", [(4, 1), (6, 2), (8, 3), (8, 11)])
def test_logical_ground_states_brute_force(N, seed):
    J = W.random_couplings(N, seed)
    e_min, G = A.logical_ground_states(N, J)
    assert e_min == O.ground_energy(N, J)[0]
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N)]
    want = set()
    best = None
    for q in itertools.product((1, -1), repeat=N):
        e = sum(int(J[k]) * q[i] * q[j] for k, (i, j) in enumerate(pairs))
        if best is None or e < best:
            best, want = e, {q}
        elif e == best:
            want.add(q)
    assert best == e_min
    assert {tuple(int(x) for x in g) for g in G} == want


def _unique_ground_instance(N, seed0):
    for seed in range(seed0, seed0 + 200):
        J = W.random_couplings(N, seed)
        if len(A.logical_ground_states(N, J)[1]) == 2:
            return J
    raise AssertionError("no instance with a unique ground pair")


@pytest.mark.parametrize("emb,N", [("lhz", 7), ("me", 8)])
def test_error_rates(emb, N):
    J = _unique_ground_instance(N, 40)
    _, G = A.logical_ground_states(N, J)
    phys = np.stack([A.embed_logical(emb, N, g) for g in G])
    used = phys[0] != 0
    n_used = int(used.sum())
    assert np.all(A.error_rates(emb, N, J, phys) == 0.0)
    one = phys[:1].copy()
    site = int(np.flatnonzero(used)[3])
    one[0, site] = -one[0, site]
    assert A.error_rates(emb, N, J, one)[0] == pytest.approx(1.0 / n_used)
    rng = np.random.default_rng(5)
    states = np.where(rng.random((20, phys.shape[1])) < 0.3, -phys[0], phys[0]).astype(np.int8)
    got = A.error_rates(emb, N, J, states)
    for s, r in zip(states, got):
        want = min(int(np.count_nonzero(s[used] != g[used])) for g in phys) / n_used
        assert r == pytest.approx(want)


@pytest.mark.parametrize("N", [3, 5, 8, 12])
def test_corner_distance_is_the_constraint_graph_distance(N):
    d = A.lhz_corner_distance(N)
    assert [int(np.count_nonzero(d == k)) for k in range(N - 1)] == [k + 1 for k in range(N - 1)]
    pb = O.Problem("lhz", N, W.random_couplings(N, 0), 9)
    nbr = {k: set() for k in range(pb.n)}
    for mem, _ in pb.terms():
        for a in mem:
            nbr[a].update(m for m in mem if m != a)
    start = A.lhz_index(N, 0, 1)
    bfs = {start: 0}
    todo = deque([start])
    while todo:
        a = todo.popleft()
        for b in nbr[a]:
            if b not in bfs:
                bfs[b] = bfs[a] + 1
                todo.append(b)
    assert all(bfs[k] == d[k] for k in range(pb.n))


def test_error_by_distance_planted_and_uniform():
    N = 8
    J = _unique_ground_instance(N, 70)
    _, G = A.logical_ground_states(N, J)
    g = A.embed_logical("lhz", N, G[0])
    dist = A.lhz_corner_distance(N)
    assert np.all(A.error_by_distance(N, J, g[None, :]) == 0.0)
    planted = np.where(dist == 3, -g, g)[None, :].astype(np.int8)
    prof = A.error_by_distance(N, J, planted)
    assert prof[3] == 1.0 and np.all(np.delete(prof, 3) == 0.0)
    rng = np.random.default_rng(9)
    noisy = A.uncorrelated_states("lhz", N, J, 0.1, 4000, rng)
    prof = A.error_by_distance(N, J, noisy)
    assert prof.shape == (N - 1,)
    assert np.all(np.abs(prof - 0.1) < 0.04), prof            # flat: no distance dependence
    assert np.mean(A.error_rates("lhz", N, J, noisy)) == pytest.approx(0.1, abs=0.01)


def test_polynomial_fit_and_cutoff():
    c = A.fit_coefficients(np.full(7, 0.25))
    assert c.shape == (7,) and c[0] == pytest.approx(0.25) and np.allclose(c[1:], 0.0, atol=1e-9)
    want = np.array([0.1, -0.2, 0.05, 0.01, -0.003, 0.0004, -0.00002])
    d = np.arange(7.0)
    y = sum(want[k] * d ** k for k in range(7))
    assert np.allclose(A.fit_coefficients(y), want, atol=1e-9)    # 7 distances: degree 6 interpolates
    c5 = A.fit_coefficients(np.array([0.1, 0.2, 0.3, 0.4, 0.5]))  # K_6: five distances, degree 4
    assert c5.shape == (7,) and np.allclose(c5, [0.1, 0.1, 0, 0, 0, 0, 0], atol=1e-9)
    flat = np.full(7, 0.2)                                          # cutoff 0.2 - 2 * 0
    assert list(A.coefficients_above([0.3, 0.1, 0.15, 0.25, -1, 0, 0.21], flat)) == \
        [True, False, False, True, False, False, True]
    spread = np.array([0.1, 0.3, 0.1, 0.3, 0.1, 0.3, 0.1])         # mean 0.186, std 0.099
    assert list(A.coefficients_above([0.0, -0.02, 0.1], spread)) == [True, False, True]
