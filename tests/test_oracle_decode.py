"""Pins of the oracle's decoders and ground-state search.

  - the star and chain trees reproduce the paper's closed forms (App. A,
    Eqs. 10-11) on arbitrary (leaked) physical states;
  - every tree decoder is exact on constraint-satisfying states (App. A);
  - Pruefer trees are spanning trees, and uniform over the N^(N-2) labelled
    trees (Cayley) for N = 4;
  - ME majority vote follows Eq. 4 with the hub breaking ties;
  - the ground-state enumeration agrees with a brute force over all 2^N
    states written independently here.
"""
import itertools
from collections import Counter

import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W


def _random_phys(pb, rng):
    s = np.where(rng.random(pb.n) < 0.5, -1, 1).astype(np.int8)
    s[pb.used == 0] = 1
    return s


@pytest.mark.parametrize("N", [2, 3, 5, 8, 16])
def test_star_and_chain_closed_forms(N):
    pb = O.Problem("lhz", N, W.random_couplings(N, 2), 3)
    rng = np.random.default_rng(N)
    for _ in range(20):
        q = _random_phys(pb, rng)
        star = O.lhz_tree_decode(N, O.star_tree(N), q)
        want_star = [1] + [int(q[O.lhz_index(N, 0, i)]) for i in range(1, N)]   # Eq. 11
        assert star.tolist() == want_star
        chain = O.lhz_tree_decode(N, O.chain_tree(N), q)
        want_chain = [int(np.prod([q[O.lhz_index(N, m, m + 1)] for m in range(i)]))
                      for i in range(N)]                                          # Eq. 10
        assert chain.tolist() == want_chain


@pytest.mark.parametrize("N", [3, 6, 9, 16])
def test_tree_decoders_exact_without_leakage(N):
    pb = O.Problem("lhz", N, W.random_couplings(N, 3), 3)
    rng = np.random.default_rng(1)
    trees = [O.star_tree(N), O.chain_tree(N)] + [O.prufer_tree(N, 5, 0, t) for t in range(7)]
    for _ in range(25):
        s = np.where(rng.random(N) < 0.5, -1, 1).astype(np.int8)
        phys = pb.embed(s)
        gauge = s * s[0]                                  # q_0 fixed to +1
        for p in trees:
            assert np.array_equal(O.lhz_tree_decode(N, p, phys), gauge)
        assert np.array_equal(O.lhz_vote_decode(N, np.stack(trees[2:]), phys), gauge)


@pytest.mark.parametrize("N", [2, 3, 7, 12])
def test_prufer_gives_spanning_trees(N):
    for t in range(20):
        parent = O.prufer_tree(N, 77, 3, t)
        assert parent[0] == -1
        for v in range(1, N):
            seen, x = set(), v
            while x != 0:
                assert x not in seen
                seen.add(x)
                x = int(parent[x])
                assert 0 <= x < N


def test_prufer_trees_uniform_n4():
    """Cayley: 4^2 = 16 labelled trees on 4 vertices, drawn uniformly."""
    N = 4
    counts = Counter()
    for inst in range(400):
        for t in range(10):
            p = O.prufer_tree(N, 123, inst, t)
            edges = frozenset(frozenset((v, int(p[v]))) for v in range(1, N))
            counts[edges] += 1
    assert len(counts) == 16
    assert stats.chisquare(list(counts.values())).pvalue > 1e-3


def test_vote_over_trees_majority():
    N = 5
    pb = O.Problem("lhz", N, W.random_couplings(N, 9), 2)
    rng = np.random.default_rng(4)
    trees = np.stack([O.prufer_tree(N, 1, 0, t) for t in range(5)])
    for _ in range(50):
        q = _random_phys(pb, rng)
        each = np.stack([O.lhz_tree_decode(N, p, q) for p in trees]).astype(int)
        want = np.sign(each.sum(axis=0))                  # Eq. 5; 5 votes never tie
        assert np.array_equal(O.lhz_vote_decode(N, trees, q), want)


def test_two_tree_vote_is_the_first_tree():
    """With an even number of trees a vertex can tie; a tie takes the first
    tree's value (reading of Eq. 5).  So a two-tree vote is the first tree's
    decode, on any state, with or without leakage."""
    N = 7
    pb = O.Problem("lhz", N, W.random_couplings(N, 5), 2)
    rng = np.random.default_rng(8)
    trees = np.stack([O.prufer_tree(N, 3, 0, t) for t in range(2)])
    ties = 0
    for _ in range(100):
        q = _random_phys(pb, rng)
        a, b = (O.lhz_tree_decode(N, p, q) for p in trees)
        ties += int((a != b).sum())
        assert np.array_equal(O.lhz_vote_decode(N, trees, q), a)
        assert np.array_equal(O.lhz_vote_decode(N, trees[::-1].copy(), q), b)
    assert ties > 0                                   # the states did exercise ties


@pytest.mark.parametrize("N", [4, 8, 12, 16])
def test_me_majority_vote(N):
    pb = O.Problem("me", N, W.random_couplings(N, 4), 2)
    rng = np.random.default_rng(N)
    chains = pb.chain_sites.reshape(N, pb.Lc + 1)
    for _ in range(50):
        q = _random_phys(pb, rng)
        out = O.me_decode(pb, q)
        for i in range(N):
            tot = int(q[chains[i]].astype(int).sum())
            want = np.sign(tot) if tot != 0 else int(q[pb.hub[i]])
            assert out[i] == want


def _bruteforce_ground(N, J):
    Jm = np.zeros((N, N))
    Jm[np.triu_indices(N, 1)] = J
    best = None
    for s in itertools.product([1, -1], repeat=N):
        s = np.array(s)
        e = int(s @ Jm @ s)
        best = e if best is None or e < best else best
    return best


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8, 10])
def test_ground_energy_bruteforce(N):
    for seed in range(3):
        J = W.random_couplings(N, 1000 * N + seed)
        e, s = O.ground_energy(N, J)
        assert e == _bruteforce_ground(N, J)
        assert O.logical_energy(N, J, s) == e
        assert O.logical_energy(N, J, -s) == e                # Z2 partner, h = 0


def test_logical_energy_definition():
    N = 5
    J = W.random_couplings(N, 3)
    s = np.array([1, -1, -1, 1, -1], np.int8)
    e = sum(int(J[O.lhz_index(N, i, j)]) * s[i] * s[j] for i in range(N) for j in range(i + 1, N))
    assert O.logical_energy(N, J, s) == e


# ---------------------------------------------------------------------------
# Minimum-weight decoding (Sec. IV A): the constraint-satisfying state nearest
# in Hamming distance to the readout, returned as the logical state with
# q_{N-1} = +1 (the Z2 partner is the same physical state).
# ---------------------------------------------------------------------------

def _all_logical(N):
    x = np.arange(2 ** (N - 1))
    q = np.where((x[:, None] >> np.arange(N - 1)[None, :]) & 1, -1, 1)
    return np.concatenate([q, np.ones((len(x), 1), int)], axis=1)      # binary order, q_{N-1} = +1


@pytest.mark.parametrize("N", [3, 5, 7, 9])
def test_mwd_is_the_nearest_valid_state(N):
    """Brute force over every logical state: the decoded state's pair
    products differ from the readout in the fewest pair spins, and among
    equally near states it is the first in binary order."""
    pb = O.Problem("lhz", N, W.random_couplings(N, 6), 3)
    rng = np.random.default_rng(N)
    Q = _all_logical(N)
    iu = np.triu_indices(N, 1)
    for _ in range(40):
        phys = _random_phys(pb, rng)
        pairs = np.array([phys[O.lhz_index(N, i, j)] for i, j in zip(*iu)])
        dist = ((Q[:, iu[0]] * Q[:, iu[1]]) != pairs[None, :]).sum(axis=1)
        want = Q[int(np.argmin(dist))]                  # argmin takes the first minimum
        assert np.array_equal(O.lhz_mwd_decode(N, phys), want)


@pytest.mark.parametrize("N", [5, 8, 12])
def test_mwd_corrects_flipped_pair_spins(N):
    """Valid states decode to themselves; with fewer than (N-1)/2 flipped pair
    spins (two valid states differ in at least N-1 pair spins) the original
    logical state comes back."""
    pb = O.Problem("lhz", N, W.random_couplings(N, 2), 3)
    rng = np.random.default_rng(3 * N)
    K = N * (N - 1) // 2
    for _ in range(20):
        s = np.where(rng.random(N) < 0.5, -1, 1).astype(np.int8)
        gauge = s * s[N - 1]
        phys = pb.embed(s)
        assert np.array_equal(O.lhz_mwd_decode(N, phys), gauge)
        bad = phys.copy()
        flips = rng.choice(K, size=(N - 2) // 2, replace=False)
        bad[flips] *= -1
        assert np.array_equal(O.lhz_mwd_decode(N, bad), gauge)


# ---------------------------------------------------------------------------
# Belief-propagation decoding (Sec. IV, App. C; reading R21): iterated
# weighted majority over the N-2 parity checks of every pair, then a tree.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [4, 7, 10])
def test_bp_keeps_valid_states_and_corrects_one_flip(N):
    """A valid state is a fixed point; one flipped pair spin is outvoted by
    its N-2 agreeing checks (N >= 5 at error rate 0.2) and the tree reads the
    encoded state."""
    pb = O.Problem("lhz", N, W.random_couplings(N, 4), 3)
    rng = np.random.default_rng(11 * N)
    tree = O.prufer_tree(N, 9, 0, 0)
    K = N * (N - 1) // 2
    for _ in range(15):
        s = np.where(rng.random(N) < 0.5, -1, 1).astype(np.int8)
        gauge = s * s[0]
        phys = pb.embed(s)
        assert np.array_equal(O.lhz_bp_decode(N, phys, 0.2, 10, tree), gauge)
        if N >= 5:
            bad = phys.copy()
            bad[rng.integers(K)] *= -1
            assert np.array_equal(O.lhz_bp_decode(N, bad, 0.2, 10, tree), gauge)


def test_bp_at_error_rate_one_half_is_the_plain_tree():
    """At e = 1/2 a reading and a check carry no weight (L0 = L2 = 0): every
    decision ties, the pair values stay the readout, and BP is the tree
    decoder on the raw readout."""
    N = 8
    pb = O.Problem("lhz", N, W.random_couplings(N, 5), 3)
    rng = np.random.default_rng(2)
    tree = O.prufer_tree(N, 4, 1, 0)
    for _ in range(20):
        phys = _random_phys(pb, rng)
        assert np.array_equal(O.lhz_bp_decode(N, phys, 0.5, 10, tree), O.lhz_tree_decode(N, tree, phys))


@pytest.mark.parametrize("N", [6, 9])
def test_bp_is_gauge_covariant(N):
    """Flipping logical spin k of the encoding flips the N-1 pair spins at k;
    BP must follow: the decoded state flips at k (k != 0, q_0 fixed) and
    nowhere else, on corrupted readouts as well."""
    pb = O.Problem("lhz", N, W.random_couplings(N, 6), 3)
    rng = np.random.default_rng(5 * N)
    tree = O.prufer_tree(N, 2, 0, 0)
    for _ in range(20):
        phys = _random_phys(pb, rng)
        k = int(rng.integers(1, N))
        flipped = phys.copy()
        for l in range(N):
            if l != k:
                flipped[O.lhz_index(N, min(k, l), max(k, l))] *= -1
        a = O.lhz_bp_decode(N, phys, 0.2, 10, tree)
        b = O.lhz_bp_decode(N, flipped, 0.2, 10, tree)
        want = a.copy()
        want[k] *= -1
        assert np.array_equal(b, want)


def test_bp_worked_example_k4():
    """K_4 readout with only pair (0,1) flipped, error rate 0.2, one
    iteration.  Pair (0,1): reading -1 (weight L0 = ln 4 = 1.386), its two
    checks through spins 2 and 3 both say +1 (weight L2 = ln(0.68/0.32) =
    0.754 each): 2 x 0.754 > 1.386, so it turns +1.  Every other pair keeps
    +1 (its checks cancel, its reading decides).  The star tree then reads
    q = (+1, +1, +1, +1); with the checks counted through the pair itself
    (three votes, one of them -1) the flip would survive."""
    N = 4
    phys = np.ones(6, np.int8)
    phys[O.lhz_index(N, 0, 1)] = -1
    star = O.star_tree(N)
    assert O.lhz_bp_decode(N, phys, 0.2, 1, star).tolist() == [1, 1, 1, 1]
    assert O.lhz_tree_decode(N, star, phys).tolist() == [1, -1, 1, 1]   # without BP
    assert math.isclose(math.log(0.8 / 0.2), 1.3862943611198906)
    assert 2 * math.log(0.68 / 0.32) > math.log(4.0) > math.log(0.68 / 0.32)
