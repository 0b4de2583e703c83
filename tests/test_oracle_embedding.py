"""Pins of the oracle's embeddings (Sec. II A/B of the paper).

Counts the paper states, Chimera structure, proper colourings, and the
energy identities of constraint-satisfying states, checked exhaustively on
small N:
  E_ME(embed s)  = E_log(s) - P * N * Lc        (every chain coupler satisfied)
  E_LHZ(embed s) = E_log(s) - lambda * C(N-1,2) (every constraint satisfied)
and, for LHZ, exactly 2^(N-1) of the 2^C(N,2) physical states satisfy every
constraint.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _logical_energy_bruteforce(N, J, s):
    e = 0
    k = 0
    for i in range(N):
        for j in range(i + 1, N):
            e += int(J[k]) * int(s[i]) * int(s[j])
            k += 1
    return e


@pytest.mark.parametrize("N", [2, 3, 4, 5, 7, 8, 9, 12, 16, 32])
def test_me_counts(N):
    J = W.random_couplings(N, N)
    pb = O.Problem("me", N, J, 6)
    Lc = math.ceil(N / 4)
    assert pb.n == 8 * Lc * Lc
    assert int(pb.used.sum()) == N * (Lc + 1)          # N(ceil(N/4)+1) used spins
    if N % 4 == 0:
        assert pb.n == N * N // 2                        # 8 L^2 = N^2/2
    chains = pb.chain_sites.reshape(N, Lc + 1)
    assert len(set(chains.ravel().tolist())) == N * (Lc + 1)  # chains disjoint
    assert pb.n_terms == N * (N - 1) // 2 + N * Lc


def _chimera_coords(site, Lc):
    k = site % 4
    u = (site // 4) % 2
    cell = site // 8
    return cell // Lc, cell % Lc, u, k


def _is_chimera_edge(a, b, Lc):
    ra, ca, ua, ka = _chimera_coords(a, Lc)
    rb, cb, ub, kb = _chimera_coords(b, Lc)
    if (ra, ca) == (rb, cb):
        return ua != ub                                  # K_{4,4} inside a cell
    if ua != ub or ka != kb:
        return False
    if ua == 0:
        return ca == cb and abs(ra - rb) == 1            # vertical shore couples up/down
    return ra == rb and abs(ca - cb) == 1                # horizontal shore couples left/right


@pytest.mark.parametrize("N", [4, 5, 8, 11, 16, 32])
def test_me_structure(N):
    J = W.random_couplings(N, 100 + N)
    pb = O.Problem("me", N, J, 4)
    Lc = pb.Lc
    chains = pb.chain_sites.reshape(N, Lc + 1)
    owner = {int(s): i for i in range(N) for s in chains[i]}
    logical_pairs = set()
    deg = np.zeros(pb.n, int)
    for mem, w in pb.terms():
        assert len(mem) == 2
        a, b = mem
        assert _is_chimera_edge(a, b, Lc), (a, b)
        deg[a] += 1
        deg[b] += 1
        if owner[a] == owner[b]:
            assert w == -4                               # ferromagnetic chain penalty
        else:
            i, j = sorted((owner[a], owner[b]))
            assert (i, j) not in logical_pairs           # one coupler per logical pair
            logical_pairs.add((i, j))
            assert w == J[O.lhz_index(N, i, j)]
    assert len(logical_pairs) == N * (N - 1) // 2
    assert deg.max() <= 6                                # Chimera has degree six
    # each chain is connected through its own couplers
    for i in range(N):
        members = set(int(s) for s in chains[i])
        adj = {s: set() for s in members}
        for mem, w in pb.terms():
            if set(mem) <= members:
                adj[mem[0]].add(mem[1])
                adj[mem[1]].add(mem[0])
        seen, stack = {int(chains[i][0])}, [int(chains[i][0])]
        while stack:
            v = stack.pop()
            for x in adj[v] - seen:
                seen.add(x)
                stack.append(x)
        assert seen == members
        assert int(pb.hub[i]) in members


@pytest.mark.parametrize("N", [2, 3, 4, 6, 8, 16, 24])
def test_lhz_counts(N):
    J = W.random_couplings(N, N)
    pb = O.Problem("lhz", N, J, 5)
    K = N * (N - 1) // 2
    Cn = (N - 1) * (N - 2) // 2
    assert pb.n == K and int(pb.used.sum()) == K
    sizes = [len(mem) for mem, w in pb.terms() if len(mem) > 1]
    assert len(sizes) == Cn                              # C = binom(N-1, 2)
    assert sizes.count(3) == max(0, N - 2)               # 3-body at the boundary
    assert sizes.count(4) == Cn - max(0, N - 2)
    fields = [(mem[0], w) for mem, w in pb.terms() if len(mem) == 1]
    assert len(fields) == K
    for k, w in fields:
        assert w == J[k]                                 # J_k is the local field of q_k
    for mem, w in pb.terms():
        if len(mem) > 1:
            assert w == -5


def test_lhz_uses_more_spins_than_me():
    """Sec. III A states N(N-1)/2 > N(ceil(N/4)+1) for N >= 8.  It holds with
    equality at N = 9 (36 spins each) and strictly for every other N >= 8."""
    for N in range(8, 200):
        lhz, me = N * (N - 1) // 2, N * (math.ceil(N / 4) + 1)
        if N == 9:
            assert lhz == me == 36
        else:
            assert lhz > me


@pytest.mark.parametrize("emb,N", [("me", 4), ("me", 8), ("me", 13), ("me", 32),
                                   ("lhz", 3), ("lhz", 6), ("lhz", 11), ("lhz", 24)])
def test_colouring_is_proper(emb, N):
    pb = O.Problem(emb, N, W.random_couplings(N, 1), 3)
    for mem, w in pb.terms():
        cols = [int(pb.colour[m]) for m in mem]
        assert all(c >= 0 for c in cols)
        assert len(set(cols)) == len(cols)
    assert np.all((pb.colour >= 0) == (pb.used == 1))


@pytest.mark.parametrize("N", range(2, 11))
def test_me_energy_identity_exhaustive(N):
    J = W.random_couplings(N, 7 * N)
    P = 5
    pb = O.Problem("me", N, J, P)
    for bits in range(2 ** N):
        s = np.array([-1 if (bits >> i) & 1 else 1 for i in range(N)], np.int8)
        phys = pb.embed(s)
        assert pb.energy(phys) == _logical_energy_bruteforce(N, J, s) - P * N * pb.Lc
        assert np.array_equal(O.me_decode(pb, phys), s)


@pytest.mark.parametrize("N", range(2, 11))
def test_lhz_energy_identity_exhaustive(N):
    J = W.random_couplings(N, 11 * N)
    lam = 4
    pb = O.Problem("lhz", N, J, lam)
    Cn = (N - 1) * (N - 2) // 2
    for bits in range(2 ** N):
        s = np.array([-1 if (bits >> i) & 1 else 1 for i in range(N)], np.int8)
        phys = pb.embed(s)
        assert pb.energy(phys) == _logical_energy_bruteforce(N, J, s) - lam * Cn


@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_lhz_constraint_satisfying_states(N):
    """Exactly 2^(N-1) physical states satisfy every constraint, and they are
    the images of the logical states."""
    J = W.random_couplings(N, N)
    pb = O.Problem("lhz", N, J, 1)
    K = pb.n
    cons = [mem for mem, w in pb.terms() if len(mem) > 1]
    states = np.array(list(itertools.product([1, -1], repeat=K)), np.int8)
    ok = np.ones(len(states), bool)
    for mem in cons:
        ok &= np.prod(states[:, mem], axis=1) == 1
    assert ok.sum() == 2 ** (N - 1)
    images = {tuple(pb.embed(np.array([1] + [-1 if (b >> i) & 1 else 1 for i in range(N - 1)])))
              for b in range(2 ** (N - 1))}
    assert images == {tuple(x) for x in states[ok]}


@pytest.mark.parametrize("emb,N", [("me", 5), ("me", 8), ("lhz", 5), ("lhz", 7)])
def test_flip_delta_is_energy_difference(emb, N):
    pb = O.Problem(emb, N, W.random_couplings(N, 3), 4)
    rng = np.random.default_rng(N)
    for _ in range(30):
        s = np.where(rng.random(pb.n) < 0.5, -1, 1).astype(np.int8)
        s[pb.used == 0] = 1
        e0 = pb.energy(s)
        for site in np.flatnonzero(pb.used):
            t = s.copy()
            t[site] = -t[site]
            assert pb.flip_delta(s, int(site)) == pb.energy(t) - e0


def test_delta_range_bounds_every_flip():
    for emb, N in [("me", 8), ("lhz", 6)]:
        pb = O.Problem(emb, N, W.random_couplings(N, 5), 9 if emb == "lhz" else 6)
        lo, hi = pb.delta_range()
        rng = np.random.default_rng(1)
        for _ in range(200):
            s = np.where(rng.random(pb.n) < 0.5, -1, 1).astype(np.int8)
            for site in np.flatnonzero(pb.used):
                d = pb.flip_delta(s, int(site))
                assert lo <= d <= hi and d % 2 == 0
