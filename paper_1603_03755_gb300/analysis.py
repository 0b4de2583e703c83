"""Host-side analyses of sampled states (arXiv:1603.03755, App. D and App. E).

Statistics over what the GPU path returns (physical energies and readouts);
no part of the sampler runs here.

- energy_distance: the total-variation distance between the empirical
  distributions of physical energy of two sets of states (App. D, the
  distance between the SQA and PT states).
- logical_ground_states, embed_logical, error_rates: the average error rate
  (App. E): for each state, the fewest spin flips to the nearest physical
  state of a degenerate logical ground state, divided by the number of
  physical spins.
- lhz_corner_distance, error_by_distance, uncorrelated_states,
  fit_coefficients, coefficients_above: the distance dependence of the error
  probability on the LHZ graph, against uncorrelated noise of the same mean
  rate, through a degree-6 polynomial fit and a cutoff (App. E).

States are sigma = +1 / -1 arrays [n_states, n_phys] in canonical site order
(as `unpack_words` gives them for one instance, transposed); sites the
embedding does not use are ignored.
"""
from __future__ import annotations

import numpy as np


def energy_distance(e_a, e_b) -> float:
    """D(p, q) = 1/2 sum_E |p(E) - q(E)| (App. D) with p, q the fractions of
    the states of each set at each physical energy E."""
    a = np.asarray(e_a).ravel()
    b = np.asarray(e_b).ravel()
    if a.size == 0 or b.size == 0:
        raise ValueError("both sets need at least one state")
    levels = np.union1d(a, b)
    p = np.array([np.count_nonzero(a == E) for E in levels], np.float64) / a.size
    q = np.array([np.count_nonzero(b == E) for E in levels], np.float64) / b.size
    return 0.5 * float(np.abs(p - q).sum())


def _pairs(N: int):
    return [(i, j) for i in range(N) for j in range(i + 1, N)]


def lhz_index(N: int, i: int, j: int) -> int:
    """Canonical index of LHZ pair spin (i, j), i < j."""
    return i * N - i * (i + 1) // 2 + (j - i - 1)


def me_chains(N: int) -> list[list[int]]:
    """Canonical sites of each logical spin's chain in the minor embedding on
    an Lc x Lc Chimera, Lc = ceil(N/4): site ((r Lc + c) 2 + u) 4 + k,
    chain(i) = vertical shore of column g from row 0 to g, then horizontal
    shore of row g from column g on (g = i/4, k = i%4)."""
    Lc = (N + 3) // 4

    def site(r, c, u, k):
        return ((r * Lc + c) * 2 + u) * 4 + k

    chains = []
    for i in range(N):
        g, m = divmod(i, 4)
        chains.append([site(r, g, 0, m) for r in range(g + 1)] + [site(g, c, 1, m) for c in range(g, Lc)])
    return chains


def embed_logical(embedding: str, N: int, q) -> np.ndarray:
    """Physical state [n_phys] of logical state q (+1 / -1): LHZ pair spins
    q_i q_j; ME chains equal to their logical spin; unused sites 0."""
    q = np.asarray(q, np.int64)
    if embedding == "lhz":
        out = np.zeros(N * (N - 1) // 2, np.int8)
        for i, j in _pairs(N):
            out[lhz_index(N, i, j)] = q[i] * q[j]
        return out
    Lc = (N + 3) // 4
    out = np.zeros(8 * Lc * Lc, np.int8)
    for i, ch in enumerate(me_chains(N)):
        out[ch] = q[i]
    return out


def logical_ground_states(N: int, J) -> tuple[int, np.ndarray]:
    """Minimum of sum_{i<j} J_ij q_i q_j (Eq. 1, h = 0) and every logical
    state reaching it, both Z2 partners, [n_ground, N] in the order of the
    enumeration (q_{N-1} = +1 halves first, then their negations).  The
    2^(N-1) states are enumerated in chunks; N <= 26."""
    if not 2 <= N <= 26:
        raise ValueError("exhaustive enumeration needs 2 <= N <= 26")
    J = np.asarray(J, np.int64)
    pairs = _pairs(N)
    e_min, found = None, []
    chunk = 1 << 16
    for x0 in range(0, 1 << (N - 1), chunk):
        x = np.arange(x0, min(x0 + chunk, 1 << (N - 1)), dtype=np.int64)
        Q = np.ones((x.size, N), np.int64)
        for i in range(N - 1):
            Q[:, i] = np.where((x >> i) & 1, -1, 1)
        E = np.zeros(x.size, np.int64)
        for k, (i, j) in enumerate(pairs):
            E += J[k] * Q[:, i] * Q[:, j]
        m = int(E.min())
        if e_min is None or m < e_min:
            e_min, found = m, [Q[E == m]]
        elif m == e_min:
            found.append(Q[E == m])
    G = np.concatenate(found)
    return e_min, np.concatenate([G, -G]).astype(np.int8)


def _ground_phys(embedding: str, N: int, ground: np.ndarray) -> np.ndarray:
    G = np.stack([embed_logical(embedding, N, q) for q in ground])
    return np.unique(G, axis=0) if embedding == "lhz" else G   # LHZ: q and -q give one state


def _nearest(states: np.ndarray, G: np.ndarray, used: np.ndarray):
    s = np.asarray(states, np.int8)[:, used]
    g = G[:, used]
    dist = (s[:, None, :] != g[None, :, :]).sum(axis=2)     # [n_states, n_ground]
    k = dist.argmin(axis=1)                                  # first of equally near states
    return dist[np.arange(len(s)), k], g[k], s


def error_rates(embedding: str, N: int, J, states) -> np.ndarray:
    """Per state: the fewest spin flips to the physical state of a degenerate
    logical ground state, over the embedding's used sites, divided by their
    number (App. E; the average error rate of an instance is the mean)."""
    _, ground = logical_ground_states(N, J)
    G = _ground_phys(embedding, N, ground)
    used = G[0] != 0
    d, _, _ = _nearest(states, G, used)
    return d / float(used.sum())


def lhz_corner_distance(N: int) -> np.ndarray:
    """Distance of each LHZ pair spin (i, j) from the corner spin (0, 1), in
    canonical order: j - 1, the graph distance when spins that share a
    constraint are neighbours (spin (i, j) is d = j - 1 constraints away;
    there are d + 1 spins at distance d, d = 0 .. N - 2)."""
    out = np.zeros(N * (N - 1) // 2, np.int64)
    for i, j in _pairs(N):
        out[lhz_index(N, i, j)] = j - 1
    return out


def error_by_distance(N: int, J, states) -> np.ndarray:
    """Probability that an LHZ spin at distance d from the corner differs from
    the nearest ground state (App. E), d = 0 .. N - 2: the mean over the states
    and over the d + 1 spins at distance d."""
    _, ground = logical_ground_states(N, J)
    G = _ground_phys("lhz", N, ground)
    used = np.ones(G.shape[1], bool)
    _, g, s = _nearest(states, G, used)
    err = (s != g).astype(np.float64).mean(axis=0)
    dist = lhz_corner_distance(N)
    return np.array([err[dist == d].mean() for d in range(N - 1)])


def uncorrelated_states(embedding: str, N: int, J, rate: float, n_states: int, rng) -> np.ndarray:
    """Reference noise (App. E): the physical state of the first logical
    ground state with every used spin flipped independently with
    probability `rate`, n_states times."""
    _, ground = logical_ground_states(N, J)
    g0 = embed_logical(embedding, N, ground[0])
    used = g0 != 0
    flips = rng.random((n_states, g0.size)) < rate
    out = np.where(flips & used[None, :], -g0[None, :], g0[None, :])
    return out.astype(np.int8)


def fit_coefficients(err_by_d, degree: int = 6) -> np.ndarray:
    """Least-squares polynomial in d of the error profile, coefficients of
    d^0 .. d^degree (degree capped at the number of distances - 1; with
    K_8's seven distances, degree 6 interpolates)."""
    y = np.asarray(err_by_d, np.float64)
    deg = min(degree, y.size - 1)
    c = np.polynomial.polynomial.polyfit(np.arange(y.size, dtype=np.float64), y, deg)
    return np.pad(c, (0, degree - deg))


def coefficients_above(coeffs, uncorrelated_err_by_d) -> np.ndarray:
    """Which coefficients count (App. E): those above the cutoff, the mean over
    distance of the uncorrelated error profile minus twice its standard
    deviation over distance."""
    u = np.asarray(uncorrelated_err_by_d, np.float64)
    cutoff = u.mean() - 2.0 * u.std()
    return np.asarray(coeffs) > cutoff
