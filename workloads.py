"""Seeded synthetic inputs for the SQA / PT hot path.

This module is the only code shared by the CPU oracle side (``oracle/``, the
tests) and the GPU side (the ``paper_1603_03755_gb300`` package, ``bench.py``).
It holds no arithmetic of the method itself: it draws random logical Ising
instances, lists the workload shapes, and writes down the paper's temperature
ladder as an input recipe.

Instance class (Sec. III of the paper): fully connected logical problems
K_N with couplings J_ij drawn iid and uniformly from a symmetric set, all local
fields zero.  The paper uses {+-0.1, ..., +-1}; the workloads here use the
integer set {+-1, +-2, +-3} so every energy is an exact integer.  The paper's
100 K_8 / K_16 instances are not published; these seeded draws stand in for
them.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), a
published 64-bit generator, restated here.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
J_VALUES_INT = (-3, -2, -1, 1, 2, 3)


class SplitMix64:
    """SplitMix64: state += golden gamma, then two xor-shift-multiply mixes."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def n_pairs(N: int) -> int:
    return N * (N - 1) // 2


def random_couplings(N: int, seed: int, values=J_VALUES_INT) -> np.ndarray:
    """One instance: J_ij for i<j in row-major upper-triangle order, int32.

    Each J_ij is ``values[x % len(values)]`` for the next SplitMix64 output x.
    """
    g = SplitMix64(seed)
    k = len(values)
    return np.array([values[g.next() % k] for _ in range(n_pairs(N))], dtype=np.int32)


def instance_seed(config_seed: int, instance: int) -> int:
    """Per-instance generator seed: the workload seed xor the instance id."""
    return (config_seed ^ instance) & MASK64


def random_instances(N: int, n_inst: int, config_seed: int = 0) -> np.ndarray:
    """``n_inst`` instances of K_N, shape [n_inst, N(N-1)/2], int32."""
    out = np.empty((n_inst, n_pairs(N)), dtype=np.int32)
    for i in range(n_inst):
        out[i] = random_couplings(N, instance_seed(config_seed, i))
    return out


def paper_beta_ladder(P: int = 64, beta_1: float = 20.0, beta_P: float = 0.1) -> np.ndarray:
    """The paper's PT ladder (App. B): beta_i = beta_1 (beta_P/beta_1)^((i-1)/(P-1)), i=1..P.

    Coldest first, strictly decreasing.
    """
    i = np.arange(1, P + 1, dtype=np.float64)
    return beta_1 * (beta_P / beta_1) ** ((i - 1.0) / (P - 1.0))


def geometric_ladder(P: int, beta_cold: float, beta_hot: float) -> np.ndarray:
    """P temperatures geometric in beta from ``beta_cold`` down to ``beta_hot``."""
    if P == 1:
        return np.array([beta_cold], dtype=np.float64)
    return paper_beta_ladder(P, beta_cold, beta_hot)


def max_abs(J: np.ndarray) -> int:
    return int(np.max(np.abs(J))) if J.size else 1


# ---------------------------------------------------------------------------
# Workload shapes.  Each is a plain dict; ``J`` is drawn on demand.
# ---------------------------------------------------------------------------

def lhz_n6_config() -> dict:
    """Plain SQA, LHZ embedding of one K_6 instance (seed 0): 15 physical spins,
    10 plaquettes, C = 3 max|J|, linear schedule, beta = 10/max|J|, L = 32,
    1000 sweeps, 64 replicas."""
    N = 6
    J = random_instances(N, 1, 0)
    m = max_abs(J)
    return dict(name="lhz_n6_l32_r64_s1000", embedding="lhz", N=N, J=J, penalty=3 * m,
                beta=10.0 / m, L=32, R=64, sweeps=1000, seed=0)


def me_n8_batch_config(n_inst: int = 1024, R: int = 256, L: int = 64, sweeps: int = 10_000) -> dict:
    """Plain SQA batched, ME of K_8 on a 2x2 Chimera (32 sites, chains of 3),
    J_F = -2 max|J|, 1024 instances x 256 replicas, L = 64, 1e4 sweeps."""
    N = 8
    J = random_instances(N, n_inst, 0)
    m = 3  # the value set's max |J|; fixed so every instance shares one table
    return dict(name=f"me_n8_i{n_inst}_r{R}_l{L}_s{sweeps}", embedding="me", N=N, J=J,
                penalty=2 * m, beta=10.0 / m, L=L, R=R, sweeps=sweeps, seed=0)


def ragged_mix_config(n_inst: int = 512, R: int = 128, sweeps: int = 10_000) -> list[dict]:
    """Ragged batch: half LHZ with N in {8,10,12,14,16}, half ME with N in
    {8..16}; L alternating 32/64; R = 128; 1e4 sweeps."""
    jobs = []
    lhz_ns = (8, 10, 12, 14, 16)
    me_ns = tuple(range(8, 17))
    for i in range(n_inst):
        if i % 2 == 0:
            N = lhz_ns[(i // 2) % len(lhz_ns)]
            emb = "lhz"
        else:
            N = me_ns[(i // 2) % len(me_ns)]
            emb = "me"
        L = 32 if (i // 2) % 2 == 0 else 64
        J = random_instances(N, 1, 1000 + i)
        m = 3
        pen = 3 * m if emb == "lhz" else 2 * m
        jobs.append(dict(name=f"ragged_{i}", embedding=emb, N=N, J=J, penalty=pen,
                         beta=10.0 / m, L=L, R=R, sweeps=sweeps, seed=1000 + i))
    return jobs


def pt_config(embedding: str, n_inst: int = 256, R: int = 32, P: int = 32,
              sweeps: int = 100_000) -> dict:
    """Classical PT at zero transverse field: ME K_32 on 8x8 Chimera or LHZ K_24;
    32 temperatures geometric in beta from 10 down to 0.1; swap every sweep."""
    N = 32 if embedding == "me" else 24
    J = random_instances(N, n_inst, 7)
    m = 3
    pen = 2 * m if embedding == "me" else 3 * m
    return dict(name=f"pt_{embedding}_n{N}_i{n_inst}", embedding=embedding, N=N, J=J,
                penalty=pen, betas=geometric_ladder(P, 10.0, 0.1), R=R, sweeps=sweeps,
                swap_every=1, seed=7)


def serving_stream(n_jobs: int, seed: int = 0, max_N: int = 40) -> list[dict]:
    """Poisson-stream job mix: embedding ME or LHZ, N uniform in 6..max_N,
    L in {16,32,64,128}, sweeps log-uniform in [1e3, 1e5], 1-256 replicas,
    kind SQA or PT.  Arrival times are left to the caller (exponential gaps)."""
    g = SplitMix64(seed)

    def unif() -> float:
        return (g.next() >> 11) * (1.0 / (1 << 53))

    jobs = []
    for j in range(n_jobs):
        emb = "me" if g.next() & 1 else "lhz"
        N = 6 + int(unif() * (max_N - 5))
        L = (16, 32, 64, 128)[g.next() % 4]
        sweeps = int(round(math.exp(math.log(1e3) + unif() * (math.log(1e5) - math.log(1e3)))))
        R = 1 + int(unif() * 256)
        kind = "pt" if g.next() & 1 else "sqa"
        J = random_couplings(N, g.next())
        pen = 6 if emb == "me" else 9
        jobs.append(dict(name=f"job{j}", kind=kind, embedding=emb, N=N, J=J, penalty=pen,
                         beta=10.0 / 3.0, L=L, R=R, sweeps=sweeps, seed=g.next(),
                         betas=geometric_ladder(8, 10.0, 0.1), swap_every=1))
    return jobs
