"""Penalty scans (Sec. III: Figs. 3, 4, 6 and 7).

For one set of instances, the success probability at every penalty of a
list: the handles of all penalties run as one persistent launch (a Batch,
replayed from a CUDA graph), each readout is decoded on the device and
counted against the exact logical ground state.  From the table:

- the optimal penalty of an instance maximises its success probability
  (Sec. III A; ties go to the smallest penalty);
- the critical penalty is where the success probability first reaches 0.5
  (Sec. III B, for PT at low temperature), interpolated linearly between the
  two scanned penalties around the crossing; NaN when it never does.

Argument marshalling over the C ABI only: every anneal, decode and success
count runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import Batch, Handle, ground_energy


@dataclass
class ScanResult:
    penalties: np.ndarray   # [P]
    success: np.ndarray     # [P, I] success probability per penalty and instance
    optimal: np.ndarray     # [I] optimal penalty
    critical: np.ndarray    # [I] critical penalty (NaN when 0.5 is never reached)
    e_ground: np.ndarray    # [I] exact logical ground-state energies
    attempts: int           # spin-flip attempts of the whole scan


def optimal_penalty(penalties, success) -> np.ndarray:
    """Per instance (columns of success [P, I]) the penalty of the highest
    success probability; the first (smallest) on ties."""
    penalties = np.asarray(penalties, float)
    order = np.argsort(penalties, kind="stable")
    s = np.asarray(success, float)[order]
    return penalties[order][np.argmax(s, axis=0)]


def critical_penalty(penalties, success, level: float = 0.5) -> np.ndarray:
    """Per instance the penalty where the success probability first reaches
    `level` scanning upward, linearly interpolated from the scanned point
    below it; the smallest penalty if it starts at or above `level`, NaN if
    it never gets there."""
    penalties = np.asarray(penalties, float)
    order = np.argsort(penalties, kind="stable")
    p = penalties[order]
    s = np.asarray(success, float)[order]
    out = np.full(s.shape[1], np.nan)
    for i in range(s.shape[1]):
        hit = np.flatnonzero(s[:, i] >= level)
        if len(hit) == 0:
            continue
        k = int(hit[0])
        if k == 0:
            out[i] = p[0]
            continue
        s0, s1 = s[k - 1, i], s[k, i]
        out[i] = p[k - 1] + (level - s0) * (p[k] - p[k - 1]) / (s1 - s0)
    return out


def penalty_scan(*, embedding: str, N: int, J, penalties, R: int, sweeps: int, seed: int = 0, kind: str = "sqa",
                 method: str | None = None, n_trees: int = 0, autotune: bool = False, stream=None,
                 **anneal) -> ScanResult:
    """Run every penalty of `penalties` (positive integers) on the instances
    J [I, N(N-1)/2] as one batch and decode every readout.  `anneal` holds the
    sampler's own keywords (SQA: L, beta, A, B, move; PT: betas,
    swap_every).  All penalties share the seed, so they see the same random
    numbers."""
    J = np.ascontiguousarray(np.atleast_2d(np.asarray(J, np.int32)))
    pens = [int(p) for p in penalties]
    if not pens or min(pens) <= 0:
        raise ValueError("penalties must be positive integers")
    e_ground = ground_energy(N, J)
    handles = [Handle(embedding=embedding, N=N, J=J, penalty=p, sweeps=sweeps, R=R, seed=seed, kind=kind, **anneal)
               for p in pens]
    try:
        batch = Batch(handles)
        try:
            if autotune:
                batch.autotune(stream=stream)
            batch.launch(stream=stream)
            counts = []
            for h in handles:
                _, _, succ = h.decode(method, n_trees, e_ground=e_ground, stream=stream)
                counts.append(succ)
        finally:
            batch.close()
        attempts = sum(h.info["attempts_per_sweep"] for h in handles) * sweeps
    finally:
        for h in handles:
            h.close()
    success = np.stack(counts).astype(float) / R
    return ScanResult(np.array(pens, float), success, optimal_penalty(pens, success),
                      critical_penalty(pens, success), e_ground, int(attempts))
