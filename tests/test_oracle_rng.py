"""Pins of the oracle's random numbers.

Philox4x32-10 is checked against the published known-answer vectors
(tests/golden/philox4x32_10_kat.txt); the per-attempt uniform, the swap
uniform and the initial spins are checked for the documented composition and
for uniformity.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
DOM_SWEEP_HI, DOM_SWEEP_LO = 0xBB67AE85, 0x3C6EF372


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    assert list(O.philox4x32_10(ctr, key)) == want


def test_philox_key_and_counter_sensitivity():
    base = O.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(O.philox4x32_10(c, [5, 6]), base)
    assert not np.array_equal(O.philox4x32_10([1, 2, 3, 4], [5, 7]), base)


def test_sweep_uniform_composition():
    """u = h * 2^25 + l: h the low 7 bits of byte (r/8) of word r%4 of the
    SWEEP_HI block at (t, slot, 2(rho/32) + (r/4)%2, inst), r = rho%32; l word
    rho%4 of the SWEEP_LO block at (t, slot, rho/4, inst), shifted right by 7."""
    seed = 0x0123456789ABCDEF
    key_hi = [seed & 0xFFFFFFFF, (seed >> 32) ^ DOM_SWEEP_HI]
    key_lo = [seed & 0xFFFFFFFF, (seed >> 32) ^ DOM_SWEEP_LO]
    for (t, slot, rho, inst) in [(0, 0, 0, 0), (7, 33, 13, 2), (99, 1000, 255, 1023), (5, 6, 38, 7)]:
        r = rho % 32
        a = O.philox4x32_10([t, slot, 2 * (rho // 32) + (r // 4) % 2, inst], key_hi)
        b = O.philox4x32_10([t, slot, rho // 4, inst], key_lo)
        h = (int(a[r % 4]) >> (8 * (r // 8))) & 0x7F
        lo = int(b[rho % 4]) >> 7
        assert O.sweep_uniform(seed, t, slot, rho, inst) == (h << 25) | lo


def test_sweep_uniform_streams_cover_every_replica_once():
    """The 32 replicas of a word take 32 distinct (block, word, byte) places of
    the two SWEEP_HI blocks, and 32 distinct (block, word) places of SWEEP_LO."""
    hi = {(2 * (rho // 32) + (rho % 32 // 4) % 2, rho % 4, rho % 32 // 8) for rho in range(64)}
    lo = {(rho // 4, rho % 4) for rho in range(64)}
    assert len(hi) == 64 and len(lo) == 64


def test_sweep_uniform_is_uniform():
    u = np.array([O.sweep_uniform(5, t, s, r, 0) for t in range(20) for s in range(10)
                  for r in range(64)], np.float64) / 2.0**32
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # the 7-bit high part is uniform over its 128 values
    h = np.floor(u * 128).astype(np.int64)
    assert stats.chisquare(np.bincount(h, minlength=128)).pvalue > 1e-3
    # high and low parts are independent streams
    lo = u * 128 - h
    assert abs(np.corrcoef(h, lo)[0, 1]) < 0.03
    # replicas of one word that share a SWEEP_HI word are not correlated
    a = np.array([O.sweep_uniform(8, t, 3, 0, 1) for t in range(3000)], np.float64)
    b = np.array([O.sweep_uniform(8, t, 3, 8, 1) for t in range(3000)], np.float64)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.06


def test_swap_uniform_is_uniform():
    u = np.array([O.swap_uniform(9, e, p, r, 3) for e in range(50) for p in range(8)
                  for r in range(32)], np.float64) / 2.0**32
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_init_spins_balanced_and_unused_up():
    J = np.ones(28, np.int32)
    pb = O.Problem("me", 8, J, 2)
    s = O.init_spins(pb, 4, 96, seed=11, inst=3)
    assert s.shape == (4, 32, 96)
    assert np.all(s[:, pb.used == 0, :] == 1)
    frac = np.mean(s[:, pb.used == 1, :] < 0)
    assert abs(frac - 0.5) < 0.02
    # different instance or seed gives a different state
    assert not np.array_equal(s, O.init_spins(pb, 4, 96, seed=11, inst=4))
    assert not np.array_equal(s, O.init_spins(pb, 4, 96, seed=12, inst=3))


def test_tree_draw_range_and_uniformity():
    N = 7
    v = np.array([O.tree_draw(3, i, t, p, N) for i in range(40) for t in range(5) for p in range(5)])
    assert v.min() >= 0 and v.max() < N
    counts = np.bincount(v, minlength=N)
    assert stats.chisquare(counts).pvalue > 1e-3


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(0)
    s = np.where(rng.random((3, 5, 70)) < 0.5, -1, 1).astype(np.int8)
    w = O.pack_bits(s)
    assert w.shape == (3, 5, 3)
    assert np.array_equal(O.unpack_bits(w, 70), s)
    # bits beyond R are zero
    assert np.all((w[..., 2] >> 6) == 0)
