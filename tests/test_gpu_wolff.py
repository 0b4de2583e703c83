"""GPU parity of the time-like cluster (Wolff) move against the oracle.

Spins and energies bit for bit.  Cases span ragged replica tails, ring
lengths that leave lanes partly empty (L = 6, 34, 100) or full (64, 128),
both slices-per-lane variants, an A = 0 stretch (bonds between equal slices
always join), resume at any sweep, words-per-unit shapes and a batch that
mixes cluster-move and single-spin jobs in one launch.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu


def _oracle(emb, N, J, pen, L, R, beta, S, seed, inst, A=None, B=None):
    pb = O.Problem(emb, N, J, pen)
    if A is None:
        A, B = O.linear_schedule(S)
    q = O.SQA(pb, L, R, beta, A, B, seed, inst, move="wolff")
    q.run(0, S)
    return pb, q


def _check(h, emb, N, J, pen, L, R, beta, S, seed, A=None, B=None, insts=None):
    st = pkg.unpack_words(h.state(stream=0), R)
    E = h.energies(stream=0)
    for i in (range(J.shape[0]) if insts is None else insts):
        pb, q = _oracle(emb, N, J[i], pen, L, R, beta, S, seed, i, A, B)
        assert np.array_equal(st[i], q.s), f"instance {i}: spins differ"
        assert np.array_equal(E[i], q.slice_energies()), f"instance {i}: energies differ"


@pytest.mark.parametrize("emb,N,L,R,S", [("lhz", 6, 32, 64, 120), ("me", 8, 64, 70, 40), ("lhz", 5, 6, 33, 150),
                                         ("me", 5, 34, 40, 60), ("lhz", 7, 100, 32, 20), ("me", 6, 128, 20, 12)])
def test_wolff_parity(emb, N, L, R, S):
    pen = 6 if emb == "me" else 9
    J = W.random_instances(N, 2, 40 + L)
    h = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=40 + L, L=L, beta=10 / 3,
                   move="wolff")
    h.run(stream=0)
    _check(h, emb, N, J, pen, L, R, 10 / 3, S, 40 + L)
    h.close()


def test_wolff_infinite_jperp_and_resume():
    """A = 0 for the last sweeps (every bond between equal slices joins);
    the run is split at an arbitrary sweep."""
    N, L, R, S = 6, 16, 48, 60
    J = W.random_instances(N, 2, 7)
    A, B = O.linear_schedule(S)
    A = A.copy()
    A[45:] = 0.0
    h = pkg.Handle(embedding="lhz", N=N, J=J, penalty=9, sweeps=S, R=R, seed=7, L=L, beta=3.0, A=A, B=B,
                   move="wolff")
    h.run_sweeps(0, 23, stream=0)
    h.run_sweeps(23, S, stream=0)
    _check(h, "lhz", N, J, 9, L, R, 3.0, S, 7, A, B)
    h.close()


@pytest.mark.parametrize("wc", [1, 2, 3])
def test_wolff_words_per_unit(wc):
    N, L, R, S = 8, 16, 150, 15                     # 5 words, ragged last word
    J = W.random_instances(N, 2, 12)
    h = pkg.Handle(embedding="me", N=N, J=J, penalty=6, sweeps=S, R=R, seed=12, L=L, beta=3.0, move="wolff")
    h.tune(wc, -1)
    assert h.launch()["words_per_unit"] == wc and h.launch()["cluster"] == 1
    h.run(stream=0)
    _check(h, "me", N, J, 6, L, R, 3.0, S, 12)
    h.close()


def test_wolff_in_a_mixed_batch():
    """The multi-job kernel runs cluster-move and single-spin jobs together."""
    mk = [dict(embedding="lhz", N=6, L=32, R=64, penalty=9, move="wolff"),
          dict(embedding="me", N=8, L=16, R=40, penalty=6, move="metropolis"),
          dict(embedding="me", N=5, L=100, R=32, penalty=6, move="wolff")]
    kws = []
    for k, m in enumerate(mk):
        kws.append(dict(m, J=W.random_instances(m["N"], 2, 60 + k), sweeps=25, seed=60 + k, beta=3.0))
    alone = []
    for kw in kws:
        h = pkg.Handle(**kw)
        h.run(stream=0)
        alone.append(h.state(stream=0))
        h.close()
    hs = [pkg.Handle(**kw) for kw in kws]
    pkg.batch_run(hs, stream=0)
    for a, h in zip(alone, hs):
        assert np.array_equal(a, h.state(stream=0))
    kw = kws[0]
    _check(hs[0], "lhz", 6, kw["J"], 9, 32, 64, 3.0, 25, 60, insts=[1])
    for h in hs:
        h.close()
