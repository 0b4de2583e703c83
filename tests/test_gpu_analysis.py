"""The host-side analyses (App. D, App. E) on the library's readouts.

SQA and PT readouts of one LHZ K_8 instance from the GPU: the energy
distance, error rates and error-by-distance profile computed from them
equal those computed from the oracle's states of the same anneal (the
states are bit-identical), and lie in their ranges.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W
from paper_1603_03755_gb300 import analysis as A

pytestmark = pytest.mark.gpu


def test_analyses_on_gpu_readouts():
    N, L, R, S, seed, pen = 8, 16, 64, 200, 21, 9
    J = W.random_couplings(N, 7)
    h = pkg.Handle(embedding="lhz", N=N, J=J, penalty=pen, sweeps=S, R=R, seed=seed, L=L, beta=10 / 3)
    h.run(stream=0)
    sqa_states = pkg.unpack_words(h.readout(stream=0), R)[0].T          # [R, n_phys]
    e_sqa = h.energies(stream=0)[0][0]                                    # slice 0
    h.close()
    betas = W.geometric_ladder(8, 10 / 3, 0.3)
    p = pkg.Handle(embedding="lhz", N=N, J=J, penalty=pen, sweeps=S, R=R, seed=seed, kind="pt", betas=betas,
                   swap_every=1)
    p.run(stream=0)
    pt_states = pkg.unpack_words(p.readout(stream=0), R)[0].T           # coldest slot
    e_pt = p.energies(stream=0)[0][0]
    p.close()

    pb = O.Problem("lhz", N, J, pen)
    A_, B_ = O.linear_schedule(S)
    q = O.SQA(pb, L, R, 10 / 3, A_, B_, seed)
    q.run(0, S)
    assert np.array_equal(sqa_states, q.s[0].T)
    assert np.array_equal(e_sqa, q.slice_energies()[0])

    D = A.energy_distance(e_sqa, e_pt)
    assert 0.0 <= D <= 1.0
    rates = A.error_rates("lhz", N, J, sqa_states)
    assert np.array_equal(rates, A.error_rates("lhz", N, J, q.s[0].T))
    assert np.all((rates >= 0) & (rates <= 1))
    prof = A.error_by_distance(N, J, sqa_states)
    assert prof.shape == (N - 1,) and np.all((prof >= 0) & (prof <= 1))
    assert np.allclose(prof, A.error_by_distance(N, J, q.s[0].T))
    rng = np.random.default_rng(0)
    ref = A.error_by_distance(N, J, A.uncorrelated_states("lhz", N, J, float(rates.mean()), 1000, rng))
    counted = A.coefficients_above(A.fit_coefficients(prof), ref)
    assert counted.shape == (7,)
