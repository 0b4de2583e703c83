"""A penalty scan in one batch launch equals one run per penalty, and its
success counts equal the oracle's on a sampled penalty."""
import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W
from paper_1603_03755_gb300.scan import penalty_scan

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("emb,kind", [("lhz", "sqa"), ("me", "sqa"), ("lhz", "pt")])
def test_scan_equals_runs_per_penalty(emb, kind):
    N, R, S = 6, 64, 60
    J = W.random_instances(N, 3, 21)
    pens = [2, 5, 9]
    anneal = dict(L=16, beta=3.0) if kind == "sqa" else dict(betas=W.geometric_ladder(6, 5.0, 0.5), swap_every=1)
    res = penalty_scan(embedding=emb, N=N, J=J, penalties=pens, R=R, sweeps=S, seed=21, kind=kind, stream=0,
                       **anneal)
    assert res.success.shape == (3, 3)
    eg = pkg.ground_energy(N, J)
    assert np.array_equal(res.e_ground, eg)
    for k, p in enumerate(pens):
        h = pkg.Handle(embedding=emb, N=N, J=J, penalty=p, sweeps=S, R=R, seed=21, kind=kind, **anneal)
        h.run(stream=0)
        _, _, succ = h.decode(None, 0, e_ground=eg, stream=0)
        assert np.array_equal(res.success[k] * R, succ)
        h.close()
    # one penalty, one instance, against the oracle end to end
    if kind == "sqa":
        pb = O.Problem(emb, N, J[1], pens[1])
        A, B = O.linear_schedule(S)
        q = O.SQA(pb, 16, R, 3.0, A, B, 21, 1)
        q.run(0, S)
        ro = q.s[0]
        cnt = 0
        for r in range(R):
            if emb == "me":
                d = O.me_decode(pb, ro[:, r])
            else:
                trees = np.stack([O.prufer_tree(N, 21, 1, t) for t in range(O.default_n_trees(N))])
                d = O.lhz_vote_decode(N, trees, ro[:, r])
            cnt += O.logical_energy(N, J[1], d) == O.ground_energy(N, J[1])[0]
        assert res.success[1, 1] * R == cnt
    assert np.all((res.optimal >= 2) & (res.optimal <= 9))
