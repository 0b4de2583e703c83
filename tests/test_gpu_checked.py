"""The bounds-checked build (-DSQA_BOUNDS_CHECK) on small parity cases.

A child process loads the checked library (SQA_GB300_CHECKED=1), runs one
small case of every kernel path (SQA on byte windows and on code tables,
the sign-folded minor-embedding tables, several words per block, a slice
split over a thread-block cluster, PT with and without a cluster, the time-
like cluster moves, a ragged multi-job batch, energies and decoding) and
compares each with the oracle bit for bit.  After every case the device
status word must be clear: no kernel index left its buffer.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_checked_build_runs_every_path_without_violations():
    env = dict(os.environ, SQA_GB300_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked cases ok" in r.stdout


def _cases():
    sys.path.insert(0, ROOT)
    from paper_1603_03755_gb300 import build as b
    b.build(checked=True)
    import oracle as O
    import paper_1603_03755_gb300 as pkg
    import workloads as W

    assert pkg.CHECKED and pkg.lib().sqa_bounds_checked() == 1

    def clean(what):
        st, rec = pkg.check_status()
        assert st == pkg.SQA_OK and rec == [0, 0, 0, 0], (what, rec, pkg.lib().sqa_last_error())

    def sqa(emb, N, L, R, S, seed, tune=None, move="metropolis", I=2):
        pen = 6 if emb == "me" else 9
        J = W.random_instances(N, I, seed)
        h = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=seed, L=L, beta=3.0, move=move)
        if tune:
            h.tune(*tune)
        h.run(stream=0)
        st = pkg.unpack_words(h.state(stream=0), R)
        E = h.energies(stream=0)
        A, B = O.linear_schedule(S)
        for i in range(I):
            pb = O.Problem(emb, N, J[i], pen)
            q = O.SQA(pb, L, R, 3.0, A, B, seed, i, move=move)
            q.run(0, S)
            assert np.array_equal(st[i], q.s), (emb, N, tune, move, i)
            assert np.array_equal(E[i, 0], pb.energies(st[i][0]))
        return h, J

    def pt(emb, N, P, R, S, seed, cluster=0):
        pen = 6 if emb == "me" else 9
        J = W.random_instances(N, 2, seed)
        betas = W.geometric_ladder(P, 5.0, 0.2)
        h = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=seed, kind="pt", betas=betas,
                       swap_every=1)
        if cluster:
            h.tune(0, -1, cluster)
        h.run(stream=0)
        st = pkg.unpack_words(h.state(stream=0), R)
        E = h.energies(stream=0)
        for i in range(2):
            o = O.PT(O.Problem(emb, N, J[i], pen), betas, R, 1, seed, i)
            o.run(0, S)
            assert np.array_equal(st[i], o.s) and np.array_equal(E[i], o.E), (emb, N, cluster, i)
        h.close()

    cases = [
        ("sqa lhz windows", lambda: sqa("lhz", 6, 8, 40, 20, 1, (0, 0))[0].close()),
        ("sqa lhz tables", lambda: sqa("lhz", 6, 8, 40, 20, 2, (0, 1))[0].close()),
        ("sqa me folded tables", lambda: sqa("me", 5, 8, 72, 20, 3, (0, 1))[0].close()),
        ("sqa me windows, 2 words per unit", lambda: sqa("me", 8, 16, 96, 15, 4, (2, 0))[0].close()),
        ("sqa me tables, cluster of 4", lambda: sqa("me", 6, 16, 40, 12, 5, (0, -1, 4))[0].close()),
        ("sqa lhz cluster of 2", lambda: sqa("lhz", 7, 16, 33, 12, 6, (0, -1, 2))[0].close()),
        ("pt me", lambda: pt("me", 6, 8, 40, 15, 7)),
        ("pt lhz, cluster of 2", lambda: pt("lhz", 6, 8, 64, 15, 8, 2)),
        ("cluster moves", lambda: sqa("me", 6, 16, 40, 10, 9, move="wolff")[0].close()),
    ]
    for what, fn in cases:
        fn()
        clean(what)
    # a ragged batch of the multi-job kernel
    specs = [("lhz", 6, 8, 40), ("me", 5, 16, 64), ("lhz", 8, 8, 33)]
    hs, want = [], []
    A, B = O.linear_schedule(12)
    for k, (emb, N, L, R) in enumerate(specs):
        pen = 6 if emb == "me" else 9
        J = W.random_instances(N, 1, 40 + k)
        hs.append(pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=12, R=R, seed=40 + k, L=L, beta=3.0))
        q = O.SQA(O.Problem(emb, N, J[0], pen), L, R, 3.0, A, B, 40 + k, 0)
        q.run(0, 12)
        want.append(q.s)
    pkg.batch_run(hs, stream=0)
    for h, w, (_, _, _, R) in zip(hs, want, specs):
        assert np.array_equal(pkg.unpack_words(h.state(stream=0)[0], R), w)
        h.close()
    clean("ragged batch")
    # decoding: majority vote (ME) and minimum-weight decoding (LHZ)
    h, J = sqa("me", 6, 8, 40, 10, 11)
    logical, _, _ = h.decode("me_mv", 0, stream=0)
    st = pkg.unpack_words(h.state(stream=0), 40)
    pb = O.Problem("me", 6, J[0], 6)
    assert all(np.array_equal(logical[0, r], O.me_decode(pb, st[0][0][:, r])) for r in range(40))
    h.close()
    clean("majority vote")
    h, J = sqa("lhz", 6, 8, 40, 10, 12)
    logical, _, _ = h.decode("lhz_mwd", 0, stream=0)
    st = pkg.unpack_words(h.state(stream=0), 40)
    assert all(np.array_equal(logical[0, r], O.lhz_mwd_decode(6, st[0][0][:, r])) for r in range(40))
    h.close()
    clean("minimum-weight decoding")
    print("checked cases ok")


if __name__ == "__main__":
    _cases()
