"""Full-size parity, sampled: the ragged batch, the PT workloads and the
cluster-move workload of the benchmark at their full instance counts and in
the launch configuration bench.py times, with sampled (instance, replica)
pairs re-run by the oracle.

The ragged batch runs its full 1e4 sweeps.  The PT ladders run 2000 sweeps
instead of 1e5 (the oracle recounts every slot's energy at every swap, so a
1e5-sweep replica would take minutes on the host); the launch shape does not
depend on the sweep count (likewise 500 sweeps for the cluster moves, whose
oracle draws all 32 bit-planes of every bond).  Energies of the sampled
replicas are recomputed from their spins.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu


def test_ragged_batch_full_size_sampled():
    jobs = W.ragged_mix_config(512, R=128, sweeps=10_000)
    hs = [pkg.Handle(embedding=j["embedding"], N=j["N"], J=j["J"], penalty=j["penalty"], sweeps=j["sweeps"],
                     R=j["R"], seed=j["seed"], L=j["L"], beta=j["beta"]) for j in jobs]
    pkg.batch_run(hs, stream=0)
    for k, (r0, r1) in [(0, (0, 3)), (1, (125, 128)), (510, (60, 63)), (511, (0, 2))]:
        j = jobs[k]
        got = pkg.unpack_words(hs[k].state(stream=0)[0], j["R"])
        pb = O.Problem(j["embedding"], j["N"], j["J"][0], j["penalty"])
        A, B = O.linear_schedule(j["sweeps"])
        q = O.SQA(pb, j["L"], j["R"], j["beta"], A, B, j["seed"], 0)
        q.run(0, j["sweeps"], r0, r1)
        assert np.array_equal(got[:, :, r0:r1], q.s[:, :, r0:r1]), k
        E = hs[k].energies(stream=0)[0]
        for z in (0, j["L"] - 1):
            assert np.array_equal(E[z, r0:r1], pb.energies(got[z])[r0:r1])
    for h in hs:
        h.close()


@pytest.mark.parametrize("emb", ["me", "lhz"])
def test_pt_full_size_sampled(emb):
    c = W.pt_config(emb, sweeps=2000)
    h = pkg.Handle(embedding=emb, N=c["N"], J=c["J"], penalty=c["penalty"], sweeps=c["sweeps"], R=c["R"],
                   seed=c["seed"], kind="pt", betas=c["betas"], swap_every=c["swap_every"])
    assert h.launch()["cluster"] == 1                      # the bench's PT launch shape
    h.run(stream=0)
    st = h.state(stream=0)
    E = h.energies(stream=0)
    for inst, (r0, r1) in [(0, (0, 2)), (255, (30, 32))]:
        pb = O.Problem(emb, c["N"], c["J"][inst], c["penalty"])
        o = O.PT(pb, c["betas"], c["R"], c["swap_every"], c["seed"], inst)
        o.run(0, c["sweeps"], r0, r1)
        got = pkg.unpack_words(st[inst], c["R"])
        assert np.array_equal(got[:, :, r0:r1], o.s[:, :, r0:r1]), inst
        assert np.array_equal(E[inst][:, r0:r1], o.E[:, r0:r1])
    h.close()


def test_cluster_moves_full_size_sampled():
    """The bench's cluster-move workload (ME K_8, 1024 instances x 256
    replicas, L = 64) and launch, 500 sweeps, sampled replicas."""
    c = W.me_n8_batch_config(sweeps=500)
    h = pkg.Handle(embedding="me", N=c["N"], J=c["J"], penalty=c["penalty"], sweeps=c["sweeps"], R=c["R"],
                   seed=c["seed"], L=c["L"], beta=c["beta"], move="wolff")
    h.run(stream=0)
    st = h.state(stream=0)
    for inst, (r0, r1) in [(0, (0, 2)), (1023, (254, 256))]:
        pb = O.Problem("me", c["N"], c["J"][inst], c["penalty"])
        A, B = O.linear_schedule(c["sweeps"])
        q = O.SQA(pb, c["L"], c["R"], c["beta"], A, B, c["seed"], inst, move="wolff")
        q.run(0, c["sweeps"], r0, r1)
        got = pkg.unpack_words(st[inst], c["R"])
        assert np.array_equal(got[:, :, r0:r1], q.s[:, :, r0:r1]), inst
    h.close()
