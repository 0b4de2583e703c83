"""Full-size parity, sampled: the benchmark's workloads at their full instance
counts and sweep counts, in the launch configuration bench.py times, with
sampled (instance, replica word) pairs re-run by the oracle on every host
thread (the oracle's C calls release the interpreter lock, so a thread pool
runs them in parallel).

- ME K_8, 1024 instances x 256 replicas, L = 64, 1e4 sweeps, the autotuned
  launch: 16 instances spread over the batch, one whole 32-replica word each
  (every word position 0-7 twice), through all 1e4 sweeps.
- The ragged LHZ/ME mix, 512 instances, its full 1e4 sweeps.
- PT on ME K_32 and LHZ K_24 (256 instances x 32 replicas, 32 temperatures,
  swap every sweep): the bench's full 1e5 sweeps, two replicas of two
  instances per embedding (the oracle recounts every slot's energy at every
  swap, about a minute per replica).
- Time-like cluster moves on the ME K_8 workload: the bench's full 2000
  sweeps, replicas sampled from four instances.

Energies of the sampled replicas are recomputed from their spins.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu


def _map(fn, items):
    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        return list(ex.map(fn, items))


def _sqa_oracle(emb, N, J, pen, L, R, beta, sweeps, seed, inst, r0, r1, move="metropolis"):
    pb = O.Problem(emb, N, J, pen)
    A, B = O.linear_schedule(sweeps)
    q = O.SQA(pb, L, R, beta, A, B, seed, inst, move=move)
    q.run(0, sweeps, r0, r1)
    return pb, q


def test_me_k8_batch_full_size_sixteen_words():
    c = W.me_n8_batch_config()
    h = pkg.Handle(embedding="me", N=c["N"], J=c["J"], penalty=c["penalty"], sweeps=c["sweeps"],
                   R=c["R"], seed=c["seed"], L=c["L"], beta=c["beta"])
    h.autotune(n_trial=20, stream=0)                       # as bench.py does before timing
    h.run(stream=0)
    st = h.state(stream=0)
    E = h.energies(stream=0)
    h.close()
    I = c["J"].shape[0]
    picks = [(int(i), k % 8) for k, i in enumerate(np.linspace(0, I - 1, 16).round())]

    def one(p):
        inst, word = p
        r0, r1 = 32 * word, 32 * word + 32
        pb, q = _sqa_oracle("me", c["N"], c["J"][inst], c["penalty"], c["L"], c["R"], c["beta"],
                            c["sweeps"], c["seed"], inst, r0, r1)
        got = pkg.unpack_words(st[inst], c["R"])
        ok_s = np.array_equal(got[:, :, r0:r1], q.s[:, :, r0:r1])
        ok_e = all(np.array_equal(E[inst, z, r0:r1], pb.energies(got[z])[r0:r1]) for z in (0, 31, 63))
        return inst, word, ok_s, ok_e

    res = _map(one, picks)
    bad = [(i, w) for i, w, s, e in res if not (s and e)]
    assert not bad, f"(instance, word) pairs that differ from the oracle: {bad}"


def test_ragged_batch_full_size_sampled():
    jobs = W.ragged_mix_config(512, R=128, sweeps=10_000)
    hs = [pkg.Handle(embedding=j["embedding"], N=j["N"], J=j["J"], penalty=j["penalty"], sweeps=j["sweeps"],
                     R=j["R"], seed=j["seed"], L=j["L"], beta=j["beta"]) for j in jobs]
    b = pkg.Batch(hs)
    b.autotune(n_trial=50, stream=0)                       # as bench.py does before timing
    b.launch(stream=0)
    b.close()
    picks = [(0, (0, 3)), (1, (125, 128)), (200, (32, 64)), (347, (96, 99)), (510, (60, 63)), (511, (0, 2))]
    states = {k: pkg.unpack_words(hs[k].state(stream=0)[0], jobs[k]["R"]) for k, _ in picks}
    energies = {k: hs[k].energies(stream=0)[0] for k, _ in picks}
    for h in hs:
        h.close()

    def one(p):
        k, (r0, r1) = p
        j = jobs[k]
        pb, q = _sqa_oracle(j["embedding"], j["N"], j["J"][0], j["penalty"], j["L"], j["R"], j["beta"],
                            j["sweeps"], j["seed"], 0, r0, r1)
        got = states[k]
        ok = np.array_equal(got[:, :, r0:r1], q.s[:, :, r0:r1])
        ok &= all(np.array_equal(energies[k][z, r0:r1], pb.energies(got[z])[r0:r1]) for z in (0, j["L"] - 1))
        return k, ok

    bad = [k for k, ok in _map(one, picks) if not ok]
    assert not bad, f"jobs that differ from the oracle: {bad}"


@pytest.mark.parametrize("emb", ["me", "lhz"])
def test_pt_full_size_sampled(emb):
    c = W.pt_config(emb, sweeps=100_000)
    h = pkg.Handle(embedding=emb, N=c["N"], J=c["J"], penalty=c["penalty"], sweeps=c["sweeps"], R=c["R"],
                   seed=c["seed"], kind="pt", betas=c["betas"], swap_every=c["swap_every"])
    assert h.launch()["cluster"] == 1                      # the bench's PT launch shape
    h.run(stream=0)
    st = h.state(stream=0)
    E = h.energies(stream=0)
    h.close()
    picks = [(0, (0, 1)), (0, (17, 18)), (255, (30, 31)), (255, (31, 32))]

    def one(p):
        inst, (r0, r1) = p
        pb = O.Problem(emb, c["N"], c["J"][inst], c["penalty"])
        o = O.PT(pb, c["betas"], c["R"], c["swap_every"], c["seed"], inst)
        o.run(0, c["sweeps"], r0, r1)
        got = pkg.unpack_words(st[inst], c["R"])
        return (inst, r0, np.array_equal(got[:, :, r0:r1], o.s[:, :, r0:r1])
                and np.array_equal(E[inst][:, r0:r1], o.E[:, r0:r1]))

    bad = [(i, r) for i, r, ok in _map(one, picks) if not ok]
    assert not bad, f"(instance, replica) pairs that differ from the oracle: {bad}"


def test_cluster_moves_full_size_sampled():
    """The bench's cluster-move workload (ME K_8, 1024 instances x 256
    replicas, L = 64) and launch, its full 2000 sweeps, sampled replicas."""
    c = W.me_n8_batch_config(sweeps=2000)
    h = pkg.Handle(embedding="me", N=c["N"], J=c["J"], penalty=c["penalty"], sweeps=c["sweeps"], R=c["R"],
                   seed=c["seed"], L=c["L"], beta=c["beta"], move="wolff")
    h.run(stream=0)
    st = h.state(stream=0)
    h.close()
    picks = [(0, (0, 2)), (341, (100, 102)), (682, (31, 33)), (1023, (254, 256))]

    def one(p):
        inst, (r0, r1) = p
        _, q = _sqa_oracle("me", c["N"], c["J"][inst], c["penalty"], c["L"], c["R"], c["beta"], c["sweeps"],
                           c["seed"], inst, r0, r1, move="wolff")
        got = pkg.unpack_words(st[inst], c["R"])
        return inst, np.array_equal(got[:, :, r0:r1], q.s[:, :, r0:r1])

    bad = [i for i, ok in _map(one, picks) if not ok]
    assert not bad, f"instances that differ from the oracle: {bad}"
