"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Spins, energies, decoded states and success counts are compared bit for bit
(integer work: the tolerance is zero).  Sizes are small enough for the oracle
to finish in seconds but span several classes, words and a ragged replica
tail; the edge cases cover L = 2, one physical spin, a partial Chimera group,
an infinite Jperp (A = 0) and PT with one slot.  The full-size launches are
checked on sampled replicas in test_gpu_fullsize.py.
"""
import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W

pytestmark = pytest.mark.gpu


def gpu_state(h):
    st = h.state(stream=0)                      # [I][Z][n_phys][W]
    return pkg.unpack_words(st, h.R)            # [I][Z][n_phys][R]


def oracle_sqa(emb, N, J, pen, L, R, beta, S, seed, inst=0, A=None, B=None, t1=None, rho=None):
    pb = O.Problem(emb, N, J, pen)
    if A is None:
        A, B = O.linear_schedule(S)
    q = O.SQA(pb, L, R, beta, A, B, seed, inst)
    r0, r1 = rho if rho is not None else (0, R)
    q.run(0, S if t1 is None else t1, r0, r1)
    return pb, q


def sqa_case(emb, N, I, L, R, S, pen, beta, seed, A=None, B=None):
    J = W.random_instances(N, I, seed)
    h = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=seed, L=L, beta=beta,
                   A=A, B=B)
    h.run(stream=0)
    got = gpu_state(h)
    for i in range(I):
        pb, q = oracle_sqa(emb, N, J[i], pen, L, R, beta, S, seed, i, A, B)
        assert np.array_equal(got[i], q.s), f"instance {i}: state differs"
    return h, J, got


def test_sqa_lhz_k6_l32_r64_s1000():
    """LHZ K_6: 15 spins, 10 plaquettes, C = 3 max|J|, beta = 10/max|J|, L = 32, R = 64, 1000 sweeps."""
    c = W.lhz_n6_config()
    h = pkg.Handle(embedding="lhz", N=c["N"], J=c["J"], penalty=c["penalty"], sweeps=c["sweeps"],
                   R=c["R"], seed=c["seed"], L=c["L"], beta=c["beta"])
    h.run(stream=0)
    got = gpu_state(h)
    pb, q = oracle_sqa("lhz", c["N"], c["J"][0], c["penalty"], c["L"], c["R"], c["beta"],
                       c["sweeps"], c["seed"])
    assert np.array_equal(got[0], q.s)
    E = h.energies(stream=0)[0]
    assert np.array_equal(E, q.slice_energies())
    ro = pkg.unpack_words(h.readout(stream=0), c["R"])[0]
    assert np.array_equal(ro, q.s[0])


@pytest.mark.parametrize("emb,N,I,L,R,S", [("me", 8, 3, 8, 80, 40), ("lhz", 8, 2, 16, 70, 30),
                                           ("me", 12, 2, 6, 40, 25), ("lhz", 5, 2, 4, 129, 20)])
def test_sqa_multi_instance_ragged_replicas(emb, N, I, L, R, S):
    pen = 6 if emb == "me" else 9
    h, J, got = sqa_case(emb, N, I, L, R, S, pen, 10 / 3, seed=11 + N)
    E = h.energies(stream=0)
    for i in range(I):
        pb = O.Problem(emb, N, J[i], pen)
        for z in range(L):
            assert np.array_equal(E[i, z], pb.energies(got[i, z]))


@pytest.mark.parametrize("emb,N,L,R,S", [("me", 4, 2, 33, 30),      # L = 2: both neighbours one slice
                                         ("lhz", 2, 6, 5, 30),      # one physical spin, no plaquette
                                         ("me", 5, 4, 32, 15),      # partial Chimera group
                                         ("me", 2, 4, 1, 10)])      # one replica
def test_sqa_edge_shapes(emb, N, L, R, S):
    sqa_case(emb, N, 2, L, R, S, 4, 1.3, seed=5)


@pytest.mark.parametrize("emb,N,L,R,S", [("lhz", 64, 4, 32, 3),      # largest N: 2016 spins, 1891 plaquettes
                                         ("me", 64, 4, 33, 3),      # largest N: 16 x 16 Chimera cells
                                         ("lhz", 3, 1024, 40, 4)])  # largest L
def test_sqa_maximum_sizes(emb, N, L, R, S):
    sqa_case(emb, N, 2, L, R, S, 9 if emb == "lhz" else 6, 1.0, seed=64)


def test_sqa_user_schedule_reaching_zero_field():
    S = 24
    A = np.linspace(1.0, 0.0, S)     # last sweep: A = 0, Jperp infinite
    B = np.linspace(0.05, 1.0, S)
    sqa_case("lhz", 4, 2, 6, 48, S, 3, 2.0, seed=3, A=A, B=B)


def test_resume_equals_one_run():
    emb, N, L, R, S, pen = "me", 8, 8, 64, 50, 6
    J = W.random_instances(N, 2, 4)
    a = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=4, L=L, beta=3.0)
    a.run(stream=0)
    b = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=4, L=L, beta=3.0)
    b.run_sweeps(0, 17, stream=0)
    b.run_sweeps(17, 18, stream=0)
    b.run_sweeps(18, S, stream=0)
    assert np.array_equal(a.state(stream=0), b.state(stream=0))


def test_per_instance_path_equals_batched():
    emb, N, L, R, S, pen = "lhz", 7, 8, 96, 20, 9
    J = W.random_instances(N, 5, 8)
    a = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=8, L=L, beta=3.0)
    a.run(stream=0)
    b = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=8, L=L, beta=3.0)
    b.run_per_instance(stream=0)
    assert np.array_equal(a.state(stream=0), b.state(stream=0))


def test_batch_run_ragged_mix_equals_alone():
    specs = [dict(embedding="lhz", N=8, L=32, R=128, penalty=9, kind="sqa"),
             dict(embedding="me", N=12, L=16, R=40, penalty=6, kind="sqa"),
             dict(embedding="me", N=5, R=64, penalty=6, kind="pt"),
             dict(embedding="lhz", N=10, L=8, R=32, penalty=9, kind="sqa")]
    mk = []
    for k, s in enumerate(specs):
        J = W.random_instances(s["N"], 2, 100 + k)
        kw = dict(embedding=s["embedding"], N=s["N"], J=J, penalty=s["penalty"], sweeps=15, R=s["R"],
                  seed=100 + k, kind=s["kind"])
        if s["kind"] == "sqa":
            kw.update(L=s["L"], beta=3.0)
        else:
            kw.update(betas=W.geometric_ladder(6, 4.0, 0.3), swap_every=2)
        mk.append(kw)
    alone = []
    for kw in mk:
        h = pkg.Handle(**kw)
        h.run(stream=0)
        alone.append(h.state(stream=0))
    mixed = [pkg.Handle(**kw) for kw in mk]
    pkg.batch_run(mixed, stream=0)
    for a, h in zip(alone, mixed):
        assert np.array_equal(a, h.state(stream=0))


@pytest.mark.parametrize("emb,N,P,R,S,swap", [("me", 5, 6, 40, 31, 3), ("lhz", 6, 8, 64, 20, 1),
                                              ("me", 8, 1, 32, 12, 1), ("lhz", 4, 2, 100, 25, 2),
                                              ("lhz", 64, 4, 32, 3, 1), ("me", 64, 3, 32, 3, 1)])
def test_pt_parity(emb, N, P, R, S, swap):
    pen = 6 if emb == "me" else 9
    J = W.random_instances(N, 2, 21)
    betas = W.geometric_ladder(P, 5.0, 0.2)
    h = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=21, kind="pt",
                   betas=betas, swap_every=swap)
    h.run(stream=0)
    got = gpu_state(h)
    E = h.energies(stream=0)
    for i in range(2):
        pb = O.Problem(emb, N, J[i], pen)
        o = O.PT(pb, betas, R, swap, 21, i)
        o.run(0, S)
        assert np.array_equal(got[i], o.s), f"instance {i}"
        assert np.array_equal(E[i], o.E)


def test_pt_run_entry_point():
    N, R = 6, 32
    J = W.random_instances(N, 1, 2)
    h = pkg.Handle(embedding="me", N=N, J=J, penalty=6, sweeps=10, R=R, seed=2, L=4, beta=2.0)
    betas = W.paper_beta_ladder(8, 20.0, 0.1)
    h.pt_run(betas, 14, 10, stream=0)
    got = gpu_state(h)
    o = O.PT(O.Problem("me", N, J[0], 6), betas, R, 10, 2, 0)
    o.run(0, 14)
    assert np.array_equal(got[0], o.s)


def _oracle_decode(pb, method, phys, seed, inst, n_trees):
    N = pb.N
    if method == "me_mv":
        return O.me_decode(pb, phys)
    if method == "lhz_star":
        return O.lhz_tree_decode(N, O.star_tree(N), phys)
    if method == "lhz_chain":
        return O.lhz_tree_decode(N, O.chain_tree(N), phys)
    if method == "lhz_mwd":
        return O.lhz_mwd_decode(N, phys)
    if method == "lhz_bp":
        return O.lhz_bp_decode(N, phys, 0.2, 10, O.prufer_tree(N, seed, inst, 0))
    trees = np.stack([O.prufer_tree(N, seed, inst, t) for t in range(n_trees)])
    return O.lhz_vote_decode(N, trees, phys)


@pytest.mark.parametrize("emb,method,N", [("me", "me_mv", 8), ("me", "me_mv", 12),
                                          ("lhz", "lhz_trees", 8), ("lhz", "lhz_star", 6),
                                          ("lhz", "lhz_chain", 7), ("lhz", "lhz_mwd", 8),
                                          ("lhz", "lhz_mwd", 11), ("lhz", "lhz_bp", 8), ("lhz", "lhz_bp", 13)])
def test_decode_parity(emb, method, N):
    I, R, L, S = 3, 70, 8, 30
    pen = 6 if emb == "me" else 9
    J = W.random_instances(N, I, 31)
    h = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=31, L=L, beta=3.0)
    h.run(stream=0)
    phys = pkg.unpack_words(h.readout(stream=0), R)     # [I][n_phys][R]
    eg = np.array([O.ground_energy(N, J[i])[0] for i in range(I)], np.int64)
    n_trees = O.default_n_trees(N)
    logical, energy, succ = h.decode(method, 0, e_ground=eg, stream=0)
    for i in range(I):
        pb = O.Problem(emb, N, J[i], pen)
        cnt = 0
        for r in range(R):
            want = _oracle_decode(pb, method, phys[i, :, r], 31, i, n_trees)
            assert np.array_equal(logical[i, r], want), (i, r)
            e = O.logical_energy(N, J[i], want)
            assert energy[i, r] == e
            cnt += e == eg[i]
        assert succ[i] == cnt


@pytest.mark.parametrize("err,iters", [(0.2, 0), (0.1, 3), (0.35, 25), (0.5, 4)])
def test_bp_decode_parameters(err, iters):
    """sqa_decode_bp at other error rates and iteration counts (0 iterations:
    the plain tree; 1/2: every decision ties) against the oracle."""
    N, R = 9, 40
    J = W.random_instances(N, 2, 71)
    h = pkg.Handle(embedding="lhz", N=N, J=J, penalty=2, sweeps=15, R=R, seed=71, L=4, beta=1.0)
    h.run(stream=0)
    phys = pkg.unpack_words(h.readout(stream=0), R)
    logical, _, _ = h.decode_bp(err, iters, stream=0)
    for i in range(2):
        tree = O.prufer_tree(N, 71, i, 0)
        for r in range(R):
            assert np.array_equal(logical[i, r], O.lhz_bp_decode(N, phys[i, :, r], err, iters, tree)), (i, r)
    h.close()


def test_mwd_decode_of_pt_readouts_k16():
    """Minimum-weight decoding of PT's coldest slot on LHZ K_16 (2^15 states
    per readout), sampled replicas against the oracle; N > 24 is refused."""
    N, R, S = 16, 64, 40
    J = W.random_instances(N, 2, 88)
    betas = W.geometric_ladder(6, 5.0, 0.5)
    h = pkg.Handle(embedding="lhz", N=N, J=J, penalty=9, sweeps=S, R=R, seed=88, kind="pt", betas=betas,
                   swap_every=1)
    h.run(stream=0)
    phys = pkg.unpack_words(h.readout(stream=0), R)
    logical, energy, _ = h.decode("lhz_mwd", 0, stream=0)
    for i in range(2):
        for r in (0, 1, 17, 40, 63):
            assert np.array_equal(logical[i, r], O.lhz_mwd_decode(N, phys[i, :, r])), (i, r)
    h.close()
    J25 = W.random_instances(25, 1, 1)
    h = pkg.Handle(embedding="lhz", N=25, J=J25, penalty=9, sweeps=2, R=32, seed=1, L=4, beta=1.0)
    h.run(stream=0)
    with pytest.raises(pkg.SQAError):
        h.decode("lhz_mwd", 0, stream=0)
    h.close()


def test_failed_pt_switch_leaves_no_program():
    """pt_run releases the handle's SQA program before it builds the PT one;
    couplings too large for PT's byte-wise windows (penalty 60) are refused
    there, and every later call but close must raise instead of launching on
    released memory."""
    J = W.random_instances(8, 2, 5)
    h = pkg.Handle(embedding="me", N=8, J=J, penalty=60, sweeps=10, R=32, seed=5, L=8, beta=1.0)
    h.run(stream=0)
    with pytest.raises(pkg.SQAError) as e:
        h.pt_run(W.geometric_ladder(4, 2.0, 0.5), 10, 1, stream=0)
    assert e.value.status == pkg.SQA_ERR_UNSUPPORTED
    for call in (lambda: h.run(stream=0), lambda: h.run_sweeps(0, 5, stream=0), lambda: h.readout(stream=0),
                 lambda: h.state(stream=0), lambda: h.energies(stream=0), lambda: h.decode("me_mv", 0, stream=0),
                 lambda: h.tune(1, 1, 1)):
        with pytest.raises(pkg.SQAError) as e:
            call()
        assert e.value.status == pkg.SQA_ERR_INVALID
    h.close()


def test_tree_decode_after_switch_to_pt():
    """Decoding trees cached by an SQA program are released with it: after a
    switch to PT the same decode equals a fresh PT handle's."""
    N, R, S = 7, 64, 30
    J = W.random_instances(N, 2, 21)
    betas = W.geometric_ladder(6, 5.0, 0.5)
    h = pkg.Handle(embedding="lhz", N=N, J=J, penalty=9, sweeps=S, R=R, seed=21, L=8, beta=1.0)
    h.run(stream=0)
    h.decode("lhz_trees", 3, stream=0)
    h.pt_run(betas, S, 1, stream=0)
    got = h.decode("lhz_trees", 3, stream=0)
    h.close()
    f = pkg.Handle(embedding="lhz", N=N, J=J, penalty=9, sweeps=S, R=R, seed=21, kind="pt", betas=betas,
                   swap_every=1)
    f.run(stream=0)
    want = f.decode("lhz_trees", 3, stream=0)
    f.close()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


@pytest.mark.parametrize("N", [2, 3, 5, 8, 11, 16])
def test_ground_energy_parity(N):
    J = W.random_instances(N, 4, 50 + N)
    got = pkg.ground_energy(N, J)
    want = [O.ground_energy(N, J[i])[0] for i in range(4)]
    assert list(got) == want


@pytest.mark.parametrize("emb,use_table,wc", [("lhz", 0, 0), ("lhz", 1, 0), ("me", 0, 1), ("me", 1, 2),
                                              ("lhz", -1, 3), ("me", 1, 5)])
def test_launch_shapes_give_the_oracle_bits(emb, use_table, wc):
    """Table or window threshold lookup, any words per block: same bits."""
    N, L, R, S = 8, 8, 150, 20                      # 5 words, ragged last word
    pen = 6 if emb == "me" else 9
    J = W.random_instances(N, 2, 77)
    h = pkg.Handle(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=77, L=L, beta=3.0)
    h.tune(wc, use_table)
    got = h.launch()
    if use_table >= 0:
        assert got["use_table"] == use_table
    if wc:
        assert got["words_per_unit"] == wc
    h.run(stream=0)
    st = gpu_state(h)
    for i in range(2):
        pb, q = oracle_sqa(emb, N, J[i], pen, L, R, 3.0, S, 77, i)
        assert np.array_equal(st[i], q.s)


@pytest.mark.parametrize("kind,emb,slices", [("sqa", "me", 1), ("sqa", "me", 3), ("sqa", "lhz", 4),
                                            ("sqa", "lhz", 2), ("pt", "me", 3), ("pt", "lhz", 1)])
def test_slices_per_task_give_the_oracle_bits(kind, emb, slices):
    """Forced slices (or slots) per thread's task, 1..4, including counts that
    do not divide the slice pairs (L = 14: 7 per parity) or the slots (P = 7):
    same bits."""
    N, R, S = 7, 70, 15
    pen = 6 if emb == "me" else 9
    J = W.random_instances(N, 2, 600 + slices)
    kw = dict(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=600 + slices, kind=kind)
    if kind == "sqa":
        kw.update(L=14, beta=3.0)
    else:
        kw.update(betas=W.geometric_ladder(7, 5.0, 0.2), swap_every=1)
    h = pkg.Handle(**kw)
    h.tune_slices(slices)
    assert h.launch()["task_slices"] == slices
    h.run(stream=0)
    st = gpu_state(h)
    E = h.energies(stream=0)
    for i in range(2):
        pb = O.Problem(emb, N, J[i], pen)
        if kind == "sqa":
            A, B = O.linear_schedule(S)
            q = O.SQA(pb, 14, R, 3.0, A, B, 600 + slices, i)
            q.run(0, S)
            assert np.array_equal(st[i], q.s)
        else:
            o = O.PT(pb, kw["betas"], R, 1, 600 + slices, i)
            o.run(0, S)
            assert np.array_equal(st[i], o.s) and np.array_equal(E[i], o.E)
    with pytest.raises(pkg.SQAError):
        h.tune_slices(5)
    h.close()


def test_oversized_unit_is_refused():
    """One 32-replica word of LHZ K_64 at L = 1024 is 8 MB of state, more than
    a 16-block cluster's shared memory: the job is refused at planning (no
    launch), not run from HBM."""
    J = W.random_instances(64, 1, 3)
    with pytest.raises(pkg.SQAError) as e:
        pkg.Handle(embedding="lhz", N=64, J=J, penalty=9, sweeps=2, R=32, seed=3, L=1024, beta=1.0)
    assert e.value.status == pkg.SQA_ERR_UNSUPPORTED


def test_planner_weighs_table_rebuilds():
    """Single-job plans take code tables where a block holds many items per
    table entry (the 1024 x 256 ME K_8 workload: one block per unit, 8 words)
    and byte windows where the per-sweep table rebuild would dominate (an
    8-block cluster of one ME K_21 instance at L = 128); batches keep tables.
    Planning only: the bits do not depend on the choice (tested above)."""
    cfg = W.me_n8_batch_config(sweeps=10)
    h = pkg.Handle(embedding="me", N=8, J=cfg["J"], penalty=cfg["penalty"], sweeps=10, R=256, seed=0, L=64,
                   beta=cfg["beta"])
    got = h.launch()
    h.close()
    assert (got["use_table"], got["cluster"], got["words_per_unit"]) == (1, 1, 8), got
    J = W.random_instances(21, 1, 80)
    h = pkg.Handle(embedding="me", N=21, J=J, penalty=6, sweeps=10, R=175, seed=80, L=128, beta=10 / 3)
    got = h.launch()
    h.close()
    assert got["use_table"] == 0 and got["cluster"] > 1, got


@pytest.mark.parametrize("kind,emb,N,Z,R,C", [("sqa", "lhz", 8, 16, 64, 2), ("sqa", "me", 12, 16, 40, 4),
                                              ("sqa", "lhz", 6, 16, 33, 8), ("pt", "me", 8, 8, 64, 2),
                                              ("pt", "lhz", 7, 8, 32, 4), ("pt", "me", 5, 16, 40, 8),
                                              ("sqa", "lhz", 6, 32, 40, 16), ("pt", "me", 6, 16, 33, 16)])
def test_cluster_split_gives_the_oracle_bits(kind, emb, N, Z, R, C):
    """A thread-block cluster sweeping one unit, each block holding Z/C slices or
    slots (temporal neighbours and swap partners across blocks)."""
    pen = 6 if emb == "me" else 9
    S = 24
    J = W.random_instances(N, 2, 500 + C)
    kw = dict(embedding=emb, N=N, J=J, penalty=pen, sweeps=S, R=R, seed=500 + C, kind=kind)
    if kind == "sqa":
        kw.update(L=Z, beta=3.0)
    else:
        kw.update(betas=W.geometric_ladder(Z, 5.0, 0.2), swap_every=1 if C != 4 else 3)
    h = pkg.Handle(**kw)
    h.tune(0, -1, C)
    assert h.launch()["cluster"] == C
    h.run(stream=0)
    st = gpu_state(h)
    E = h.energies(stream=0)
    for i in range(2):
        pb = O.Problem(emb, N, J[i], pen)
        if kind == "sqa":
            A, B = O.linear_schedule(S)
            q = O.SQA(pb, Z, R, 3.0, A, B, 500 + C, i)
            q.run(0, S)
            assert np.array_equal(st[i], q.s)
        else:
            o = O.PT(pb, kw["betas"], R, kw["swap_every"], 500 + C, i)
            o.run(0, S)
            assert np.array_equal(st[i], o.s)
            assert np.array_equal(E[i], o.E)


def test_word_larger_than_one_block_is_split_across_a_cluster():
    """LHZ K_40 at L = 128: one 32-replica word of state is 400 KB, more than
    one block's shared memory; the planner splits the slices over a cluster."""
    N, L, R, S = 40, 128, 32, 3
    J = W.random_instances(N, 1, 9)
    h = pkg.Handle(embedding="lhz", N=N, J=J, penalty=9, sweeps=S, R=R, seed=9, L=L, beta=10 / 3)
    assert h.launch()["cluster"] >= 2
    h.run(stream=0)
    pb, q = oracle_sqa("lhz", N, J[0], 9, L, R, 10 / 3, S, 9)
    assert np.array_equal(gpu_state(h)[0], q.s)
