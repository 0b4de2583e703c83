"""Host-side checks of the C ABI (no GPU needed).

  - the shared library loads and exports every function include/sqa.h declares;
  - the library's own embedding, acceptance tables, swap tables and decoding
    trees (computed on the host by the library, independently of the oracle)
    equal the oracle's, bit for bit;
  - argument validation answers before any device work.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_1603_03755_gb300 as pkg
import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sqa.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sqa_\w+|pt_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_1603_03755_gb300 import build as b
    b.build()
    return pkg.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "sqa_create" in names and "pt_run" in names and "sqa_batch_run" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(pkg._SIGS)


def _plan_terms(L, emb, N, J, penalty):
    cap = 8000
    nphys, nt = C.c_int32(), C.c_int32()
    ts = np.zeros(cap, np.int32)
    tm = np.zeros(cap * 4, np.int32)
    tw = np.zeros(cap, np.int32)
    col = np.zeros(4096, np.int32)
    st = L.sqa_plan_terms(pkg.EMB[emb], N, J.ctypes.data, penalty, cap, C.byref(nphys), C.byref(nt),
                          ts.ctypes.data, tm.ctypes.data, tw.ctypes.data, col.ctypes.data)
    assert st == 0
    terms = sorted((tuple(sorted(tm[4 * t:4 * t + ts[t]].tolist())), int(tw[t])) for t in range(nt.value))
    return nphys.value, terms, col[:nphys.value]


@pytest.mark.parametrize("emb,N", [("me", 2), ("me", 5), ("me", 8), ("me", 13), ("me", 32),
                                   ("lhz", 2), ("lhz", 3), ("lhz", 6), ("lhz", 16), ("lhz", 24)])
def test_library_embedding_equals_oracle(L, emb, N):
    J = W.random_couplings(N, 40 + N)
    pen = 6 if emb == "me" else 9
    nphys, terms, col = _plan_terms(L, emb, N, J, pen)
    pb = O.Problem(emb, N, J, pen)
    assert nphys == pb.n
    assert terms == sorted((tuple(sorted(m)), w) for m, w in pb.terms())
    assert np.array_equal(col, pb.colour)


def _desc(kind, emb, N, J, pen, S, R=32, L=8, beta=10 / 3, A=None, B=None, betas=None):
    d = pkg._Desc()
    J = np.ascontiguousarray(np.atleast_2d(J), np.int32)
    keep = [J]
    d.kind, d.embedding, d.n_logical, d.n_instances = pkg.KIND[kind], pkg.EMB[emb], N, J.shape[0]
    d.J, d.h, d.penalty, d.n_sweeps, d.n_replicas, d.seed = J.ctypes.data, None, pen, S, R, 1
    d.n_slices, d.beta = L, beta
    if A is not None:
        A = np.ascontiguousarray(A, np.float64)
        B = np.ascontiguousarray(B, np.float64)
        keep += [A, B]
        d.A, d.B = A.ctypes.data, B.ctypes.data
    if betas is not None:
        betas = np.ascontiguousarray(betas, np.float64)
        keep.append(betas)
        d.betas, d.n_temps = betas.ctypes.data, len(betas)
    d.swap_every = 1
    return d, keep


def _tables(Llib, d, keep):
    dmin, dmax = C.c_int32(), C.c_int32()
    assert Llib.sqa_plan_tables(C.byref(d), None, 0, C.byref(dmin), C.byref(dmax)) == 0
    nd = (dmax.value - dmin.value) // 2 + 1
    rows = d.n_sweeps * 3 if d.kind == 0 else d.n_temps
    T = np.zeros(rows * nd, np.uint32)
    assert Llib.sqa_plan_tables(C.byref(d), T.ctypes.data, T.size, C.byref(dmin), C.byref(dmax)) == 0
    return T, dmin.value, dmax.value


@pytest.mark.parametrize("emb,N,S,Ls,beta", [("lhz", 6, 1000, 32, 10 / 3), ("me", 8, 300, 64, 10 / 3),
                                             ("me", 5, 50, 2, 0.7), ("lhz", 9, 80, 16, 20.0)])
def test_sqa_tables_equal_oracle(L, emb, N, S, Ls, beta):
    J = W.random_instances(N, 3, 5)
    pen = 6 if emb == "me" else 9
    d, keep = _desc("sqa", emb, N, J, pen, S, L=Ls, beta=beta)
    T, dmin, dmax = _tables(L, d, keep)
    lo = min(O.Problem(emb, N, J[i], pen).delta_range()[0] for i in range(3))
    assert dmin == lo and dmax == -lo
    A, B = O.linear_schedule(S)
    want = O.sqa_table(A, B, beta, Ls, 0, S, dmin, dmax)
    assert np.array_equal(T, want.ravel())


def test_sqa_tables_user_schedule_with_zero_field(L):
    """A user schedule reaching A = 0 (infinite Jperp) and B = 0."""
    N, S = 4, 12
    J = W.random_couplings(N, 2)
    A = np.linspace(1.0, 0.0, S)
    B = np.linspace(0.0, 1.0, S)
    d, keep = _desc("sqa", "lhz", N, J, 3, S, L=4, beta=2.0, A=A, B=B)
    T, dmin, dmax = _tables(L, d, keep)
    assert np.array_equal(T, O.sqa_table(A, B, 2.0, 4, 0, S, dmin, dmax).ravel())


def test_pt_and_swap_tables_equal_oracle(L):
    N = 8
    J = W.random_instances(N, 2, 9)
    betas = W.geometric_ladder(32, 10.0, 0.1)
    d, keep = _desc("pt", "me", N, J, 6, 10, betas=betas)
    T, dmin, dmax = _tables(L, d, keep)
    assert np.array_equal(T, O.pt_table(betas, dmin, dmax).ravel())
    bp = np.ascontiguousarray(betas, np.float64)
    for pair in (0, 7, 30):
        n = C.c_int32()
        out = np.zeros(100000, np.uint32)
        assert L.sqa_plan_swap_table(bp.ctypes.data, len(bp), pair, out.ctypes.data, out.size, C.byref(n)) == 0
        want = [O.swap_threshold(bp[pair], bp[pair + 1], dE) for dE in range(1, n.value + 2)]
        assert list(out[:n.value]) == want[:-1]
        assert want[-1] == 0 and want[-2] > 0


@pytest.mark.parametrize("N", [2, 3, 8, 17])
def test_decoding_trees_equal_oracle(L, N):
    for inst in (0, 5):
        for tree in range(4):
            p = np.zeros(N, np.int32)
            assert L.sqa_plan_tree(N, 77, inst, tree, p.ctypes.data) == 0
            assert np.array_equal(p, O.prufer_tree(N, 77, inst, tree))


def test_validation_before_device_work(L):
    J = W.random_couplings(6, 0)
    h = C.c_void_p()
    d, keep = _desc("sqa", "lhz", 6, J, 9, 10, L=3)          # odd L
    assert L.sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_INVALID and not h.value
    d, keep = _desc("sqa", "lhz", 6, J, 0, 10)                # penalty 0
    assert L.sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_INVALID
    d, keep = _desc("pt", "me", 6, J, 6, 10, betas=[1.0, 2.0])  # increasing ladder
    assert L.sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_INVALID
    d, keep = _desc("sqa", "me", 6, J, 6, 10)
    hf = np.ones(6, np.int32)
    d.h = hf.ctypes.data
    assert L.sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_UNSUPPORTED
    assert L.sqa_create(None, C.byref(h)) == pkg.SQA_ERR_INVALID
    assert L.sqa_strerror(pkg.SQA_ERR_INVALID) == b"invalid argument"
    d, keep = _desc("sqa", "lhz", 6, J, 9, 10)
    d.move = 2                                                # no such move
    assert L.sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_INVALID
    d, keep = _desc("sqa", "lhz", 6, J, 9, 10, L=130)
    d.move = 1                                                # cluster moves need L <= 128
    assert L.sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_UNSUPPORTED
    Jbig = J.copy()
    Jbig[3] = np.iinfo(np.int32).min                          # |J| beyond any site sum
    d, keep = _desc("sqa", "me", 6, Jbig, 6, 10)
    assert L.sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_UNSUPPORTED
    d, keep = _desc("sqa", "me", 6, J, 1 << 25, 10)          # penalty beyond any site sum
    assert L.sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_UNSUPPORTED


@pytest.mark.parametrize("emb,N,S,Ls,beta", [("me", 8, 40, 64, 10 / 3), ("lhz", 6, 30, 16, 1.0)])
def test_cluster_move_tables_equal_oracle(L, emb, N, S, Ls, beta):
    """Bond thresholds and per-sweep acceptance rows, built by the library,
    equal the oracle's bond_threshold and threshold(alpha * D), bit for bit;
    each row ends where the threshold reaches 0 or at L * dmax."""
    J = W.random_instances(N, 2, 3)
    pen = 6 if emb == "me" else 9
    A, B = O.linear_schedule(S)
    A = A.copy()
    A[-3:] = 0.0                                  # infinite Jperp: bonds always join
    d, keep = _desc("sqa", emb, N, J, pen, S, L=Ls, beta=beta, A=A, B=B)
    d.move = 1
    n = C.c_int64()
    assert L.sqa_plan_wolff_tables(C.byref(d), None, None, None, None, 0, C.byref(n)) == 0
    Tb = np.zeros(S, np.uint32)
    off = np.zeros(S, np.int32)
    ln = np.zeros(S, np.int32)
    Tacc = np.zeros(max(n.value, 1), np.uint32)
    assert L.sqa_plan_wolff_tables(C.byref(d), Tb.ctypes.data, off.ctypes.data, ln.ctypes.data, Tacc.ctypes.data,
                                   len(Tacc), C.byref(n)) == 0
    dmin, dmax = C.c_int32(), C.c_int32()
    assert L.sqa_plan_tables(C.byref(d), None, 0, C.byref(dmin), C.byref(dmax)) == 0
    for t in range(S):
        assert Tb[t] == O.bond_threshold(beta, A[t], Ls)
        alpha = beta * B[t] / Ls
        row = Tacc[off[t]:off[t] + ln[t]]
        want = [O.threshold(alpha * D) for D in range(2, 2 * ln[t] + 1, 2)]
        assert np.array_equal(row, np.array(want, np.uint32))
        # the row stops at the first zero or at the largest cluster change
        if ln[t] < Ls * dmax.value // 2:
            assert O.threshold(alpha * 2 * (ln[t] + 1)) == 0
    assert Tb[-1] == 0xFFFFFFFF


def test_cluster_move_device_bytes(L):
    """The admission estimate of a cluster-move job counts its own tables
    (bond thresholds, per-sweep acceptance rows) instead of the single-spin
    threshold table."""
    J = W.random_instances(8, 3, 1)
    kw = dict(embedding="me", N=8, J=J, penalty=6, sweeps=200, R=64, L=64, beta=10 / 3)
    metro = pkg.plan_device_bytes(**kw)
    wolff = pkg.plan_device_bytes(move="wolff", **kw)
    assert metro > 0 and wolff > 0 and wolff != metro


def test_no_device_is_reported():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    J = W.random_couplings(6, 0)
    d, keep = _desc("sqa", "lhz", 6, J, 9, 10)
    h = C.c_void_p()
    assert pkg.lib().sqa_create(C.byref(d), C.byref(h)) == pkg.SQA_ERR_NO_DEVICE
    with pytest.raises(pkg.SQAError):
        pkg.Handle(embedding="lhz", N=6, J=J, penalty=9, sweeps=10, R=32)


def test_unchecked_build_reports_a_clear_status(L):
    """The normal build has no bounds checks: sqa_bounds_checked() is 0 and
    sqa_check_status() answers SQA_OK with a zero record (no device call)."""
    assert L.sqa_bounds_checked() == 0
    rec = (C.c_uint32 * 4)(7, 7, 7, 7)
    assert L.sqa_check_status(rec) == pkg.SQA_OK and list(rec) == [0, 0, 0, 0]
    assert L.sqa_check_status(None) == pkg.SQA_ERR_INVALID
    assert L.sqa_strerror(pkg.SQA_ERR_BOUNDS) == b"bounds check"


def test_checked_build_compiles_and_exports_every_symbol():
    """The bounds-checked variant (-DSQA_BOUNDS_CHECK) builds for sm_103a and
    exports the same ABI; loaded in a child process it reports itself as
    checked."""
    import subprocess
    import sys
    from paper_1603_03755_gb300 import build as b
    path = b.build(checked=True)
    names = _declared()
    code = ("import ctypes, sys; L = ctypes.CDLL(sys.argv[1]); "
            "missing = [n for n in sys.argv[2:] if not hasattr(L, n)]; "
            "assert not missing, missing; assert L.sqa_bounds_checked() == 1; print('ok')")
    r = subprocess.run([sys.executable, "-c", code, path, *names], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr


def test_slices_knob_validates_before_device_work(L):
    """sqa_tune_slices / sqa_get_task_slices answer a NULL handle with
    SQA_ERR_INVALID, before any device call."""
    v = C.c_int32()
    assert L.sqa_tune_slices(None, 2) == pkg.SQA_ERR_INVALID
    assert L.sqa_get_task_slices(None, C.byref(v)) == pkg.SQA_ERR_INVALID
