"""Python handle on the C oracle (ctypes; numpy arrays in and out).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain CPU restatement of the
SQA / PT hot path of arXiv:1603.03755 that the GPU library is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library never does.

Spin arrays are int8 sigma = +-1, shaped [Z][n][R] (Z = Trotter slices for
SQA, temperature slots for PT; n = physical sites in canonical numbering;
R = replicas).
"""
from __future__ import annotations

import ctypes as C
import math
import threading

import numpy as np

from . import build as _build

_lib = None
_lib_lock = threading.Lock()


def lib():
    global _lib
    if _lib is None:
        with _lib_lock:  # threads of one process build and load it once
            if _lib is None:
                L = C.CDLL(_build.build())
                _declare(L)
                _lib = L
    return _lib


_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_terms", C.c_int32), ("term_size", C.c_void_p),
                ("term_mem", C.c_void_p), ("term_w", C.c_void_p), ("used", C.c_void_p),
                ("colour", C.c_void_p), ("n_colours", C.c_int32), ("inc_ptr", C.c_void_p),
                ("inc_term", C.c_void_p)]


class _SqaParams(C.Structure):
    _fields_ = [("L", C.c_int32), ("R", C.c_int32), ("S", C.c_int32), ("beta", C.c_double),
                ("A", C.c_void_p), ("B", C.c_void_p), ("seed", C.c_uint64)]


class _PtParams(C.Structure):
    _fields_ = [("P", C.c_int32), ("R", C.c_int32), ("swap_every", C.c_int32),
                ("betas", C.c_void_p), ("seed", C.c_uint64)]


def _declare(L):
    i32, u32, i64, u64, dbl = C.c_int32, C.c_uint32, C.c_int64, C.c_uint64, C.c_double
    P = C.POINTER
    sig = {
        "orc_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
        "orc_me_lc": (i32, [i32]), "orc_me_n_sites": (i32, [i32]), "orc_me_n_terms": (i32, [i32]),
        "orc_me_site": (i32, [i32, i32, i32, i32, i32]),
        "orc_me_build": (i32, [i32, _i32p, i32, _i32p, _i32p, _i32p, _u8p, _i32p, _i32p, _i32p]),
        "orc_lhz_index": (i32, [i32, i32, i32]), "orc_lhz_n_sites": (i32, [i32]),
        "orc_lhz_n_terms": (i32, [i32]),
        "orc_lhz_build": (i32, [i32, _i32p, i32, _i32p, _i32p, _i32p, _u8p, _i32p]),
        "orc_incidence": (None, [i32, i32, _i32p, _i32p, _i32p, _i32p]),
        "orc_energy": (i64, [P(_Problem), _i8p, i32, i32]),
        "orc_flip_delta": (i64, [P(_Problem), _i8p, i32, i32, i32]),
        "orc_jperp": (dbl, [dbl, dbl, i32]),
        "orc_sqa_x": (dbl, [dbl, dbl, i32, i32]),
        "orc_threshold": (u32, [dbl]),
        "orc_sqa_table": (None, [_f64p, _f64p, dbl, i32, i32, i32, i32, i32, _u32p]),
        "orc_pt_table": (None, [_f64p, i32, i32, i32, _u32p]),
        "orc_swap_threshold": (u32, [dbl, dbl, i64]),
        "orc_sweep_uniform": (u32, [u64, u32, u32, u32, u32]),
        "orc_swap_uniform": (u32, [u64, u32, u32, u32, u32]),
        "orc_tree_draw": (u32, [u64, i32, i32, i32, i32]),
        "orc_init_spins": (None, [P(_Problem), i32, i32, u64, i32, _i8p]),
        "orc_sqa_run": (i32, [P(_Problem), P(_SqaParams), _i8p, i32, i32, i32, i32, i32]),
        "orc_sqa_wolff_run": (i32, [P(_Problem), P(_SqaParams), _i8p, i32, i32, i32, i32, i32]),
        "orc_bond_threshold": (u32, [dbl, dbl, i32]),
        "orc_wolff_start": (u32, [u64, u32, u32, u32, u32, i32]),
        "orc_wolff_bond_uniform": (u32, [u64, u32, u32, i32, i32, u32, u32]),
        "orc_wolff_accept_uniform": (u32, [u64, u32, u32, u32, u32]),
        "orc_pt_run": (i32, [P(_Problem), P(_PtParams), _i8p, _i64p, i32, i32, i32, i32, i32]),
        "orc_me_decode": (None, [i32, _i32p, _i32p, _i8p, _i8p]),
        "orc_prufer_tree": (None, [i32, u64, i32, i32, _i32p]),
        "orc_star_tree": (None, [i32, _i32p]), "orc_chain_tree": (None, [i32, _i32p]),
        "orc_lhz_tree_decode": (None, [i32, _i32p, _i8p, _i8p]),
        "orc_lhz_vote_decode": (None, [i32, i32, _i32p, _i8p, _i8p]),
        "orc_lhz_mwd_decode": (None, [i32, _i8p, _i8p]),
        "orc_lhz_bp_decode": (None, [i32, _i8p, dbl, i32, _i32p, _i8p]),
        "orc_logical_energy": (i64, [i32, _i32p, _i8p]),
        "orc_ground_energy": (i64, [i32, _i32p, _i8p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


class Problem:
    """A physical problem: n sites, terms w * prod(sigma), colours.

    ``embedding`` is "me" (minor embedding on Chimera, penalty = chain
    strength) or "lhz" (penalty = constraint strength lambda).
    """

    def __init__(self, embedding: str, N: int, J, penalty: int):
        L = lib()
        J = np.ascontiguousarray(J, np.int32)
        assert J.shape == (N * (N - 1) // 2,)
        self.embedding, self.N, self.J, self.penalty = embedding, N, J, int(penalty)
        if embedding == "me":
            n, nt = L.orc_me_n_sites(N), L.orc_me_n_terms(N)
            self.Lc = L.orc_me_lc(N)
        elif embedding == "lhz":
            n, nt = L.orc_lhz_n_sites(N), L.orc_lhz_n_terms(N)
        else:
            raise ValueError(embedding)
        self.n = n
        self.term_size = np.zeros(nt, np.int32)
        self.term_mem = np.full(nt * 4, -1, np.int32)
        self.term_w = np.zeros(nt, np.int32)
        self.used = np.zeros(n, np.uint8)
        self.colour = np.full(n, -1, np.int32)
        if embedding == "me":
            self.chain_sites = np.zeros(N * (self.Lc + 1), np.int32)
            self.hub = np.zeros(N, np.int32)
            got = L.orc_me_build(N, J, self.penalty, self.term_size, self.term_mem, self.term_w,
                                 self.used, self.colour, self.chain_sites, self.hub)
            self.n_colours = 2
        else:
            got = L.orc_lhz_build(N, J, self.penalty, self.term_size, self.term_mem, self.term_w,
                                  self.used, self.colour)
            self.n_colours = 4
        assert got == nt, (got, nt)
        self.n_terms = nt
        self.inc_ptr = np.zeros(n + 1, np.int32)
        self.inc_term = np.zeros(max(1, int(self.term_size.sum())), np.int32)
        L.orc_incidence(n, nt, self.term_size, self.term_mem, self.inc_ptr, self.inc_term)
        self._c = _Problem(n, nt, self.term_size.ctypes.data, self.term_mem.ctypes.data,
                           self.term_w.ctypes.data, self.used.ctypes.data, self.colour.ctypes.data,
                           self.n_colours, self.inc_ptr.ctypes.data, self.inc_term.ctypes.data)

    @property
    def c(self):
        return C.byref(self._c)

    def terms(self):
        for t in range(self.n_terms):
            sz = int(self.term_size[t])
            yield [int(x) for x in self.term_mem[4 * t:4 * t + sz]], int(self.term_w[t])

    def energy(self, sigma) -> int:
        """Energy of one configuration sigma[n] (+-1)."""
        s = np.ascontiguousarray(np.asarray(sigma, np.int8).reshape(self.n, 1))
        return int(lib().orc_energy(self.c, s, 1, 0))

    def energies(self, s) -> np.ndarray:
        """Energies of a state [n][R] -> [R]."""
        s = np.ascontiguousarray(s, np.int8)
        R = s.shape[1]
        return np.array([lib().orc_energy(self.c, s, R, r) for r in range(R)], np.int64)

    def flip_delta(self, sigma, site: int) -> int:
        s = np.ascontiguousarray(np.asarray(sigma, np.int8).reshape(self.n, 1))
        return int(lib().orc_flip_delta(self.c, s, 1, 0, site))

    def embed(self, logical) -> np.ndarray:
        """The physical image of a logical state (+-1): ME chains aligned with
        their logical spin, LHZ pair spins q_ij = s_i s_j.  Unused sites +1."""
        s = np.asarray(logical, np.int64)
        out = np.ones(self.n, np.int8)
        if self.embedding == "me":
            for i in range(self.N):
                out[self.chain_sites[i * (self.Lc + 1):(i + 1) * (self.Lc + 1)]] = s[i]
        else:
            for i in range(self.N):
                for j in range(i + 1, self.N):
                    out[lhz_index(self.N, i, j)] = s[i] * s[j]
        return out

    def delta_range(self) -> tuple[int, int]:
        """Bounds on the energy change of one flip: +-2 sum of |w| over the
        terms containing a site, maximised over sites."""
        m = 0
        for site in range(self.n):
            tot = sum(abs(int(self.term_w[t])) for t in self.inc_term[self.inc_ptr[site]:self.inc_ptr[site + 1]])
            m = max(m, tot)
        return -2 * m, 2 * m


def lhz_index(N: int, i: int, j: int) -> int:
    return i * N - i * (i + 1) // 2 + (j - i - 1)


def jperp(beta: float, A: float, L: int) -> float:
    return float(lib().orc_jperp(beta, A, L))


def sqa_x(alpha: float, jp: float, delta: int, m: int) -> float:
    return float(lib().orc_sqa_x(alpha, jp, delta, m))


def threshold(x: float) -> int:
    return int(lib().orc_threshold(float(x)))


def linear_schedule(S: int) -> tuple[np.ndarray, np.ndarray]:
    """A(s) = 1 - s, B(s) = s at s_t = (t + 1/2)/S."""
    s = (np.arange(S, dtype=np.float64) + 0.5) / S
    return 1.0 - s, s.copy()


def sqa_table(A, B, beta, L, t0, t1, dmin, dmax) -> np.ndarray:
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    nd = (dmax - dmin) // 2 + 1
    T = np.zeros((t1 - t0) * nd * 3, np.uint32)
    lib().orc_sqa_table(A, B, beta, L, t0, t1, dmin, dmax, T)
    return T.reshape(t1 - t0, nd, 3)


def pt_table(betas, dmin, dmax) -> np.ndarray:
    betas = np.ascontiguousarray(betas, np.float64)
    nd = (dmax - dmin) // 2 + 1
    T = np.zeros(len(betas) * nd, np.uint32)
    lib().orc_pt_table(betas, len(betas), dmin, dmax, T)
    return T.reshape(len(betas), nd)


def swap_threshold(bp: float, bq: float, dE: int) -> int:
    return int(lib().orc_swap_threshold(bp, bq, dE))


def sweep_uniform(seed, t, slot, rho, inst) -> int:
    return int(lib().orc_sweep_uniform(seed, t, slot, rho, inst))


def bond_threshold(beta: float, A: float, L: int) -> int:
    return int(lib().orc_bond_threshold(float(beta), float(A), L))


def wolff_start(seed, t, site, rho, inst, L) -> int:
    return int(lib().orc_wolff_start(seed, t, site, rho, inst, L))


def wolff_bond_uniform(seed, t, site, L, tau, rho, inst) -> int:
    return int(lib().orc_wolff_bond_uniform(seed, t, site, L, tau, rho, inst))


def wolff_accept_uniform(seed, t, site, rho, inst) -> int:
    return int(lib().orc_wolff_accept_uniform(seed, t, site, rho, inst))


def swap_uniform(seed, event, pair, rho, inst) -> int:
    return int(lib().orc_swap_uniform(seed, event, pair, rho, inst))


def init_spins(pb: Problem, Z: int, R: int, seed: int, inst: int) -> np.ndarray:
    s = np.zeros((Z, pb.n, R), np.int8)
    lib().orc_init_spins(pb.c, Z, R, seed, inst, s)
    return s


class SQA:
    """Path-integral SQA of one instance; state [L][n][R] int8.  move is
    "metropolis" (single-spin sweep) or "wolff" (one time-like cluster move
    per site and replica per sweep)."""

    def __init__(self, pb: Problem, L: int, R: int, beta: float, A, B, seed: int, inst: int = 0,
                 move: str = "metropolis"):
        if move not in ("metropolis", "wolff"):
            raise ValueError("move is 'metropolis' or 'wolff'")
        self.move = move
        self.pb, self.L, self.R, self.beta, self.seed, self.inst = pb, L, R, beta, seed, inst
        self.A = np.ascontiguousarray(A, np.float64)
        self.B = np.ascontiguousarray(B, np.float64)
        self.S = len(self.A)
        self._prm = _SqaParams(L, R, self.S, beta, self.A.ctypes.data, self.B.ctypes.data, seed)
        self.s = init_spins(pb, L, R, seed, inst)

    def run(self, t0: int, t1: int, rho0: int = 0, rho1: int | None = None):
        rho1 = self.R if rho1 is None else rho1
        run = lib().orc_sqa_wolff_run if self.move == "wolff" else lib().orc_sqa_run
        rc = run(self.pb.c, C.byref(self._prm), self.s, self.inst, t0, t1, rho0, rho1)
        if rc != 0:
            raise ValueError("orc_sqa_run rejected its arguments")
        return self.s

    def slice_energies(self) -> np.ndarray:
        """E_P of every slice and replica, [L][R]."""
        return np.stack([self.pb.energies(self.s[z]) for z in range(self.L)])


class PT:
    """Parallel tempering of one instance; state [P][n][R] int8."""

    def __init__(self, pb: Problem, betas, R: int, swap_every: int, seed: int, inst: int = 0):
        self.pb, self.R, self.swap_every, self.seed, self.inst = pb, R, swap_every, seed, inst
        self.betas = np.ascontiguousarray(betas, np.float64)
        self.P = len(self.betas)
        self._prm = _PtParams(self.P, R, swap_every, self.betas.ctypes.data, seed)
        self.s = init_spins(pb, self.P, R, seed, inst)
        self.E = np.zeros((self.P, R), np.int64)

    def run(self, t0: int, t1: int, rho0: int = 0, rho1: int | None = None):
        rho1 = self.R if rho1 is None else rho1
        rc = lib().orc_pt_run(self.pb.c, C.byref(self._prm), self.s, self.E, self.inst, t0, t1,
                              rho0, rho1)
        if rc != 0:
            raise ValueError("orc_pt_run rejected its arguments")
        return self.s


# ---- decoding ----

def me_decode(pb: Problem, phys) -> np.ndarray:
    out = np.zeros(pb.N, np.int8)
    lib().orc_me_decode(pb.N, pb.chain_sites, pb.hub, np.ascontiguousarray(phys, np.int8), out)
    return out


def star_tree(N: int) -> np.ndarray:
    p = np.zeros(N, np.int32)
    lib().orc_star_tree(N, p)
    return p


def chain_tree(N: int) -> np.ndarray:
    p = np.zeros(N, np.int32)
    lib().orc_chain_tree(N, p)
    return p


def prufer_tree(N: int, seed: int, inst: int, tree: int) -> np.ndarray:
    p = np.zeros(N, np.int32)
    lib().orc_prufer_tree(N, seed, inst, tree, p)
    return p


def tree_draw(seed, inst, tree, pos, N) -> int:
    return int(lib().orc_tree_draw(seed, inst, tree, pos, N))


def lhz_tree_decode(N: int, parent, phys) -> np.ndarray:
    out = np.zeros(N, np.int8)
    lib().orc_lhz_tree_decode(N, np.ascontiguousarray(parent, np.int32),
                              np.ascontiguousarray(phys, np.int8), out)
    return out


def lhz_mwd_decode(N: int, phys) -> np.ndarray:
    """Minimum-weight decoding (exact, by enumeration; q_{N-1} = +1)."""
    out = np.zeros(N, np.int8)
    lib().orc_lhz_mwd_decode(N, np.ascontiguousarray(phys, np.int8), out)
    return out


def lhz_bp_decode(N: int, phys, error_rate: float, iterations: int, parent) -> np.ndarray:
    """Belief-propagation decoding: iterated weighted majority over the N-2
    parity checks of every pair, then a spanning-tree readout."""
    out = np.zeros(N, np.int8)
    lib().orc_lhz_bp_decode(N, np.ascontiguousarray(phys, np.int8), float(error_rate), int(iterations),
                            np.ascontiguousarray(parent, np.int32), out)
    return out


def lhz_vote_decode(N: int, parents, phys) -> np.ndarray:
    parents = np.ascontiguousarray(parents, np.int32)
    out = np.zeros(N, np.int8)
    lib().orc_lhz_vote_decode(N, parents.shape[0], parents.reshape(-1),
                              np.ascontiguousarray(phys, np.int8), out)
    return out


def logical_energy(N: int, J, s) -> int:
    return int(lib().orc_logical_energy(N, np.ascontiguousarray(J, np.int32),
                                        np.ascontiguousarray(s, np.int8)))


def ground_energy(N: int, J) -> tuple[int, np.ndarray]:
    s = np.zeros(N, np.int8)
    e = int(lib().orc_ground_energy(N, np.ascontiguousarray(J, np.int32), s))
    return e, s


def default_n_trees(N: int) -> int:
    """Votes for LHZ tree decoding: the ME chain length ceil(N/4) + 1, made odd."""
    n = math.ceil(N / 4) + 1
    return n if n % 2 else n + 1


def pack_bits(sigma: np.ndarray) -> np.ndarray:
    """[..., R] int8 sigma -> [..., ceil(R/32)] uint32 words (bit = sigma<0)."""
    s = np.asarray(sigma)
    R = s.shape[-1]
    W = (R + 31) // 32
    bits = np.zeros(s.shape[:-1] + (W * 32,), np.uint64)
    bits[..., :R] = (s < 0)
    bits = bits.reshape(s.shape[:-1] + (W, 32))
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (bits * weights).sum(axis=-1).astype(np.uint32)


def unpack_bits(words: np.ndarray, R: int) -> np.ndarray:
    """Inverse of :func:`pack_bits`."""
    w = np.asarray(words, np.uint32)
    bits = (w[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    bits = bits.reshape(w.shape[:-1] + (w.shape[-1] * 32,))[..., :R]
    return np.where(bits == 1, -1, 1).astype(np.int8)
