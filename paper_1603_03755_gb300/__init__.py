"""GB300 (sm_103a) library for the SQA / PT hot path of arXiv:1603.03755.

A thin ctypes binding over ``_build/libsqa_gb300.so`` (C ABI in
``include/sqa.h``).  Every step of the path runs in the library's CUDA
kernels; this module only marshals arguments.  PyTorch supplies device
buffers and streams.  There is no CPU fallback: importing works without a
GPU, but every compute call needs the compiled library and a CUDA device and
raises otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SQA_OK, SQA_ERR_INVALID, SQA_ERR_UNSUPPORTED, SQA_ERR_NOMEM = 0, -1, -2, -3
SQA_ERR_CUDA, SQA_ERR_TIMEOUT, SQA_ERR_NO_DEVICE, SQA_ERR_BUSY = -4, -5, -6, -7
SQA_ERR_BOUNDS = -8
EMB = {"me": 0, "lhz": 1}
KIND = {"sqa": 0, "pt": 1}
MOVE = {"metropolis": 0, "wolff": 1}
DECODE = {"me_mv": 0, "lhz_trees": 1, "lhz_star": 2, "lhz_chain": 3, "lhz_mwd": 4, "lhz_bp": 5}

# SQA_GB300_CHECKED=1 loads the bounds-checked build (see build.build(checked=True))
CHECKED = os.environ.get("SQA_GB300_CHECKED", "") == "1"
LIB_PATH = _build.LIB_CHECKED if CHECKED else _build.LIB


class SQAError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({detail})")


class _Desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("embedding", C.c_int32), ("n_logical", C.c_int32),
                ("n_instances", C.c_int32), ("J", C.c_void_p), ("h", C.c_void_p),
                ("penalty", C.c_int32), ("n_sweeps", C.c_int32), ("n_replicas", C.c_int32),
                ("seed", C.c_uint64), ("n_slices", C.c_int32), ("beta", C.c_double),
                ("A", C.c_void_p), ("B", C.c_void_p), ("n_temps", C.c_int32),
                ("betas", C.c_void_p), ("swap_every", C.c_int32), ("move", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("n_phys", C.c_int32), ("n_used", C.c_int32), ("n_terms", C.c_int32),
                ("z", C.c_int32), ("words", C.c_int32), ("delta_min", C.c_int32),
                ("delta_max", C.c_int32), ("attempts_per_sweep", C.c_int64),
                ("device_bytes", C.c_int64), ("h2d_bytes", C.c_int64),
                ("launches_per_run", C.c_int32), ("pad_", C.c_int32)]


# Every symbol the header declares, with its ctypes signature.
_SIGS = {
    "sqa_create": (C.c_int, [C.POINTER(_Desc), C.POINTER(C.c_void_p)]),
    "sqa_destroy": (None, [C.c_void_p]),
    "sqa_get_info": (C.c_int, [C.c_void_p, C.POINTER(_Info)]),
    "sqa_tune": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "sqa_tune_slices": (C.c_int, [C.c_void_p, C.c_int32]),
    "sqa_get_task_slices": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "sqa_get_launch": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32)]),
    "sqa_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sqa_run_sweeps": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    "sqa_run_per_instance": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pt_run": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "sqa_batch_run": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "sqa_batch_create": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "sqa_batch_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sqa_batch_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double)]),
    "sqa_batch_destroy": (None, [C.c_void_p]),
    "sqa_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "sqa_readout": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sqa_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sqa_energies": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sqa_decode": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_int32, C.c_void_p]),
    "sqa_decode_bp": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_int32, C.c_void_p]),
    "sqa_ground_energy": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]),
    "sqa_ground_energy_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sqa_plan_terms": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sqa_plan_tables": (C.c_int, [C.POINTER(_Desc), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "sqa_plan_swap_table": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]),
    "sqa_plan_wolff_tables": (C.c_int, [C.POINTER(_Desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int64, C.POINTER(C.c_int64)]),
    "sqa_plan_tree": (C.c_int, [C.c_int32, C.c_uint64, C.c_int32, C.c_int32, C.c_void_p]),
    "sqa_int_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double)]),
    "sqa_bounds_checked": (C.c_int32, []),
    "sqa_check_status": (C.c_int, [C.POINTER(C.c_uint32)]),
    "sqa_server_create": (C.c_int, [C.c_int64, C.c_int64, C.POINTER(C.c_void_p)]),
    "sqa_server_submit": (C.c_int, [C.c_void_p, C.POINTER(_Desc), C.POINTER(C.c_uint64)]),
    "sqa_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p]),
    "sqa_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double]),
    "sqa_server_result": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    "sqa_server_release": (C.c_int, [C.c_void_p, C.c_uint64]),
    "sqa_server_get_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sqa_server_destroy": (None, [C.c_void_p]),
    "sqa_plan_device_bytes": (C.c_int64, [C.POINTER(_Desc)]),
    "sqa_strerror": (C.c_char_p, [C.c_int]),
    "sqa_last_error": (C.c_char_p, []),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded library.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1603_03755_gb300.build.build("
                              f"{'checked=True' if CHECKED else ''})")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != SQA_OK:
        detail = lib().sqa_last_error().decode(errors="replace")
        raise SQAError(status, where, detail)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x):
    """(address, is_device) of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, 0
    assert x.is_contiguous()
    return x.data_ptr(), int(x.is_cuda)


def _make_desc(*, embedding: str, N: int, J, penalty: int, sweeps: int, R: int, seed: int = 0,
               kind: str = "sqa", L: int = 32, beta: float = 1.0, A=None, B=None, betas=None,
               swap_every: int = 1, move: str = "metropolis"):
    """An sqa_desc and the arrays it points into (keep them alive)."""
    J = np.ascontiguousarray(np.atleast_2d(np.asarray(J, np.int32)))
    keep = [J]
    d = _Desc()
    d.kind, d.embedding, d.n_logical, d.n_instances = KIND[kind], EMB[embedding], N, J.shape[0]
    d.J = J.ctypes.data
    d.h = None
    d.penalty, d.n_sweeps, d.n_replicas, d.seed = int(penalty), int(sweeps), int(R), int(seed)
    d.n_slices, d.beta = int(L), float(beta)
    if A is not None:
        A = np.ascontiguousarray(A, np.float64)
        B = np.ascontiguousarray(B, np.float64)
        keep += [A, B]
        d.A, d.B = A.ctypes.data, B.ctypes.data
    if betas is not None:
        betas = np.ascontiguousarray(betas, np.float64)
        keep.append(betas)
        d.betas, d.n_temps = betas.ctypes.data, len(betas)
    d.swap_every = int(swap_every)
    d.move = MOVE[move]
    meta = {"N": N, "I": J.shape[0], "R": int(R), "kind": kind, "embedding": embedding,
            "Z": int(L) if kind == "sqa" else (len(betas) if betas is not None else 0)}
    return d, keep, meta


def plan_n_phys(embedding: str, N: int) -> int:
    """Canonical physical sites of an embedding of K_N (host only)."""
    return 8 * ((N + 3) // 4) ** 2 if embedding == "me" else N * (N - 1) // 2


def plan_device_bytes(**kw) -> int:
    """Device bytes sqa_create would allocate (host only)."""
    d, keep, _ = _make_desc(**kw)
    return int(lib().sqa_plan_device_bytes(C.byref(d)))


class Handle:
    """One problem (I instances sharing every parameter but J) and its
    resident device state.  ``kind`` 'sqa' or 'pt'; ``embedding`` 'me' or
    'lhz'.  J has shape [I, N(N-1)/2] (int32)."""

    def __init__(self, **kw):
        d, keep, meta = _make_desc(**kw)
        self.N, self.I, self.R, self.kind, self.embedding = meta["N"], meta["I"], meta["R"], meta["kind"], meta["embedding"]
        self._keep = keep
        h = C.c_void_p()
        _check(lib().sqa_create(C.byref(d), C.byref(h)), "sqa_create")
        self._h = h
        self._refresh_info()

    def _refresh_info(self):
        info = _Info()
        _check(lib().sqa_get_info(self._h, C.byref(info)), "sqa_get_info")
        self.info = {k: getattr(info, k) for k, _ in _Info._fields_}

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().sqa_destroy(self._h)
            self._h = None

    __del__ = close

    # ---- launch shape ----
    def tune(self, words_per_unit: int = 0, use_table: int = -1, cluster: int = 0):
        _check(lib().sqa_tune(self._h, words_per_unit, use_table, cluster), "sqa_tune")

    def tune_slices(self, slices: int = 0):
        """Slices (or slots) per thread's task of the sweep, 1..4; 0 = automatic."""
        _check(lib().sqa_tune_slices(self._h, int(slices)), "sqa_tune_slices")

    def autotune(self, n_trial: int = 20, stream=None) -> dict:
        """Times every launch shape that fits on n_trial sweeps and keeps the
        fastest (spins saved and restored); returns the choice."""
        wc, lut, cl, rate = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        _check(lib().sqa_autotune(self._h, int(n_trial), _stream_ptr(stream), C.byref(wc), C.byref(lut),
                                  C.byref(cl), C.byref(rate)), "sqa_autotune")
        return {"words_per_unit": wc.value, "use_table": lut.value, "cluster": cl.value,
                "trial_attempts_per_s": rate.value}

    def launch(self) -> dict:
        wc, lut, smem, cl = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().sqa_get_launch(self._h, C.byref(wc), C.byref(lut), C.byref(smem), C.byref(cl)),
               "sqa_get_launch")
        ts = C.c_int32()
        _check(lib().sqa_get_task_slices(self._h, C.byref(ts)), "sqa_get_task_slices")
        return {"words_per_unit": wc.value, "use_table": lut.value, "smem_bytes": smem.value,
                "cluster": cl.value, "task_slices": ts.value}

    # ---- running ----
    def run(self, stream=None):
        _check(lib().sqa_run(self._h, _stream_ptr(stream)), "sqa_run")

    def run_sweeps(self, t0: int, t1: int, stream=None):
        _check(lib().sqa_run_sweeps(self._h, t0, t1, _stream_ptr(stream)), "sqa_run_sweeps")

    def run_per_instance(self, stream=None):
        _check(lib().sqa_run_per_instance(self._h, _stream_ptr(stream)), "sqa_run_per_instance")

    def pt_run(self, betas, sweeps: int, swap_every: int, stream=None):
        b = np.ascontiguousarray(betas, np.float64)
        _check(lib().pt_run(self._h, b.ctypes.data, len(b), sweeps, swap_every, _stream_ptr(stream)), "pt_run")
        self.kind = "pt"
        self._refresh_info()

    # ---- outputs (numpy on the host, or torch tensors given as out=) ----
    def _words_out(self, fn, zc, out, stream):
        shape = (self.I, zc, self.info["n_phys"], self.info["words"])
        if out is None:
            out = np.zeros(shape, np.uint32)
        p, dev = _ptr(out)
        _check(fn(self._h, p, dev, _stream_ptr(stream)), fn.__name__)
        return out

    def readout(self, out=None, stream=None):
        """Slice 0 / coldest slot, [I, n_phys, W] uint32."""
        if out is None:
            out = np.zeros((self.I, self.info["n_phys"], self.info["words"]), np.uint32)
        p, dev = _ptr(out)
        _check(lib().sqa_readout(self._h, p, dev, _stream_ptr(stream)), "sqa_readout")
        return out

    def state(self, out=None, stream=None):
        """All slices / slots, [I, Z, n_phys, W] uint32."""
        return self._words_out(lib().sqa_state, self.info["z"], out, stream)

    def energies(self, out=None, stream=None):
        """E_P per (instance, slice/slot, replica), [I, Z, R] int32."""
        if out is None:
            out = np.zeros((self.I, self.info["z"], self.R), np.int32)
        p, dev = _ptr(out)
        _check(lib().sqa_energies(self._h, p, dev, _stream_ptr(stream)), "sqa_energies")
        return out

    def decode_bp(self, error_rate: float = 0.2, iterations: int = 10, e_ground=None, stream=None):
        """Belief-propagation decoding (LHZ); returns as decode()."""
        logical = np.zeros((self.I, self.R, self.N), np.int8)
        energy = np.zeros((self.I, self.R), np.int64)
        succ = np.zeros(self.I, np.int32)
        eg = None if e_ground is None else np.ascontiguousarray(e_ground, np.int64)
        _check(lib().sqa_decode_bp(self._h, float(error_rate), int(iterations), logical.ctypes.data,
                                   energy.ctypes.data, None if eg is None else eg.ctypes.data,
                                   succ.ctypes.data if eg is not None else None, 0, _stream_ptr(stream)),
               "sqa_decode_bp")
        return logical, energy, (succ if eg is not None else None)

    def decode(self, method: str | None = None, n_trees: int = 0, e_ground=None, stream=None):
        """Host arrays: logical [I, R, N] int8, energy [I, R] int64, success [I] int32
        (None unless e_ground is given)."""
        if method is None:
            method = "me_mv" if self.embedding == "me" else "lhz_trees"
        logical = np.zeros((self.I, self.R, self.N), np.int8)
        energy = np.zeros((self.I, self.R), np.int64)
        succ = np.zeros(self.I, np.int32)
        eg = None
        if e_ground is not None:
            eg = np.ascontiguousarray(e_ground, np.int64)
        _check(lib().sqa_decode(self._h, DECODE[method], n_trees, logical.ctypes.data,
                                energy.ctypes.data, None if eg is None else eg.ctypes.data,
                                succ.ctypes.data if eg is not None else None, 0, _stream_ptr(stream)),
               "sqa_decode")
        return logical, energy, (succ if eg is not None else None)


class _JobInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("device_bytes", C.c_int64)]


class _ServerStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("jobs_submitted", "jobs_done", "jobs_failed", "chunks", "attempts",
                                         "resident", "queued", "max_resident", "bytes_in_use", "max_bytes")] + \
               [(n, C.c_double) for n in ("admit_s", "advance_s", "idle_s")] + \
               [("worker_status", C.c_int32), ("pad_", C.c_int32), ("packs", C.c_int64),
                ("pack_s", C.c_double), ("retire_s", C.c_double), ("create_s", C.c_double), ("pad2_", C.c_double)]


JOB_STATES = ("queued", "running", "done", "failed")


class Server:
    """Continuous-batching server on the current CUDA device (a worker thread
    in the library).  submit() takes the same keywords as Handle."""

    def __init__(self, mem_budget_bytes: int, unit_attempts_per_chunk: int = 0):
        s = C.c_void_p()
        _check(lib().sqa_server_create(int(mem_budget_bytes), int(unit_attempts_per_chunk), C.byref(s)),
               "sqa_server_create")
        self._s = s
        self._meta = {}

    def submit(self, **kw) -> int:
        d, keep, meta = _make_desc(**kw)
        jid = C.c_uint64()
        _check(lib().sqa_server_submit(self._s, C.byref(d), C.byref(jid)), "sqa_server_submit")
        meta["n_phys"] = plan_n_phys(meta["embedding"], meta["N"])
        self._meta[jid.value] = meta
        return jid.value

    def poll(self, job_id: int) -> dict:
        info = _JobInfo()
        _check(lib().sqa_server_poll(self._s, job_id, C.byref(info)), "sqa_server_poll")
        out = {k: getattr(info, k) for k, _ in _JobInfo._fields_}
        out["state"] = JOB_STATES[out["state"]]
        return out

    def wait(self, job_id: int, timeout: float = 600.0):
        _check(lib().sqa_server_wait(self._s, job_id, float(timeout)), "sqa_server_wait")

    def result(self, job_id: int):
        """(state [I, Z, n_phys, W] uint32, energies [I, Z, R] int32)."""
        m = self._meta[job_id]
        W = (m["R"] + 31) // 32
        st = np.zeros((m["I"], m["Z"], m["n_phys"], W), np.uint32)
        en = np.zeros((m["I"], m["Z"], m["R"]), np.int32)
        _check(lib().sqa_server_result(self._s, job_id, st.ctypes.data, en.ctypes.data), "sqa_server_result")
        return st, en

    def release(self, job_id: int):
        _check(lib().sqa_server_release(self._s, job_id), "sqa_server_release")
        self._meta.pop(job_id, None)

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().sqa_server_get_stats(self._s, C.byref(st)), "sqa_server_get_stats")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_ if not k.startswith("pad")}

    def close(self):
        if getattr(self, "_s", None):
            lib().sqa_server_destroy(self._s)
            self._s = None

    __del__ = close


def batch_run(handles, stream=None):
    """One persistent launch over every unit of several handles."""
    arr = (C.c_void_p * len(handles))(*[h.handle for h in handles])
    _check(lib().sqa_batch_run(arr, len(handles), _stream_ptr(stream)), "sqa_batch_run")


class Batch:
    """Several handles planned once for one persistent launch, replayed from
    a CUDA graph.  The handles must stay open (and untuned) while it lives."""

    def __init__(self, handles):
        self._hs = list(handles)
        arr = (C.c_void_p * len(self._hs))(*[h.handle for h in self._hs])
        b = C.c_void_p()
        _check(lib().sqa_batch_create(arr, len(self._hs), C.byref(b)), "sqa_batch_create")
        self._b = b

    def launch(self, stream=None):
        _check(lib().sqa_batch_launch(self._b, _stream_ptr(stream)), "sqa_batch_launch")

    def autotune(self, n_trial: int = 20, stream=None) -> dict:
        wc, rate = C.c_int32(), C.c_double()
        _check(lib().sqa_batch_autotune(self._b, int(n_trial), _stream_ptr(stream), C.byref(wc), C.byref(rate)),
               "sqa_batch_autotune")
        return {"words_per_unit": wc.value, "trial_attempts_per_s": rate.value}

    def close(self):
        if self._b:
            lib().sqa_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ground_energy(N: int, J) -> np.ndarray:
    """Exact logical ground-state energies on the GPU, J [I, N(N-1)/2]."""
    J = np.ascontiguousarray(np.atleast_2d(np.asarray(J, np.int32)))
    out = np.zeros(J.shape[0], np.int64)
    _check(lib().sqa_ground_energy(N, J.shape[0], J.ctypes.data, out.ctypes.data), "sqa_ground_energy")
    return out


INT_PEAK_KINDS = ("lop3", "iadd3", "imad", "imad_wide", "imad_hi", "lop3_imad", "philox_blocks",
                  "philox_wide_blocks")


def check_status() -> tuple[int, list[int]]:
    """Status and record of the bounds checks since the last call (a
    bounds-checked build; an unchecked one returns SQA_OK and zeros):
    [violations, check site, index, bound]."""
    rec = (C.c_uint32 * 4)()
    st = lib().sqa_check_status(rec)
    return st, list(rec)


def int_peak(kind: str) -> float:
    """Measured integer lane-ops per SM clock for one instruction kind."""
    v = C.c_double()
    _check(lib().sqa_int_peak(INT_PEAK_KINDS.index(kind), C.byref(v)), "sqa_int_peak")
    return v.value


def ground_energy_noalloc(N: int, J_dev, e_dev, stream=None):
    """Allocation-free ground-state search: J_dev [I, N(N-1)/2] int32 and
    e_dev [I] int64 are caller-owned CUDA tensors; asynchronous on stream."""
    import torch

    I = e_dev.shape[0] if e_dev.dim() == 1 else -1
    if not (J_dev.is_cuda and e_dev.is_cuda and J_dev.is_contiguous() and e_dev.is_contiguous()):
        raise ValueError("ground_energy_noalloc: J_dev and e_dev must be contiguous CUDA tensors")
    if J_dev.dtype != torch.int32 or e_dev.dtype != torch.int64:
        raise ValueError("ground_energy_noalloc: J_dev must be int32 and e_dev int64")
    if I < 1 or tuple(J_dev.shape) != (I, N * (N - 1) // 2):
        raise ValueError(f"ground_energy_noalloc: J_dev must be [I, N(N-1)/2] and e_dev [I], "
                         f"got {tuple(J_dev.shape)} and {tuple(e_dev.shape)}")
    cur = torch.cuda.current_device()
    if J_dev.device.index != cur or e_dev.device.index != cur:
        raise ValueError("ground_energy_noalloc: J_dev and e_dev must be on the current CUDA device")
    _check(lib().sqa_ground_energy_noalloc(N, e_dev.shape[0], J_dev.data_ptr(), e_dev.data_ptr(),
                                           _stream_ptr(stream)), "sqa_ground_energy_noalloc")


def unpack_words(words, R: int) -> np.ndarray:
    """[..., W] uint32 -> [..., R] int8 sigma (+1 / -1)."""
    w = np.asarray(words, np.uint32)
    bits = (w[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    bits = bits.reshape(w.shape[:-1] + (w.shape[-1] * 32,))[..., :R]
    return np.where(bits == 1, -1, 1).astype(np.int8)
