"""Benchmark of the SQA hot path: spin-flip attempts/s on one GB300.

Workload (one step): ME of K_8 on a 2x2 Chimera (24 used of 32 sites, chains
of 3, J_F = -2 max|J|), 1024 instances x 256 replicas, L = 64 Trotter slices,
1e4 sweeps of the linear schedule at beta = 10/max|J|.  A step runs the whole
path on the device: initial spins, the 1e4 sweeps (one persistent launch),
energies of every slice, the readout and its majority-vote decoding with
success counts.  Inputs (couplings, tables) are resident when the timed region
starts; L2 is flushed between steps by writing a 256 MiB buffer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU oracle (the only reference this method has:
the paper publishes no code) on a bounded sample of the same workload.
Under torchrun every rank runs the whole workload (weak scaling, independent
replicas); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The serving loop keeps many streams' work in flight (chunks, packs, uploads,
# result copies); with the default 8 hardware work queues unrelated streams
# share queues and wait on each other.  Set before CUDA starts (a serving
# deployment sets it the same way); no other part of the bench depends on it.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import workloads as W  # noqa: E402

METRIC = "spin-flip attempts/s batched vs one-launch-per-instance; p50/p99 job latency"
UNIT = "attempts/s"
# Integer operations one attempt needs in this formulation (per replica):
# 16 random bits = 1/8 of a Philox4x32-10 block (10 rounds x 2 IMAD.WIDE +
# 2 LOP3 = 40) -> 5; threshold-index extraction 2; table load, compare and
# flip-mask update 3.  Work shared by the 32 replicas of a word is not counted.
OPS_PER_ATTEMPT = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps", type=int, default=10_000, help="sweeps per anneal (default: the workload's 1e4)")
    ap.add_argument("--instances", type=int, default=1024)
    ap.add_argument("--per-instance-sample", type=int, default=8,
                    help="instances timed on the one-launch-per-instance path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the planner's launch shape (profiling captures then see only timed launches)")
    ap.add_argument("--no-extra", action="store_true", help="skip the ragged-batch and PT workloads")
    ap.add_argument("--pt-sweeps", type=int, default=100_000)
    ap.add_argument("--ragged-sweeps", type=int, default=10_000)
    ap.add_argument("--pt-instances", type=int, default=256)
    ap.add_argument("--wolff-sweeps", type=int, default=2000)
    ap.add_argument("--scan-sweeps", type=int, default=2000)
    ap.add_argument("--wolff-only", action="store_true",
                    help="time only the cluster-move workload (a small case for profiling with --instances)")
    ap.add_argument("--pt-only", choices=["me", "lhz"],
                    help="time only the PT workload on this embedding (a small case for profiling)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving measurement")
    ap.add_argument("--serving-capacity", type=float, default=0.0, metavar="ATTEMPTS_PER_S",
                    help="offered loads relative to this rate (default: the server's saturated rate on the "
                         "same job stream, measured first)")
    ap.add_argument("--serving-jobs", type=int, default=200)
    return ap.parse_args()


def kernels_code_sha256(path):
    """SHA-256 of a CUDA source with its comments and whitespace removed, so
    that the record below follows the code, not the comments."""
    import hashlib
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return hashlib.sha256(" ".join(src.split()).encode()).hexdigest()


def kernel_capture(n_instances):
    """The committed ncu capture of the sweep kernel: DRAM bytes of one launch
    (read + write per instance, scaled to n_instances) and the kernel's own
    instruction counters (warp instructions x 32 per attempt, issue-active
    fraction, pipe utilisation).  None when the code of kernels.cu changed
    since that capture."""
    p = os.path.join(ROOT, "profiles", "sweep_kernel_traffic.json")
    src = os.path.join(ROOT, "paper_1603_03755_gb300", "csrc", "kernels.cu")
    if not os.path.exists(p):
        return None, "no capture", None
    rec = json.load(open(p))
    if rec.get("kernels_cu_code_sha256") != kernels_code_sha256(src):
        return None, "kernel changed since the capture", None
    counters = {k: rec.get(k) for k in ("instr_per_attempt", "issue_active", "pipe_alu", "pipe_fma",
                                        "shared_bank_conflicts_per_wavefront")}
    return rec["dram_bytes_per_instance"] * n_instances, rec["note"], counters


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {}, "fallback"


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except FileNotFoundError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 8 for k in range(4)
                          if r[4 + k].lower() == "active"})
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": reasons}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return world, rank, local, dist
    return 1, 0, 0, None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_sample(cfg, seconds_budget=15.0, first_instance=0):
    """The oracle, as it stands, on instance(s) of the workload: 32 replicas,
    the first sweeps of the same 1e4-sweep schedule.  Returns (attempts/s,
    description, attempts)."""
    import oracle as O
    N, L, pen, beta, S = cfg["N"], cfg["L"], cfg["penalty"], cfg["beta"], cfg["sweeps"]
    A, B = O.linear_schedule(S)
    pb = O.Problem("me", N, cfg["J"][first_instance], pen)
    R = 32
    q = O.SQA(pb, L, R, beta, A, B, cfg["seed"], first_instance)
    n_used = int(pb.used.sum())
    t0 = time.perf_counter()
    t = 0
    chunk = 50
    while time.perf_counter() - t0 < seconds_budget and t + chunk <= S:
        q.run(t, t + chunk)
        t += chunk
    dt = time.perf_counter() - t0
    attempts = n_used * L * R * t
    desc = f"instance {first_instance}, replicas 0-31, sweeps 0-{t - 1} of the {S}-sweep anneal, 1 thread"
    return attempts / dt, desc, attempts


def cpu_oracle_all_cores(cfg, seconds_budget=10.0):
    """The same oracle on every host core at once: one thread per core, each
    annealing its own instance (the oracle keeps no global state; its C calls
    release the GIL).  Returns (attempts/s, threads, description)."""
    from concurrent.futures import ThreadPoolExecutor
    n = os.cpu_count() or 1
    with ThreadPoolExecutor(n) as ex:
        res = list(ex.map(lambda k: cpu_oracle_sample(cfg, seconds_budget, k % cfg["J"].shape[0]), range(n)))
    t_wall = seconds_budget  # every thread stops at the same budget
    total = sum(r[2] for r in res)
    rates = sum(r[0] for r in res)
    return rates, n, (f"{n} threads, instance k on thread k, replicas 0-31, the first sweeps of the "
                      f"1e4-sweep anneal for {t_wall:.0f} s each; value = sum of the threads' rates "
                      f"({total:.3g} attempts)")


def timed(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1) / 1e3


def extra_workloads(pkg, stream, args):
    """The ragged LHZ/ME mix in one persistent launch, and PT on ME K_32 and
    LHZ K_24 (32 temperatures, swap every sweep).  Each timed once after a
    short warm-up run of the same shapes."""
    sp = stream.cuda_stream
    out = {}
    jobs = W.ragged_mix_config(512, R=128, sweeps=args.ragged_sweeps)

    def make(js, sweeps):
        return [pkg.Handle(embedding=j["embedding"], N=j["N"], J=j["J"], penalty=j["penalty"], sweeps=sweeps,
                           R=j["R"], seed=j["seed"], L=j["L"], beta=j["beta"]) for j in js]

    warm = make(jobs, 20)
    pkg.batch_run(warm, stream=sp)
    stream.synchronize()
    for h in warm:
        h.close()
    hs = make(jobs, args.ragged_sweeps)
    att = sum(h.info["attempts_per_sweep"] for h in hs) * args.ragged_sweeps
    t_plain = timed(stream, lambda: pkg.batch_run(hs, stream=sp))
    b = pkg.Batch(hs)
    tune = b.autotune(n_trial=50, stream=sp)
    b.launch(stream=sp)                                  # captures the graph
    t = timed(stream, lambda: b.launch(stream=sp))       # replays it
    out["ragged_mix"] = {"workload": f"ragged LHZ N 8-16 / ME N 8-16, L 32/64, 512 instances x 128 replicas, "
                                     f"{args.ragged_sweeps} sweeps, one persistent launch replayed from a CUDA "
                                     f"graph, words per unit autotuned",
                         "value": att / t, "unit": UNIT, "seconds": t, "autotune": tune,
                         "planner_shapes_batch_run": {"value": att / t_plain, "seconds": t_plain}}
    b.close()
    for h in hs:
        h.close()
    out.update(pt_workloads(pkg, stream, args, ("me", "lhz")))
    out["wolff_me"] = wolff_workload(pkg, stream, args)
    out["penalty_scans"] = scan_workloads(pkg, stream, args)
    if not args.no_serving:
        out.update(serving_suite(pkg, args))
    return out


def wolff_workload(pkg, stream, args):
    """The benchmark's ME K_8 anneal (1024 instances x 256 replicas, L = 64)
    with one time-like cluster move per (site, replica) per sweep instead of
    single-spin sweeps.  Reported per (site, slice, replica) per sweep, the
    unit of the single-spin attempts, and per cluster move."""
    sp = stream.cuda_stream
    cfg = W.me_n8_batch_config(n_inst=args.instances, sweeps=args.wolff_sweeps)
    kw = dict(embedding="me", N=cfg["N"], J=cfg["J"], penalty=cfg["penalty"], R=cfg["R"], seed=cfg["seed"],
              L=cfg["L"], beta=cfg["beta"], move="wolff")
    w = pkg.Handle(sweeps=20, **kw)
    w.run(stream=sp)
    stream.synchronize()
    w.close()
    h = pkg.Handle(sweeps=args.wolff_sweeps, **kw)
    spin_slices = h.info["attempts_per_sweep"] * args.wolff_sweeps
    moves = spin_slices // cfg["L"]
    t = timed(stream, lambda: h.run(stream=sp))
    out = {"workload": cfg["name"] + ", time-like cluster moves", "value": spin_slices / t,
           "unit": "spin-slice updates/s", "cluster_moves_per_s": moves / t, "seconds": t, "launch": h.launch()}
    h.close()
    return out


def scan_workloads(pkg, stream, args):
    """Penalty scans of 32 K_8 instances (J in {+-1, +-2, +-3}) at penalties
    1, 2, 3, 4, 6, 8, 10, 12, each scan one batch launch: SQA (L = 64, beta = 1,
    256 readouts per instance and penalty) for the optimal penalty, and PT on
    the paper's ladder (32 temperatures, beta 20 down to 0.1, readouts from
    beta = 20) for the critical penalty."""
    from paper_1603_03755_gb300.scan import penalty_scan
    sp = stream.cuda_stream
    pens = [1, 2, 3, 4, 6, 8, 10, 12]
    J = W.random_instances(8, 32, 5)
    out = {}
    for emb in ("me", "lhz"):
        for kind in ("sqa", "pt"):
            anneal = (dict(L=64, beta=1.0) if kind == "sqa"
                      else dict(betas=W.paper_beta_ladder(32, 20.0, 0.1), swap_every=1))
            t0 = time.perf_counter()
            res = penalty_scan(embedding=emb, N=8, J=J, penalties=pens, R=256, sweeps=args.scan_sweeps, seed=5,
                               kind=kind, stream=sp, **anneal)
            dt = time.perf_counter() - t0
            best = res.success.max(axis=0)
            out[f"{kind}_{emb}"] = {
                "sweeps": args.scan_sweeps, "penalties": pens, "seconds_end_to_end": dt,
                "attempts_per_s_end_to_end": res.attempts / dt,
                "mean_success_at_optimal": float(best.mean()),
                "mean_optimal_penalty": float(res.optimal.mean()),
                "mean_critical_penalty": (float(np.nanmean(res.critical)) if np.isfinite(res.critical).any()
                                          else None),
                "instances_reaching_half": int(np.isfinite(res.critical).sum())}
    return out


def pt_workloads(pkg, stream, args, embs):
    """PT on ME K_32 / LHZ K_24: 32 temperatures, swap every sweep, R = 32."""
    sp = stream.cuda_stream
    out = {}
    for emb in embs:
        c = W.pt_config(emb, n_inst=args.pt_instances, sweeps=args.pt_sweeps)
        kw = dict(embedding=emb, N=c["N"], J=c["J"], penalty=c["penalty"], R=c["R"], seed=c["seed"], kind="pt",
                  betas=c["betas"], swap_every=c["swap_every"])
        w = pkg.Handle(sweeps=50, **kw)
        w.run(stream=sp)
        stream.synchronize()
        w.close()
        h = pkg.Handle(sweeps=args.pt_sweeps, **kw)
        att = h.info["attempts_per_sweep"] * args.pt_sweeps
        t = timed(stream, lambda: h.run(stream=sp))
        out[f"pt_{emb}"] = {"workload": c["name"] + f", 32 temperatures, {args.pt_sweeps} sweeps, swap every sweep",
                            "value": att / t, "unit": UNIT, "seconds": t, "launch": h.launch()}
        h.close()
    return out


def job_attempts(j) -> int:
    n = j["N"] * (math.ceil(j["N"] / 4) + 1) if j["embedding"] == "me" else j["N"] * (j["N"] - 1) // 2
    Z = j["L"] if j["kind"] == "sqa" else len(j["betas"])
    return n * Z * j["R"] * j["sweeps"]


def _job_kw(j):
    kw = {k: j[k] for k in ("embedding", "N", "J", "penalty", "sweeps", "R", "seed", "kind")}
    if j["kind"] == "sqa":
        kw.update(L=j["L"], beta=j["beta"])
    else:
        kw.update(betas=j["betas"], swap_every=j["swap_every"])
    return kw


def serving_saturation(pkg, n_jobs=200, seed=0):
    """The server's capacity on the serving job stream: every job submitted
    at once (all resident if memory allows), capacity = the stream's
    attempts / makespan."""
    jobs = W.serving_stream(n_jobs, seed)
    att = np.array([job_attempts(j) for j in jobs], float)
    srv = pkg.Server(64 << 30)
    ids = [srv.submit(**_job_kw(j)) for j in jobs]
    for jid in ids:
        srv.wait(jid, timeout=900)
    infos = [srv.poll(jid) for jid in ids]
    st = srv.stats()
    srv.close()
    t_first = min(i["t_submit"] for i in infos)
    span = max(i["t_done"] for i in infos) - t_first
    done = np.array([i["state"] == "done" for i in infos])
    ends = np.array([i["t_done"] - t_first for i in infos])
    return {"jobs": n_jobs, "jobs_done": int(done.sum()), "attempts": float(att.sum()),
            "attempts_per_s": float(att[done].sum() / span), "makespan_s": span,
            "p50_done_s": float(np.percentile(ends, 50)), "p99_done_s": float(np.percentile(ends, 99)),
            "max_resident_jobs": st["max_resident"], "chunks": st["chunks"]}


def serving_suite(pkg, args):
    """Saturated capacity first, then Poisson streams at 50 / 80 / 95 % of it
    (or of --serving-capacity)."""
    sat = serving_saturation(pkg, args.serving_jobs)
    cap = args.serving_capacity if args.serving_capacity > 0 else sat["attempts_per_s"]
    loads = [serving_workload(pkg, cap, load, args.serving_jobs) for load in (0.5, 0.8, 0.95)]
    return {"serving_capacity": dict(sat, basis="measured saturation" if args.serving_capacity <= 0
                                     else "--serving-capacity"),
            "serving": loads}


def serving_workload(pkg, capacity, load, n_jobs=200, seed=0):
    """Poisson stream of SQA/PT jobs (ME or LHZ, N 6-40, L 16-128, sweeps
    log-uniform 1e3-1e5, 1-256 replicas) at `load` x capacity attempts/s,
    served with continuous batching under a 64 GiB budget.  Latency is
    submit-to-done on the server's clock."""
    jobs = W.serving_stream(n_jobs, seed)
    att = np.array([job_attempts(j) for j in jobs], float)
    rate = load * capacity / att.mean()                 # jobs per second
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, n_jobs)
    srv = pkg.Server(64 << 30)
    ids, kws = [], []
    t0 = time.perf_counter()
    t_next = 0.0
    for j, gap in zip(jobs, gaps):
        t_next += gap
        delay = t0 + t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        kw = _job_kw(j)
        ids.append(srv.submit(**kw))
        kws.append(kw)
    infos = []
    for jid in ids:
        srv.wait(jid, timeout=900)
        infos.append(srv.poll(jid))
    st = srv.stats()
    # the three cheapest jobs again, each alone through sqa_run: same bits
    alone_equal = []
    for k in np.argsort(att)[:3]:
        if infos[k]["state"] != "done":
            continue
        got, _ = srv.result(ids[k])
        h = pkg.Handle(**kws[k])
        h.run(stream=0)
        alone_equal.append(bool(np.array_equal(got, h.state(stream=0))))
        h.close()
    srv.close()
    lat = np.array([i["t_done"] - i["t_submit"] for i in infos])
    qwait = np.array([i["t_start"] - i["t_submit"] for i in infos])
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    done = [i["state"] == "done" for i in infos]
    return {"offered_load": load, "offered_attempts_per_s": load * capacity, "jobs": n_jobs,
            "jobs_done": int(sum(done)), "arrival_rate_per_s": rate, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "p50_queue_s": float(np.percentile(qwait, 50)),
            "attempts_per_s": float(att[np.array(done)].sum() / span), "makespan_s": span,
            "chunks": st["chunks"], "max_resident_jobs": st["max_resident"],
            "worker_s": {"admit": st["admit_s"], "advance": st["advance_s"], "idle": st["idle_s"]},
            "failed_status": sorted({int(i["status"]) for i in infos if i["state"] != "done"}),
            "alone_vs_served_same_bits": alone_equal}


def run_reference(args, cfg, world, rank, dist):
    """Reference arm: the CPU oracle, as it stands, on every host core (one
    thread per core, each annealing its own instance; the oracle's C calls
    release the GIL), a bounded sample of the workload per step."""
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor
    import oracle as O
    N, L, pen, beta, S = cfg["N"], cfg["L"], cfg["penalty"], cfg["beta"], cfg["sweeps"]
    A, B = O.linear_schedule(S)
    R, sweeps_per_step = 32, 300
    n = os.cpu_count() or 1
    n_inst = cfg["J"].shape[0]

    def anneal(inst):
        pb = O.Problem("me", N, cfg["J"][inst], pen)
        q = O.SQA(pb, L, R, beta, A, B, cfg["seed"], inst)
        q.run(0, sweeps_per_step)
        return int(pb.used.sum()) * L * R * sweeps_per_step

    times, total = [], 0
    with ThreadPoolExecutor(n) as ex:
        for k in range(args.warmup + args.steps):
            insts = [(k * n + j) % n_inst for j in range(n)]
            t0 = time.perf_counter()
            attempts = sum(ex.map(anneal, insts))
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                times.append(dt)
                total += attempts
    value = total / sum(times)
    sample = (f"per step: {n} instances of the workload, one per host thread, replicas 0-31 of each, "
              f"sweeps 0-{sweeps_per_step - 1} of the {S}-sweep anneal")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "instances": int(cfg["J"].shape[0]), "replicas": cfg["R"],
                   "slices": L, "sweeps": S, "parallelism": "replicas"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    world, rank, local, dist = dist_setup()
    cfg = W.me_n8_batch_config(n_inst=args.instances, sweeps=args.sweeps)
    if args.impl == "reference":
        run_reference(args, cfg, world, rank, dist)
        return

    import torch
    import oracle as O  # noqa: F401  (only the cpu_baseline leg calls it)
    import paper_1603_03755_gb300 as pkg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    if args.pt_only:
        res = pt_workloads(pkg, stream, args, (args.pt_only,))
        if rank == 0:
            print(json.dumps({"pt_only": res}))
        return
    if args.serving_only:
        res = serving_suite(pkg, args)
        if rank == 0:
            print(json.dumps({"serving_only": res}))
        return
    if args.wolff_only:
        res = wolff_workload(pkg, stream, args)
        if rank == 0:
            print(json.dumps({"wolff_only": res}))
        return
    N, R, L, S, I = cfg["N"], cfg["R"], cfg["L"], cfg["sweeps"], cfg["J"].shape[0]
    h = pkg.Handle(embedding="me", N=N, J=cfg["J"], penalty=cfg["penalty"], sweeps=S, R=R,
                   seed=cfg["seed"], L=L, beta=cfg["beta"])
    attempts = h.info["attempts_per_sweep"] * S
    tuned = (h.autotune(n_trial=20, stream=sp) if not args.no_autotune  # launch shape by measurement
             else {"trial_attempts_per_s": None})
    e_ground = pkg.ground_energy(N, cfg["J"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    E_dev = torch.empty((I, L, R), dtype=torch.int32, device=dev)
    ro_dev = torch.empty((I, h.info["n_phys"], h.info["words"]), dtype=torch.uint32, device=dev)
    log_dev = torch.empty((I, R, N), dtype=torch.int8, device=dev)
    en_dev = torch.empty((I, R), dtype=torch.int64, device=dev)
    succ_dev = torch.empty((I,), dtype=torch.int32, device=dev)
    L_ = pkg.lib()
    import ctypes as C

    def device_step():
        h.run(stream=sp)                                            # init + sweeps
        L_.sqa_energies(h.handle, E_dev.data_ptr(), 1, sp)         # energies
        L_.sqa_readout(h.handle, ro_dev.data_ptr(), 1, sp)         # readout
        st = L_.sqa_decode(h.handle, 0, 0, log_dev.data_ptr(), en_dev.data_ptr(),
                           C.c_void_p(e_ground.ctypes.data), succ_dev.data_ptr(), 1, sp)
        assert st == 0

    launches_per_step = h.info["launches_per_run"] + 3  # + energy, readout, decode kernels

    # the dominant kernel's own duration, on the stream it runs on
    def timed_sweeps():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            h.run(stream=sp)
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / 1e3

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        device_step()
    stream.synchronize()

    clocks = Clocks(local)
    clocks.start()
    times = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        barrier(dist)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        device_step()
        e1.record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        barrier(dist)
        times.append(e0.elapsed_time(e1) / 1e3)
    sweep_times = [timed_sweeps() for _ in range(2)]
    clk = clocks.stop()
    t_step = max_over_ranks(dist, statistics.mean(times))
    value = world * attempts / t_step
    # correctness of what was timed: success counts vs a host recount
    succ = succ_dev.cpu().numpy()
    en = en_dev.cpu().numpy()
    assert np.array_equal(succ, (en == e_ground[:, None]).sum(axis=1))

    # end to end through the public API with host buffers
    e2e_times = []
    for k in range(max(2, min(args.steps, 3))):
        barrier(dist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh = pkg.Handle(embedding="me", N=N, J=cfg["J"], penalty=cfg["penalty"], sweeps=S, R=R,
                        seed=cfg["seed"], L=L, beta=cfg["beta"])
        hh.run(stream=sp)
        logical, energy, succ_h = hh.decode("me_mv", 0, e_ground=e_ground, stream=sp)
        dt = time.perf_counter() - t0
        h2d = hh.info["h2d_bytes"]
        hh.close()
        e2e_times.append(max_over_ranks(dist, dt))
    d2h = logical.nbytes + energy.nbytes + succ_h.nbytes
    e2e_value = world * attempts / statistics.mean(e2e_times)

    # the plain one-launch-per-instance path on a sample of instances
    ns = max(1, min(args.per_instance_sample, I))
    hp = pkg.Handle(embedding="me", N=N, J=cfg["J"][:ns], penalty=cfg["penalty"], sweeps=S, R=R,
                    seed=cfg["seed"], L=L, beta=cfg["beta"])
    hp.run_per_instance(stream=sp)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hp.run_per_instance(stream=sp)
    e1.record(stream)
    stream.synchronize()
    per_inst_rate = hp.info["attempts_per_sweep"] * S / (e0.elapsed_time(e1) / 1e3)
    same = np.array_equal(hp.state(stream=sp), h.state(stream=sp)[:ns])
    hp.close()

    if rank != 0:
        barrier(dist)
        return
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    f_mhz = (clk or {}).get("sm_mhz") or 1462.0
    peaks, src = load_peaks()
    peak_gops = n_sm * 4 * 32 * f_mhz * 1e6 / 1e9
    intpeak = {k: round(pkg.int_peak(k), 2) for k in pkg.INT_PEAK_KINDS}
    t_sweep = statistics.mean(sweep_times)
    achieved_gops = attempts * OPS_PER_ATTEMPT / t_sweep / 1e9
    traffic, traffic_note, counters = kernel_capture(I)
    extra = None if args.no_extra else extra_workloads(pkg, stream, args)
    cpu = None
    if not args.no_cpu_baseline:
        rate1, desc1, _ = cpu_oracle_sample(cfg, 5.0)
        rate, cores, desc = cpu_oracle_all_cores(cfg, 10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "single_thread": {"value": rate1, "sample": desc1}}
    mixed = intpeak["lop3_imad"]                         # lane-ops / SM clock, ALU and FMA pipes interleaved
    mixed_gops = n_sm * f_mhz * 1e6 * mixed / 1e9
    ipa = (counters or {}).get("instr_per_attempt")
    per_inst = {"value": per_inst_rate, "unit": UNIT, "instances_sampled": ns,
                "same_bits_as_batched": bool(same), "batched_over_per_instance": value / world / per_inst_rate}
    rates = None
    if extra:
        rates = {k: extra[k]["value"] for k in ("ragged_mix", "pt_me", "pt_lhz") if k in extra}
        if "wolff_me" in extra:
            rates["wolff_me_spin_slice_updates"] = extra["wolff_me"]["value"]
        if "serving_capacity" in extra:
            rates["serving_capacity"] = extra["serving_capacity"]["attempts_per_s"]
        rates["unit"] = UNIT
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": cfg["name"], "embedding": "me_chimera_2x2", "N": N, "instances": I,
                   "replicas": R, "slices": L, "sweeps": S, "parallelism": "replicas",
                   "l2": "flushed between steps (256 MiB write)"},
        "per_instance_path": per_inst,
        "workload_rates": rates,
        "roofline": {"bound": "alu", "achieved": achieved_gops, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved_gops / peak_gops, "traffic": traffic, "traffic_note": traffic_note,
                     "kernel": "sweep_kernel", "ops_per_attempt": OPS_PER_ATTEMPT,
                     "peak_basis": f"{n_sm} SMs x 4 SMSP x 32 lanes x {f_mhz:.0f} MHz (median SM clock under load)",
                     "instr_per_attempt": ipa,
                     "issue_active": (counters or {}).get("issue_active"),
                     "pipes": None if not counters else {"alu": counters.get("pipe_alu"),
                                                         "fma": counters.get("pipe_fma")},
                     "counters_source": "ncu capture of the sweep kernel (profiles/sweep_kernel_traffic.json)"
                                        if counters else traffic_note,
                     "mixed_pipe_ceiling": {
                         "lane_ops_per_sm_clk": mixed, "gops": mixed_gops,
                         "frac": achieved_gops / mixed_gops,
                         "attempts_per_s_at_kernel_instr": (n_sm * f_mhz * 1e6 * mixed / ipa) if ipa else None,
                         "basis": "measured LOP3/IMAD interleaved issue rate x SMs x median SM clock"},
                     "sweep_kernel_s": t_sweep,
                     "measured_lane_ops_per_sm_clk": intpeak},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "cpu_baseline": cpu,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "latency": None if not extra or "serving" not in extra else dict(
            {f"load_{int(100 * x['offered_load'])}pct": {"p50_s": x["p50_latency_s"], "p99_s": x["p99_latency_s"]}
             for x in extra["serving"]},
            loads_relative_to={"attempts_per_s": extra["serving_capacity"]["attempts_per_s"],
                               "basis": extra["serving_capacity"]["basis"]}),
        "launch": dict(h.launch(), autotune_trial_attempts_per_s=tuned["trial_attempts_per_s"]),
        "peaks_source": src,
        "other_workloads": extra,
    }
    print(json.dumps(out))
    barrier(dist)


if __name__ == "__main__":
    main()
