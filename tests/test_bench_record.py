"""The bench line's kernel counters come from a committed ncu capture record
(profiles/sweep_kernel_traffic.json) tied to the code of kernels.cu by a
hash; this checks, on the CPU, that the record is present, complete and
taken on the current code, and that bench.py reads it."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    # bench.py sets a CUDA environment default at import: keep this process's own
    keep = os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS")
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    if keep is None:
        os.environ.pop("CUDA_DEVICE_MAX_CONNECTIONS", None)
    else:
        os.environ["CUDA_DEVICE_MAX_CONNECTIONS"] = keep
    return mod


def test_capture_record_matches_the_kernel_code():
    b = _bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "sweep_kernel_traffic.json")))
    for k in ("dram_bytes_per_instance", "instr_per_attempt", "issue_active", "pipe_alu", "pipe_fma",
              "captured_attempts", "capture_command"):
        assert k in rec, k
    assert "--clock-control none" in rec["capture_command"]
    src = os.path.join(ROOT, "paper_1603_03755_gb300", "csrc", "kernels.cu")
    assert rec["kernels_cu_code_sha256"] == b.kernels_code_sha256(src), \
        "kernels.cu changed since the ncu capture: re-capture the record"
    traffic, note, counters = b.kernel_capture(1024)
    assert traffic is not None and traffic > 0 and counters["instr_per_attempt"] > 10


def test_code_hash_ignores_comments_and_whitespace(tmp_path):
    b = _bench()
    a = tmp_path / "a.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x) { return x + 1; } // one\n/* two */\n")
    c.write_text("int  f(int x)\n{\n    return x + 1;   /* other words */\n}\n")
    assert b.kernels_code_sha256(str(a)) == b.kernels_code_sha256(str(c))
    c.write_text("int f(int x) { return x + 2; }\n")
    assert b.kernels_code_sha256(str(a)) != b.kernels_code_sha256(str(c))
