"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the C oracle (a dropped factor, a
flipped sign, a wrong index or member, a wrong constant), builds the copy,
and runs the oracle's pin tests (test_oracle_*.py) against it in a separate
process: they must fail.  An unmutated copy must pass, so a failure is the
mistake's doing and not the harness's.  Everything runs on the CPU.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_TESTS = ["test_oracle_rng.py", "test_oracle_embedding.py", "test_oracle_tables.py",
             "test_oracle_decode.py", "test_oracle_statistics.py", "test_oracle_wolff.py"]

# (name, file, original text, planted mistake)
MUTANTS = [
    ("philox multiplier", "philox.c", "(uint64_t)0xD2511F53u * c[0]", "(uint64_t)0xD2511F55u * c[0]"),
    ("philox key bump", "philox.c", "k[0] += 0x9E3779B9u;", "k[0] += 0x9E3779BBu;"),
    ("ME chain coupler sign", "embed.c",
     "int32_t mem[2] = {orc_me_site(Lc, g, g, 0, m), orc_me_site(Lc, g, g, 1, m)};\n"
     "            put_term(t++, 2, mem, -penalty,",
     "int32_t mem[2] = {orc_me_site(Lc, g, g, 0, m), orc_me_site(Lc, g, g, 1, m)};\n"
     "            put_term(t++, 2, mem, penalty,"),
    ("ME logical edge on the wrong shore", "embed.c",
     "mem[0] = orc_me_site(Lc, gi, gj, 1, mi);", "mem[0] = orc_me_site(Lc, gi, gj, 0, mi);"),
    ("ME colouring ignores the cell parity", "embed.c",
     "colour[s] = u ^ ((r + c) & 1);", "colour[s] = u;"),
    ("LHZ colouring with three colours", "embed.c",
     "colour[k] = 2 * (i & 1) + (j & 1);", "colour[k] = (i & 1) + (j & 1);"),
    ("LHZ 4-body plaquette member", "embed.c",
     "pair_index(N, i + 1, j), pair_index(N, i + 1, j + 1)};",
     "pair_index(N, i + 1, j), pair_index(N, i, j + 1)};"),
    ("LHZ constraint sign", "embed.c", "put_term(t++, 4, mem, -lambda,", "put_term(t++, 4, mem, lambda,"),
    ("flip energy sign", "embed.c", "return -2 * before;", "return 2 * before;"),
    ("Jperp sign", "anneal.c", "return -0.5 * log(tanh(a));", "return 0.5 * log(tanh(a));"),
    ("alpha without 1/L in the sweep", "anneal.c",
     "double alpha = prm->beta * prm->B[t] / (double)L;\n        double jp",
     "double alpha = prm->beta * prm->B[t];\n        double jp"),
    ("alpha without 1/L in the cluster move", "anneal.c",
     "double alpha = prm->beta * prm->B[t] / (double)L;\n        uint32_t Tb",
     "double alpha = prm->beta * prm->B[t];\n        uint32_t Tb"),
    ("temporal term without its factor 2", "anneal.c",
     "xt = 2.0 * jperp * (double)m;", "xt = jperp * (double)m;"),
    ("open instead of periodic imaginary time", "anneal.c",
     "int32_t up = (tau + L - 1) % L, dn = (tau + 1) % L;",
     "int32_t up = tau > 0 ? tau - 1 : tau, dn = tau + 1 < L ? tau + 1 : tau;"),
    ("threshold scaled by 2^31", "anneal.c", "floor(ldexp(exp(-x), 32))", "floor(ldexp(exp(-x), 31))"),
    ("PT swap exponent sign", "anneal.c", "double dbeta = beta_p - beta_q;", "double dbeta = beta_q - beta_p;"),
    ("PT slot temperature reversed", "anneal.c",
     "double x = prm->betas[p] * (double)delta;", "double x = prm->betas[P - 1 - p] * (double)delta;"),
    ("PT swaps only the even pairs", "anneal.c",
     "for (int32_t p = e & 1; p + 1 < P; p += 2)", "for (int32_t p = 0; p + 1 < P; p += 2)"),
    ("SQA sweep skips the odd slices", "anneal.c",
     "for (int32_t tau = parity; tau < L; tau += 2)", "for (int32_t tau = 0; tau < L; tau += 2)"),
    ("ME chain loses a vertical coupler", "embed.c",
     "for (int32_t r = 0; r < g; r++) {\n            int32_t mem[2]",
     "for (int32_t r = 0; r + 1 < g; r++) {\n            int32_t mem[2]"),
    ("cluster bond probability e^(-2 Jperp)", "anneal.c",
     "double v = floor(ldexp(1.0 - tanh(a), 32));", "double v = floor(ldexp(tanh(a), 32));"),
    ("cluster grows forward only", "anneal.c",
     "while (back < L - 1 - fwd && ORC_JOINS(", "while (0 && ORC_JOINS("),
    ("cluster bonds ignore spin equality", "anneal.c",
     "(*at(s, n, R, (tau), site, rho) == *at(s, n, R, ((tau) + 1) % L, site, rho) &&",
     "(1 &&"),
    ("cluster energy taken from its start slice only", "anneal.c",
     "D += orc_flip_delta(pb, s + (int64_t)tau * n * R, R, rho, site);",
     "D += orc_flip_delta(pb, s + (int64_t)tau0 * n * R, R, rho, site);"),
    ("ME majority-vote tie rule", "decode.c", "logical[i] = phys[hub[i]];", "logical[i] = 1;"),
    ("LHZ tree vote tie rule", "decode.c", "(sum < 0 ? -1 : tmp[i])", "(sum < 0 ? -1 : 1)"),
    ("minimum-weight decoding keeps the last of equally near states", "decode.c",
     "if (!have || score > best) {\n            best = score;\n            have = 1;\n            for (int32_t i = 0; i < N; i++) logical[i] = q[i];",
     "if (!have || score >= best) {\n            best = score;\n            have = 1;\n            for (int32_t i = 0; i < N; i++) logical[i] = q[i];"),
    ("minimum-weight decoding maximises disagreement", "decode.c",
     "score += (int64_t)phys[orc_lhz_index(N, i, j)] * q[i] * q[j];",
     "score -= (int64_t)phys[orc_lhz_index(N, i, j)] * q[i] * q[j];"),
    ("BP ties take +1", "decode.c", "q[i * N + j] = d > 0.0 ? 1 : (d < 0.0 ? -1 : p[i * N + j]);",
     "q[i * N + j] = d >= 0.0 ? 1 : -1;"),
    ("BP check weight without its factor 2", "decode.c",
     "const double L2 = log(((1.0 - e) * (1.0 - e) + e * e) / (2.0 * e * (1.0 - e)));",
     "const double L2 = log(((1.0 - e) * (1.0 - e) + e * e) / (e * (1.0 - e)));"),
    ("BP checks through the pair itself", "decode.c",
     "if (l != i && l != j) S += p[i * N + l] * p[l * N + j];",
     "if (l != i) S += p[i * N + l] * p[l * N + j];"),
    ("ground-state enumeration half short", "decode.c",
     "int have = 0;\n    uint64_t count = (uint64_t)1 << (N - 1);\n    for (uint64_t x = 0; x < count; x++) {\n        for (int32_t i = 0; i < N - 1; i++) s[i]",
     "int have = 0;\n    uint64_t count = (uint64_t)1 << (N - 2);\n    for (uint64_t x = 0; x < count; x++) {\n        for (int32_t i = 0; i < N - 1; i++) s[i]"),
]


def _run_pins(tmp):
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([tmp, ROOT]))
    args = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--rootdir", ROOT,
            "-c", os.path.join(ROOT, "pytest.ini")] + [os.path.join(ROOT, "tests", f) for f in PIN_TESTS]
    r = subprocess.run(args, cwd=tmp, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def _copy_oracle(tmp):
    dst = os.path.join(tmp, "oracle")
    os.makedirs(dst)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h", ".py")):
            shutil.copy(os.path.join(ROOT, "oracle", f), dst)
    return dst


def _case(m):
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        dst = _copy_oracle(tmp)
        if m is not None:
            _, fname, old, new = m
            p = os.path.join(dst, fname)
            src = open(p).read()
            if src.count(old) != 1:
                return "text", f"expected one occurrence of the mutated text in {fname}"
            open(p, "w").write(src.replace(old, new))
        rc, out = _run_pins(tmp)
        return rc, out
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


@pytest.fixture(scope="module")
def results():
    cases = [None] + MUTANTS
    with ThreadPoolExecutor(max(2, min(len(cases), os.cpu_count() or 2))) as ex:
        out = list(ex.map(_case, cases))
    return dict(zip(["unmutated"] + [m[0] for m in MUTANTS], out))


def test_unmutated_copy_passes_the_pins(results):
    rc, out = results["unmutated"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(results, name):
    rc, out = results[name]
    assert rc != "text", out
    assert rc != 0, f"no pin caught the planted mistake '{name}':\n{out}"
