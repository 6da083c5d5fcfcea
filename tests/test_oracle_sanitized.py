"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer: every entry
point (p-FHT-FSCL in FP64 and int64, FHT-FSCL, Aut-SSC, the FHTL/SPCL node functions, the
transform) runs on codes of every supported shape in a child process with the sanitizer
runtimes preloaded, and any report fails the test. Skipped where gcc has no sanitizer
runtime."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np
import oracle
oracle._LIB_PATH = LIB
oracle.build = lambda force=False: LIB
from paper_2108_12550_gb300 import inputs as I

for m, r, P, L in [(4, 2, 2, 8), (5, 2, 4, 2), (5, 3, 3, 4), (6, 3, 2, 8), (7, 2, 8, 4), (9, 2, 4, 4), (9, 3, 2, 8)]:
    fr = I.make_frames(m, r, 40, 2.5, seed=m * 10 + r)
    tab = I.perm_table(m, r, P, L, seed=L)
    oracle.decode(m, r, P, L, tab, fr["llr"], want_ops=True)
    oracle.decode(m, r, P, L, tab, I.quantize_i8(fr["llr"]).astype(np.int64), integer=True)
    oracle.decode_fhtfscl(m, r, L, fr["llr"])
for m, r in [(5, 1), (7, 2), (9, 3)]:
    fr = I.make_frames(m, r, 20, 3.0, seed=7)
    oracle.aut_ssc(m, r, I.ssc_perm_table(m, 16, seed=3), fr["llr"])
rng = np.random.default_rng(0)
for s in (1, 3, 8):
    for L in (1, 4, 8):
        a = rng.normal(size=(L, 1 << s))
        pm = rng.random(L)
        oracle.fhtl(a, pm)
        if s >= 2:
            oracle.spcl(a, pm)
    oracle.fht(rng.normal(size=1 << s))
print("sanitized oracle ok")
"""


def _runtime(name):
    try:
        path = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True,
                              timeout=30).stdout.strip()
    except (OSError, subprocess.TimeoutExpired):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_runs_clean_under_address_and_undefined_behavior_sanitizers(tmp_path):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("gcc has no sanitizer runtime here")
    lib = str(tmp_path / "librmoracle_sanitized.so")
    src = os.path.join(ROOT, "oracle", "rm_oracle.c")
    subprocess.check_call(["gcc", "-O1", "-g", "-std=gnu11", "-Wall", "-shared", "-fPIC", "-pthread",
                           "-fsanitize=address,undefined", "-fno-omit-frame-pointer",
                           "-fno-sanitize-recover=undefined", src, "-o", lib, "-lm"])
    env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}", ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    code = f"ROOT = {ROOT!r}\nLIB = {lib!r}\n" + CHILD
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    report = res.stderr[-4000:]
    assert res.returncode == 0, report
    assert "runtime error" not in res.stderr and "AddressSanitizer" not in res.stderr, report
    assert "sanitized oracle ok" in res.stdout
