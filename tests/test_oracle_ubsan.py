"""The oracle built with UndefinedBehaviorSanitizer, and with AddressSanitizer (CPU
only): round trips of every format and width, edge lengths and every operator run
without a sanitizer report (undefined shifts, overflow of signed values, reads or
writes outside a buffer)."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, ROOT_DIR)
import numpy as np
import oracle
from paper_2004_09350_gb300 import synth
for n in (0, 1, 15, 511, 512, 513, 1500):
    for b in (0, 1, 7, 31, 32, 33, 63, 64):
        x = (synth.splitmix64(n + b, n) >> np.uint64(64 - b)) if b else np.zeros(n, dtype=np.uint64)
        for f in range(5):
            bw = max(1, int(x.max()).bit_length()) if n else 1
            buf = oracle.compress(f, x, bw=bw if f == 1 else 0)
            assert (oracle.decompress(f, n, buf, bw=bw if f == 1 else 0) == x).all()
x = synth.skewed_widths(3, 3000)
k = synth.sorted_gaps(4, 3000)
for cmp in range(7):
    p = oracle.select(x, cmp, 17, 1 << 20)
    oracle.agg_sum(oracle.project(k, p))
for op in range(3):
    oracle.calc(op, x, k)
    oracle.calc(op, x, None, 2**64 - 3)
oracle.group_sum(x % np.uint64(7), k, 7)
oracle.semijoin(x % np.uint64(1000), np.arange(0, 1000, 3, dtype=np.uint64), 1000)
print("clean")
'''.replace("ROOT_DIR", repr(ROOT))


def test_oracle_under_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    lib = str(tmp_path / "liboracle_ubsan.so")
    r = subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-shared", "-fPIC", "-fsanitize=undefined",
                        "-fno-sanitize-recover=undefined", "-o", lib, os.path.join(ROOT, "oracle", "oracle.c")],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no UBSan runtime: " + r.stderr[-300:])
    env = dict(os.environ, ORACLE_LIB=lib, UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0 and "clean" in r.stdout, r.stderr[-3000:]
    assert "runtime error" not in r.stderr, r.stderr[-3000:]


def test_oracle_under_asan(tmp_path):
    """Out-of-bounds reads and writes of the oracle's buffers (heap and stack)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    runtime = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not runtime or not os.path.exists(runtime):
        pytest.skip("no ASan runtime")
    lib = str(tmp_path / "liboracle_asan.so")
    r = subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-shared", "-fPIC", "-fsanitize=address",
                        "-fno-omit-frame-pointer", "-o", lib, os.path.join(ROOT, "oracle", "oracle.c")],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("ASan build failed: " + r.stderr[-300:])
    env = dict(os.environ, ORACLE_LIB=lib, LD_PRELOAD=os.path.realpath(runtime),
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0 and "ERROR: AddressSanitizer" not in r.stderr and "clean" not in r.stdout:
        pytest.skip("the interpreter does not start under the ASan runtime: " + r.stderr[-300:])
    assert r.returncode == 0 and "clean" in r.stdout, r.stderr[-3000:]
    assert "AddressSanitizer" not in r.stderr, r.stderr[-3000:]
