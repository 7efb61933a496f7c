"""The host side of libtn (order search, tree validation, planning, chain
re-association, UAI parsing) and the C oracle built with the address and
undefined-behaviour sanitizers and run on small inputs of every structure
class: any out-of-bounds access, use after free or undefined operation (and,
for the planner, any leak) fails the test."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2405_14060_gb300", "csrc")
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer",
       "-g", "-O1"]
ENV = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
           UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")


def _gxx():
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    probe = subprocess.run([gxx] + SAN + ["-x", "c++", "-", "-o", os.devnull],
                           input="int main(){return 0;}", capture_output=True, text=True)
    if probe.returncode != 0:
        pytest.skip("the sanitizer runtimes are not installed")
    return gxx


def test_planner_and_model_io_under_sanitizers():
    gxx = _gxx()
    srcs = [os.path.join(CSRC, f) for f in ("plan.cpp", "order_part.cpp", "reassoc.cpp", "model.cpp")]
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "driver")
        cmd = [gxx, "-std=c++17"] + SAN + ["-I", CSRC, "-I", os.path.join(ROOT, "include"),
                                            os.path.join(ROOT, "tests", "host_sanitize_driver.cpp")]
        r = subprocess.run(cmd + srcs + ["-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
        r = subprocess.run([exe, d], capture_output=True, text=True, env=ENV, timeout=600)
        assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
        assert "host sanitizer driver ok" in r.stdout


def test_oracle_under_sanitizers():
    """The oracle's C library, built with the sanitizers, driven through its
    Python binding on small models (brute force, elimination, MAP, MMAP,
    sampling).  Leak detection is off here: the uninstrumented interpreter's
    own allocations at exit would be reported; out-of-bounds accesses, use
    after free and undefined operations in the oracle still fail the run."""
    gxx = _gxx()
    gcc = shutil.which("gcc") or gxx
    src = os.path.join(ROOT, "oracle", "tn_oracle.c")
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "liboracle_san.so")
        r = subprocess.run([gcc, "-shared", "-fPIC"] + SAN + [src, "-o", so, "-lm"],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-3000:]
        code = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, %r)
import oracle
oracle._lib = ctypes.CDLL(%r)
from paper_2405_14060_gb300 import synth
m = synth.random_markov(9, 12, 3, 4, cards=(2, 3, 4))
ev = np.full(m.nvars, -1, np.int32); ev[2] = 1
lz = oracle.brute_pr(m, ev)
assert abs(oracle.ve_pr(m, ev) - lz) < 1e-10
_, mb = oracle.brute_mar(m, ev); _, mv = oracle.ve_mar(m, ev)
assert max(abs(a - b).max() for a, b in zip(mb, mv)) < 1e-10
xb, lb = oracle.brute_map(m, ev); xv, lv = oracle.ve_map(m, ev)
assert abs(lb - lv) < 1e-10
qb, vb = oracle.brute_mmap(m, [0, 5], ev); qv, vv = oracle.ve_mmap(m, [0, 5], ev)
assert abs(vb - vv) < 1e-10
u = np.random.default_rng(0).random(200 * m.nvars)
s = oracle.ve_sample(m, 200, u, ev)
assert (s[:, 2] == 1).all()
bn = synth.bayes_net(40, 3)
assert abs(oracle.ve_pr(bn)) < 1e-9
print("oracle sanitizer run ok")
""" % (ROOT, so)
        env = dict(ENV, LD_PRELOAD=_asan_runtime(gcc), ASAN_OPTIONS="detect_leaks=0")
        r = subprocess.run([os.environ.get("PYTHON", "python3"), "-c", code], capture_output=True,
                           text=True, env=env, timeout=600)
        assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
        assert "oracle sanitizer run ok" in r.stdout


def _asan_runtime(cc):
    """The ASan runtime must be loaded first when an instrumented shared
    library is used from an uninstrumented interpreter."""
    r = subprocess.run([cc, "-print-file-name=libasan.so"], capture_output=True, text=True)
    path = r.stdout.strip()
    if not path or not os.path.isabs(path) or not os.path.exists(path):
        pytest.skip("ASan runtime not found")
    return path
