"""Selection logic of the autotuner (csrc/tune.cpp, compiled here with g++):
the fastest candidate by the median of its measurements, ties to the lower
index, candidates that cannot run skipped, one decision per size bucket and
kind (a second query measures nothing), buckets a factor sqrt(2) apart."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1902_01818_gb300", "csrc")
OUT = os.path.join(HERE, "_build")
_D = C.POINTER(C.c_double)


@pytest.fixture(scope="module")
def tn():
    os.makedirs(OUT, exist_ok=True)
    so = os.path.join(OUT, "libtune.so")
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CSRC, os.path.join(CSRC, "tune.cpp"),
                    os.path.join(HERE, "tune_shim.cpp"), "-o", so], check=True)
    lib = C.CDLL(so)
    lib.tn_choose.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _D, C.POINTER(C.c_int)]
    lib.tn_bucket.argtypes = [C.c_longlong]
    return lib


def _choose(tn, kind, bucket, times):
    t = np.ascontiguousarray(times, dtype=np.float64)
    calls = C.c_int()
    c = tn.tn_choose(kind, bucket, t.shape[0], t.shape[1], t.ctypes.data_as(_D), C.byref(calls))
    return c, calls.value


def test_fastest_median_wins_and_is_remembered(tn):
    tn.tn_clear()
    # candidate 1 has one slow outlier but the smallest median
    times = [[3.0, 3.1, 2.9], [1.0, 9.0, 1.1], [2.0, 2.0, 2.0]]
    c, calls = _choose(tn, 0, 20, times)
    assert c == 1 and calls == 9
    c, calls = _choose(tn, 0, 20, [[0.1, 0.1, 0.1], [5.0, 5.0, 5.0], [5.0, 5.0, 5.0]])
    assert c == 1 and calls == 0  # cached: no measurement
    c, calls = _choose(tn, 1, 20, [[0.1, 0.1, 0.1], [5.0, 5.0, 5.0], [5.0, 5.0, 5.0]])
    assert c == 0 and calls == 9  # another kind, its own decision
    assert tn.tn_size() == 2


def test_ties_and_candidates_that_cannot_run(tn):
    tn.tn_clear()
    c, _ = _choose(tn, 0, 7, [[2.0, 2.0], [2.0, 2.0]])
    assert c == 0
    c, calls = _choose(tn, 0, 8, [[-1.0, 0.0], [4.0, 4.0], [3.0, 3.0]])
    assert c == 2 and calls == 5  # candidate 0 stops after its first (negative) measurement
    # nothing runs: candidate 0, not remembered
    c, _ = _choose(tn, 0, 9, [[-1.0], [-1.0]])
    assert c == 0 and tn.tn_size() == 2


def test_buckets(tn):
    assert tn.tn_bucket(1) == 0 and tn.tn_bucket(2) == 2 and tn.tn_bucket(3) == 3 and tn.tn_bucket(4) == 4
    # a factor sqrt(2) apart
    for n in (100, 1000, 123456):
        assert tn.tn_bucket(int(n * 1.5)) == tn.tn_bucket(n) + 1 or tn.tn_bucket(int(n * 1.5)) == tn.tn_bucket(n) + 2
    assert tn.tn_bucket(0) == 0
