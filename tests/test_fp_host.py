"""The integer-pipe FP64 helpers of the CUDA library (pdg_fp.cuh), compiled for
the host, against IEEE arithmetic: the reciprocal fl(1/w) of step A1 (Eq. RT's
resistive weights) and the conversion fl(x 2^-S) of an exact fixed-point path
sum of step A3 (Eq. RT).  Python's float division and int-to-float conversion
are correctly rounded to nearest-even, so they are the reference."""
import ctypes
import math
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _dbl(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b))[0]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("fp") / "fp_host_check.so")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                           os.path.join(ROOT, "paper_2508_20403_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "fp_host_check.cc"), "-o", out])
    return ctypes.CDLL(out)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def test_reciprocal_matches_ieee_division(lib):
    rng = np.random.default_rng(20250831)
    n = 200_000
    e = rng.integers(1023 - 900, 1023 + 900, size=n, dtype=np.uint64)
    f = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    special = np.array([0, 1, 2, 3, (1 << 52) - 1, (1 << 52) - 2, 1 << 51, (1 << 51) + 1, (1 << 51) - 1,
                        0x5555555555555, 0xAAAAAAAAAAAAA, 0x8000000000001], dtype=np.uint64)
    f[: special.size * 50] = np.tile(special, 50)
    w = (e << np.uint64(52)) | f
    out = np.zeros(n, dtype=np.uint64)
    ok = np.zeros(n, dtype=np.int32)
    lib.pdg_host_rcp_bits(_p(w), _p(out), _p(ok), ctypes.c_int64(n))
    assert ok.all()
    bad = [i for i in range(n) if int(out[i]) != _bits(1.0 / _dbl(int(w[i])))]
    assert not bad, f"{len(bad)} reciprocals differ, first w={_dbl(int(w[bad[0]])).hex()}"


def test_fixed_point_conversion_matches_exact_rounding(lib):
    import random

    rng = random.Random(97)
    n = 200_000
    xs, S = [], []
    for i in range(n):
        top = rng.randint(1, 114)  # bit length (path sums stay below 2^97; the helper is exact below 2^115)
        x = rng.getrandbits(top) | (1 << (top - 1))
        if i % 3 == 0 and top > 53:  # ties and near-ties of the rounding
            sh = top - 53
            half = 1 << (sh - 1)
            x = ((x >> sh) << sh) | rng.choice([half, half - 1, half + 1, (1 << sh) - 1, 0])
        xs.append(x)
        S.append(rng.randint(-20, 180))
    hi = np.array([x >> 64 for x in xs], dtype=np.uint64)
    lo = np.array([x & ((1 << 64) - 1) for x in xs], dtype=np.uint64)
    Sa = np.array(S, dtype=np.int32)
    out = np.zeros(n, dtype=np.uint64)
    lib.pdg_host_fixed_bits(_p(hi), _p(lo), _p(Sa), _p(out), ctypes.c_int64(n))
    bad = [i for i in range(n) if int(out[i]) != _bits(math.ldexp(float(xs[i]), -S[i]))]
    assert not bad, f"{len(bad)} conversions differ, first x={xs[bad[0]]} S={S[bad[0]]}"
