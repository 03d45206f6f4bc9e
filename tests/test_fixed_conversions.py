"""The integer-pipe binary64 <-> int64 conversions of the fixed-point
defect correction (paper_1201_3185_gb300/csrc/fixed_conv.h), built for the
host with g++ and checked against correctly rounded references: numpy's rint
(round half to even) and Python's int -> float conversion (correctly
rounded, ties to even), scaled by exact powers of two.  Ties, signs, zero,
subnormals and every magnitude from 2^-3 to 2^62 are covered."""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1201_3185_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "fixed_conv.h"
int main(int argc, char** argv)
{
    FILE* f = fopen(argv[1], "rb");
    long long nd = 0, ni = 0;
    fread(&nd, 8, 1, f);
    std::vector<double> xd(nd);
    fread(xd.data(), 8, nd, f);
    fread(&ni, 8, 1, f);
    std::vector<long long> xi(ni);
    std::vector<int> ei(ni);
    fread(xi.data(), 8, ni, f);
    fread(ei.data(), 4, ni, f);
    fclose(f);
    FILE* g = fopen(argv[2], "wb");
    for (long long q = 0; q < nd; ++q) {
        const long long r = qumond::f64_to_i64_rn(xd[q]);
        fwrite(&r, 8, 1, g);
    }
    for (long long q = 0; q < ni; ++q) {
        const double r = qumond::i64_to_f64_rn_scaled(xi[q], ei[q]);
        fwrite(&r, 8, 1, g);
    }
    fclose(g);
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "drv.cpp")
    open(src, "w").write(DRIVER)
    exe = os.path.join(d, "drv")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, src, "-o", exe], check=True)
    yield exe, d
    shutil.rmtree(d, ignore_errors=True)


def _inputs(rng):
    # doubles: random magnitudes 2^-3 .. 2^62, exact ties k + 1/2, integers, signs, zero, subnormals
    mags = np.ldexp(rng.random(200000) + 0.5, rng.integers(-3, 62, 200000))
    d = mags * rng.choice([-1.0, 1.0], mags.size)
    k = rng.integers(-(1 << 51), 1 << 51, 50000).astype(np.float64)
    ties = np.concatenate([k + 0.5, np.arange(-20, 21) + 0.5, np.array([0.5, -0.5, 1.5, -1.5, 2.5, -2.5])])
    ints = rng.integers(-(1 << 61), 1 << 61, 20000).astype(np.float64)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 0.49999999999999994, 0.5000000000000001, 2.0 ** 62 - 1024,
                        -(2.0 ** 62 - 1024)])
    xd = np.concatenate([d, ties, ints, special])
    # int64: every bit length 1 .. 62, halfway cases beyond 53 bits, signs; scales e in [-100, 40]
    bits = rng.integers(1, 63, 200000)
    xi = (rng.integers(0, 1 << 62, 200000) >> (62 - bits)) | (np.int64(1) << (bits - 1))
    xi = xi * rng.choice([-1, 1], xi.size)
    half = []
    for b in range(54, 63):
        for _ in range(200):
            m = int(rng.integers(1 << 52, 1 << 53))
            sh = b - 53
            half.append((m << sh) | (1 << (sh - 1)))  # exactly halfway between two representable values
    xi = np.concatenate([xi, np.array(half, dtype=np.int64), -np.array(half, dtype=np.int64),
                         np.array([1, -1, (1 << 62) - 1, -((1 << 62) - 1)], dtype=np.int64)])
    ei = rng.integers(-100, 41, xi.size).astype(np.int32)
    return xd, xi.astype(np.int64), ei


def test_conversions_round_to_nearest_even(driver):
    exe, d = driver
    rng = np.random.default_rng(5)
    xd, xi, ei = _inputs(rng)
    inp = os.path.join(d, "in.bin")
    out = os.path.join(d, "out.bin")
    with open(inp, "wb") as f:
        np.array([xd.size], dtype=np.int64).tofile(f)
        xd.tofile(f)
        np.array([xi.size], dtype=np.int64).tofile(f)
        xi.tofile(f)
        ei.tofile(f)
    subprocess.run([exe, inp, out], check=True)
    raw = np.fromfile(out, dtype=np.uint8)
    got_d = raw[:8 * xd.size].view(np.int64)
    got_i = raw[8 * xd.size:].view(np.float64)
    want_d = np.rint(xd).astype(np.int64)
    assert np.array_equal(got_d, want_d)
    want_i = np.array([math.ldexp(float(int(v)), int(e)) for v, e in zip(xi, ei)])
    assert np.array_equal(got_i.view(np.int64), want_i.view(np.int64))
