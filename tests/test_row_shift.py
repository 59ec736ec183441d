"""The row shift s_i = floor(s + 0.5) of §3.1 in FP32 (csrc/row_shift.cuh), checked on the
host against the exact value floor(s + 0.5) in FP64 (s + 0.5 is exact in FP64 for every
float s): every float in bands around the ties, random floats over all magnitudes, and the
special values.  The header compiles for host and device alike."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_06017_gb300", "csrc")

PROG = r'''
#include <stdio.h>
#include <stdint.h>
#include <string.h>
#include "row_shift.cuh"
int main(void) {
  uint32_t bits;
  while (fread(&bits, 4, 1, stdin) == 1) {
    float s; memcpy(&s, &bits, 4);
    float r = sgb::round_half_up(s);
    fwrite(&r, 4, 1, stdout);
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def rounder(tmp_path_factory):
    d = tmp_path_factory.mktemp("rowshift")
    src = d / "rs.cpp"
    src.write_text(PROG)
    exe = d / "rs"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)

    def run(x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        out = subprocess.run([str(exe)], input=x.tobytes(), capture_output=True, check=True).stdout
        return np.frombuffer(out, dtype=np.float32)
    return run


def exact(x):
    return np.floor(x.astype(np.float64) + 0.5).astype(np.float32)


def test_bands_around_the_ties(rounder):
    ties = np.concatenate([np.arange(-40, 41) + 0.5, [0.0, 1.0, -1.0, 2.0 ** 22 + 0.5, -(2.0 ** 22) - 0.5]])
    xs = []
    for t in ties.astype(np.float32):
        b = np.array([t], dtype=np.float32).view(np.int32)[0]
        xs.append(np.arange(b - 300, b + 301, dtype=np.int64))   # every float within 300 ulps
    x = np.concatenate(xs).astype(np.int32).view(np.float32)
    x = x[np.isfinite(x)]
    assert np.array_equal(rounder(x), exact(x))
    # float32 rounding of s + 0.5 gets the first one wrong; the helper does not
    s = np.float32(0.5 - 2.0 ** -25)
    assert np.floor(s + np.float32(0.5)) == 1.0 and rounder(np.array([s]))[0] == 0.0


def test_random_floats_of_every_magnitude(rounder):
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2 ** 32, 400000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    x = bits[np.isfinite(bits)]
    assert np.array_equal(rounder(x), exact(x))


def test_special_values(rounder):
    x = np.array([0.0, -0.0, np.inf, -np.inf, 2.0 ** 23, -(2.0 ** 23) + 0.5, 2.0 ** 22 - 0.5,
                  3.4e38, -3.4e38, 1e-45, -1e-45], dtype=np.float32)
    r = rounder(x)
    assert np.array_equal(r[np.isfinite(x)], exact(x[np.isfinite(x)]))
    assert r[2] == np.inf and r[3] == -np.inf
    assert np.isnan(rounder(np.array([np.nan], dtype=np.float32))[0])
