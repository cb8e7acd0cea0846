"""Pins of the oracle's noise source: its Philox4x32-10 against an independent
implementation (the header-only engine shipped with PyTorch, compiled here with g++),
and the Box-Muller normals against the moments of a standard normal."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import rflbm_oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_ATEN_PROG = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
// reads lines "c0 c1 c2 c3 k0 k1" (hex) and prints the four output words
int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%x %x %x %x %x %x", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    // engine(seed, subsequence, offset): key = seed, counter = (offset, subsequence)
    at::Philox4_32 e((uint64_t(k1) << 32) | k0, (uint64_t(c3) << 32) | c2,
                     (uint64_t(c1) << 32) | c0);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%08x %08x %08x %08x\n", a, b, c, d);
  }
  return 0;
}
"""


def _aten_philox_binary():
    torch = pytest.importorskip("torch")
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch headers not installed")
    out = os.path.join(ROOT, "tests", "_bin")
    os.makedirs(out, exist_ok=True)
    src, exe = os.path.join(out, "aten_philox.cpp"), os.path.join(out, "aten_philox")
    with open(src, "w") as fh:
        fh.write(_ATEN_PROG)
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, src, "-o", exe], check=True)
    return exe


def test_philox_matches_independent_engine():
    exe = _aten_philox_binary()
    g = np.random.default_rng(123)
    cases = [(0, 0, 0, 0, 0, 0), (0xFFFFFFFF,) * 6, (5, 0, 7, 0, 2, 1)]
    cases += [tuple(int(v) for v in g.integers(0, 2 ** 32, 6, dtype=np.uint64))
              for _ in range(200)]
    stdin = "\n".join(" ".join(f"{v:x}" for v in cs) for cs in cases) + "\n"
    res = subprocess.run([exe], input=stdin, capture_output=True, text=True, check=True)
    ref = [[int(t, 16) for t in line.split()] for line in res.stdout.strip().splitlines()]
    assert len(ref) == len(cases)
    for idx, cs in enumerate(cases):
        got = o.philox4x32_10(cs[:4], (cs[4], cs[5]))
        assert [int(v) for v in got] == ref[idx], (idx, cs)


def test_box_muller_normals_have_standard_normal_moments():
    """Mean 0, variance 1, skewness 0, kurtosis 3 and pair independence over 2.4e6 draws
    of the oracle's per-site normals (24 per site)."""
    sites = np.arange(100_000, dtype=np.uint64)
    n = o.normals(seed=42, step=3, sites=sites)
    assert n.shape == (24, sites.size)
    z = n.ravel()
    se = 1.0 / np.sqrt(z.size)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0) * se
    assert abs((z ** 3).mean()) < 5 * np.sqrt(15.0) * se
    assert abs((z ** 4).mean() - 3.0) < 5 * np.sqrt(96.0) * se
    # the two members of a Box-Muller pair and two different calls are uncorrelated
    for a, b in ((0, 1), (2, 3), (0, 4), (5, 23)):
        assert abs(np.mean(n[a] * n[b])) < 5 / np.sqrt(sites.size)


def test_normals_depend_on_every_key_and_counter_word():
    s = np.arange(64, dtype=np.uint64)
    base = o.normals(1, 0, s, 0)
    for other in (o.normals(2, 0, s, 0), o.normals(1 + (1 << 32), 0, s, 0),
                  o.normals(1, 1, s, 0), o.normals(1, 0, s + 1, 0), o.normals(1, 0, s, 1)):
        assert not np.any(np.isclose(base, other))
