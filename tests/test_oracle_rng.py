"""Pins of the oracle's noise source: Philox4x32-10 against an independent
implementation (PyTorch's header-only engine, called, not copied), the exact
uniform mapping, and the Box-Muller normal statistics."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

_TORCH_PHILOX_DRIVER = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
// Reads lines "c0 c1 c2 c3 k0 k1" and prints the four output words of one
// Philox4x32-10 block with that counter and key. at::philox_engine builds its
// counter as (offset_lo, offset_hi, subsequence_lo, subsequence_hi) and its key
// as (seed_lo, seed_hi).
int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint64_t seed = (uint64_t(k1) << 32) | k0;
    uint64_t subseq = (uint64_t(c3) << 32) | c2;
    uint64_t offset = (uint64_t(c1) << 32) | c0;
    at::philox_engine e(seed, subseq, offset);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _torch_include():
    try:
        import torch  # noqa: F401
    except Exception:
        return None
    inc = os.path.join(os.path.dirname(__import__("torch").__file__), "include")
    if os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        return inc
    return None


def test_philox_matches_independent_implementation(oracle_mod):
    inc = _torch_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("PyTorch's Philox header or g++ not available")
    rng = np.random.default_rng(20)
    cases = [[0, 0, 0, 0, 0, 0], [0xFFFFFFFF] * 6, [1, 2, 3, 4, 5, 6]]
    cases += rng.integers(0, 2 ** 32, size=(200, 6), dtype=np.uint64).tolist()
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "drv.cpp")
        exe = os.path.join(td, "drv")
        with open(src, "w") as fh:
            fh.write(_TORCH_PHILOX_DRIVER)
        subprocess.run(["g++", "-O1", "-std=c++17", "-I", inc, src, "-o", exe], check=True)
        inp = "\n".join(" ".join(str(int(x)) for x in cs) for cs in cases) + "\n"
        res = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True)
    got_ref = [list(map(int, line.split())) for line in res.stdout.strip().splitlines()]
    assert len(got_ref) == len(cases)
    for cs, ref in zip(cases, got_ref):
        out = oracle_mod.philox(cs[:4], cs[4:])
        assert [int(x) for x in out] == ref, cs


def test_uniform_mapping_is_exact_and_open(oracle_mod):
    assert oracle_mod.uniform(0) == 2.0 ** -24
    assert oracle_mod.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle_mod.uniform(0x1FF) == 2.0 ** -24  # the low 9 bits are discarded
    assert oracle_mod.uniform(1 << 31) == 0.5 + 2.0 ** -24
    rng = np.random.default_rng(21)
    for w in rng.integers(0, 2 ** 32, 1000, dtype=np.uint64):
        u = oracle_mod.uniform(int(w))
        assert 0.0 < u < 1.0
        assert u == ((int(w) >> 9) + 0.5) / 2 ** 23
        assert np.float32(u) == u  # exactly representable in FP32


def test_box_muller_normals(oracle_mod):
    scipy_stats = pytest.importorskip("scipy.stats")
    z = np.concatenate([oracle_mod.normals_block(7, s // 97, s % 97, 0, s % 6) for s in range(60000)])
    n = len(z)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert z.var() == pytest.approx(1.0, abs=5 * np.sqrt(2 / n))
    kurt = ((z - z.mean()) ** 4).mean() / z.var() ** 2
    assert kurt == pytest.approx(3.0, abs=5 * np.sqrt(24 / n))
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    # The two members of a Box-Muller pair are uncorrelated.
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 5 / np.sqrt(len(zz))
    # Tail truncation at u >= 2^-24 bounds |z| by sqrt(2 * 24 ln 2) ~ 5.77.
    assert np.abs(z).max() <= np.sqrt(-2 * np.log(2.0 ** -24)) + 1e-12


def test_site_eta_layout(oracle_mod):
    # Noisy mode v uses normal n = v - D - 1: block n // 4, slot n % 4.
    for lat, D, Q in ((0, 2, 9), (1, 3, 27)):
        eta = oracle_mod.site_eta(lat, 123, 45, 678)
        assert np.all(eta[:D + 1] == 0.0)
        for v in range(D + 1, Q):
            n = v - D - 1
            assert eta[v] == oracle_mod.normals_block(123, 45, 678, 0, n // 4)[n % 4]


def test_noise_keys_are_distinct(oracle_mod):
    base = oracle_mod.normals_block(5, 10, 20, 0, 0)
    for args in ((6, 10, 20, 0, 0), (5, 11, 20, 0, 0), (5, 10, 21, 0, 0), (5, 10, 20, 1, 0),
                 (5, 10, 20, 0, 1), (5, 10 + (1 << 32), 20, 0, 0), (5 + (1 << 32), 10, 20, 0, 0)):
        assert not np.array_equal(base, oracle_mod.normals_block(*args)), args
