"""Pins of the oracle's generated dense sketches (SRHT, hash-drawn Gaussian)
against what the mathematics fixes: the Sylvester-Hadamard matrix built by
SciPy, orthogonality of the sampled rows, a permutation's distinctness,
unit columns, the Box-Muller formula on the scalar SplitMix64 definition,
and the normal law of the entries.  Planted mistakes in a copy of the
generator source must fail them.  CPU only."""
import importlib.util
import math
import os
import sys
import types

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "oracle", "sketch.py")).read()


def load_sketch(src: str):
    name = f"sketch_variant_{abs(hash(src))}"
    mod = types.ModuleType(name)
    sys.modules[name] = mod
    exec(compile(src, f"<{name}>", "exec"), mod.__dict__)
    return mod


def srht_pins(sk) -> bool:
    ok = True
    for seed, s, length in ((3, 16, 64), (11, 40, 100), (2**63 + 5, 64, 64), (9, 1, 1)):
        M = 1 << sk.srht_order(length)
        rho = sk.srht_rows(seed, s, length)
        ok &= len(set(rho.tolist())) == s and rho.min() >= 0 and rho.max() < M
        d = sk.srht_signs(seed, length)
        H = scipy.linalg.hadamard(M).astype(np.float64)
        ref = math.sqrt(M / s) * (H[rho, :length] / math.sqrt(M)) * np.where(d == 1, -1.0, 1.0)[None, :]
        S = sk.srht_dense(seed, s, length)
        ok &= np.allclose(S, ref, rtol=0, atol=1e-15)
        ok &= np.allclose(np.linalg.norm(S, axis=0), 1.0, rtol=0, atol=1e-14)
        if length == M:
            ok &= np.allclose(S @ S.T, (M / s) * np.eye(s), rtol=0, atol=1e-12)
    # s = M: the sampled rows are a permutation of [0, M)
    ok &= sorted(sk.srht_rows(21, 256, 256).tolist()) == list(range(256))
    # signs are balanced
    d = sk.srht_signs(5, 20000)
    ok &= abs(d.mean() - 0.5) < 4 * 0.5 / math.sqrt(20000)
    return bool(ok)


def gaussian_pins(sk) -> bool:
    ok = True
    seed, s, length = 17, 5, 7
    G = sk.gaussian_hash_dense(seed, s, length)
    # one entry from the scalar SplitMix64 definition and the Box-Muller formula
    r, c = 3, 4
    key = r * length + c
    h1 = sk.splitmix64_stream((seed ^ sk.TAG_GAUSS) ^ (2 * key), 1)[0]
    h2 = sk.splitmix64_stream((seed ^ sk.TAG_GAUSS) ^ (2 * key + 1), 1)[0]
    u1 = ((h1 >> 11) + 1) * 2.0 ** -53
    u2 = (h2 >> 11) * 2.0 ** -53
    g = math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2) / math.sqrt(s)
    ok &= abs(G[r, c] - g) <= 4e-16 * max(1.0, abs(g))
    # the entries follow N(0, 1/s): moments and a Kolmogorov-Smirnov test
    s2, n2 = 100, 10000
    x = (sk.gaussian_hash_dense(99, s2, n2) * math.sqrt(s2)).ravel()
    N = x.size
    ok &= abs(x.mean()) < 5 / math.sqrt(N)
    ok &= abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / N)
    ok &= abs(scipy.stats.kurtosis(x, fisher=False) - 3.0) < 0.05
    ok &= scipy.stats.kstest(x[:200000], "norm").pvalue > 1e-4
    return bool(ok)


def test_srht_pins():
    assert srht_pins(O.sketch)


def test_gaussian_hash_pins():
    assert gaussian_pins(O.sketch)


@pytest.mark.parametrize("old,new", [
    ("par = (_popcount32(rho[:, None] & c[None, :]) + srht_signs(seed, length)[None, :]) & 1",
     "par = (_popcount32(rho[:, None] | c[None, :]) + srht_signs(seed, length)[None, :]) & 1"),   # wrong index set
    ("par = (_popcount32(rho[:, None] & c[None, :]) + srht_signs(seed, length)[None, :]) & 1",
     "par = (_popcount32(rho[:, None] & c[None, :])) & 1"),                                          # dropped signs
    ("    return (1.0 - 2.0 * par) / math.sqrt(s)", "    return (1.0 - 2.0 * par) / math.sqrt(length)"),   # wrong scale
    ("            x = ((x * K) & 0xFFFFFFFF) & mask", "            x = ((x * (K + 1)) & 0xFFFFFFFF) & mask"),  # even multiplier
    ("    x = (x + (x >> np.uint32(4))) & np.uint32(0x0F0F0F0F)", "    x = (x + (x >> np.uint32(4))) & np.uint32(0x0F0F0F0E)"),
])
def test_srht_planted_mistakes_fail(old, new):
    assert SRC.count(old) == 1, old
    assert not srht_pins(load_sketch(SRC.replace(old, new)))


@pytest.mark.parametrize("old,new", [
    ("    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)",
     "    g = np.sqrt(-1.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)"),                    # wrong variance
    ("    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)",
     "    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(3.141592653589793 * u2)"),                    # half circle
    ("        h2 = _mix_vec(base ^ (key * np.uint64(2) + np.uint64(1)))",
     "        h2 = _mix_vec(base ^ (key * np.uint64(2)))"),                                     # correlated uniforms
])
def test_gaussian_planted_mistakes_fail(old, new):
    assert SRC.count(old) == 1, old
    assert not gaussian_pins(load_sketch(SRC.replace(old, new)))
