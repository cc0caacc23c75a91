"""Sketching operators for the oracle (test infrastructure; plain FP64 CPU).

Section 2.7 of the paper lists Gaussian sketches and CountSketch-like sparse
sketches; the sparse-sign sketch used here generalises CountSketch to `zeta`
nonzeros per column (zeta = 1 is CountSketch).  Its entries are *regenerated*
from a counter-based hash rather than stored, so the GPU path and this oracle
each implement the same published generator independently:

  * SplitMix64 (G. L. Steele Jr., D. Lea, C. H. Flood, "Fast splittable
    pseudorandom number generators", OOPSLA 2014): state advances by the golden
    gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
    mix function  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
    z *= 0x94D049BB133111EB; z ^= z >> 31.
  * h(seed, c, t) = the first SplitMix64 output of a generator whose state is
    seed XOR (c * 2^32 + t), for column c and draw counter t = 0, 1, 2, ...
  * candidate row r = floor(h * s / 2^64); accepted if not yet chosen for
    column c; sign = +1 if bit 0 of h is 0, else -1; value = sign / sqrt(zeta).
    Draws continue until column c has `zeta` distinct rows.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB


def splitmix64_mix(z: int) -> int:
    """The SplitMix64 output function applied to an already-advanced state."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def splitmix64_stream(state: int, count: int) -> list[int]:
    """`count` consecutive SplitMix64 outputs from the given initial state."""
    out = []
    for _ in range(count):
        state = (state + GOLDEN_GAMMA) & MASK64
        out.append(splitmix64_mix(state))
    return out


def draw_hash(seed: int, c: int, t: int) -> int:
    """h(seed, c, t): first SplitMix64 output from state seed ^ (c*2^32 + t)."""
    return splitmix64_stream((seed ^ ((c << 32) + t)) & MASK64, 1)[0]


def sparse_sign_column(seed: int, s: int, zeta: int, c: int) -> list[tuple[int, int]]:
    """The (row, sign) pairs of column c, in draw order (pure-Python definition)."""
    if not (1 <= zeta <= s):
        raise ValueError("need 1 <= zeta <= s")
    rows: list[int] = []
    signs: list[int] = []
    t = 0
    while len(rows) < zeta:
        h = draw_hash(seed, c, t)
        r = (h * s) >> 64
        if r not in rows:
            rows.append(r)
            signs.append(1 if (h & 1) == 0 else -1)
        t += 1
    return list(zip(rows, signs))


def _hash_vec(seed: int, cols: np.ndarray, t: int) -> np.ndarray:
    """Vectorised draw_hash over many columns (numpy uint64 wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        x = np.uint64(seed) ^ ((cols.astype(np.uint64) << np.uint64(32)) + np.uint64(t))
        z = x + np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def _mulhi_s(h: np.ndarray, s: int) -> np.ndarray:
    """floor(h * s / 2^64) for uint64 h and s < 2^31, without 128-bit integers."""
    hi = h >> np.uint64(32)
    lo = h & np.uint64(0xFFFFFFFF)
    s64 = np.uint64(s)
    with np.errstate(over="ignore"):
        return (hi * s64 + ((lo * s64) >> np.uint64(32))) >> np.uint64(32)


def sparse_sign_rows(seed: int, s: int, zeta: int, ncols: int) -> tuple[np.ndarray, np.ndarray]:
    """Rows (ncols, zeta) int64 and signs (ncols, zeta) of every column, in draw
    order; same definition as sparse_sign_column, vectorised over columns."""
    if not (1 <= zeta <= s):
        raise ValueError("need 1 <= zeta <= s")
    rows = np.full((ncols, zeta), -1, dtype=np.int64)
    signs = np.zeros((ncols, zeta), dtype=np.int64)
    filled = np.zeros(ncols, dtype=np.int64)
    cols = np.arange(ncols, dtype=np.int64)
    t = 0
    active = cols
    while active.size:
        h = _hash_vec(seed, active, t)
        r = _mulhi_s(h, s).astype(np.int64)
        sg = np.where((h & np.uint64(1)) == 0, 1, -1)
        dup = (rows[active] == r[:, None]).any(axis=1)
        ok = ~dup
        acc = active[ok]
        rows[acc, filled[acc]] = r[ok]
        signs[acc, filled[acc]] = sg[ok]
        filled[acc] += 1
        active = active[filled[active] < zeta]
        t += 1
    return rows, signs


class Sketch:
    """An s x length sketching matrix with apply() and dense()."""

    def __init__(self, s: int, length: int):
        self.s, self.length = s, length

    def apply(self, v: np.ndarray) -> np.ndarray:
        raise NotImplementedError

    def dense(self) -> np.ndarray:
        raise NotImplementedError


class SparseSign(Sketch):
    """Sparse-sign sketch: column c has zeta entries +-1/sqrt(zeta) (CountSketch for zeta=1)."""

    def __init__(self, seed: int, s: int, zeta: int, length: int):
        super().__init__(s, length)
        self.seed, self.zeta = seed, zeta
        rows, signs = sparse_sign_rows(seed, s, zeta, length)
        vals = signs.astype(np.float64) / math.sqrt(zeta)
        cols = np.repeat(np.arange(length), zeta)
        self.mat = sp.csc_matrix((vals.ravel(), (rows.ravel(), cols)), shape=(s, length))

    def apply(self, v):
        return self.mat @ v

    def dense(self):
        return self.mat.toarray()


class DenseSketch(Sketch):
    """Explicit dense sketch (e.g. Gaussian with N(0,1) entries, Corollary 1)."""

    def __init__(self, S: np.ndarray):
        super().__init__(S.shape[0], S.shape[1])
        self.S = np.asarray(S, dtype=np.float64)

    def apply(self, v):
        return self.S @ v

    def dense(self):
        return self.S


class IdentitySketch(Sketch):
    """S = I (s = length): turns the sketched LS into the unsketched one."""

    def __init__(self, length: int):
        super().__init__(length, length)

    def apply(self, v):
        return np.array(v, dtype=np.float64, copy=True)

    def dense(self):
        return np.eye(self.length)


def gaussian(rng: np.random.Generator, s: int, length: int) -> DenseSketch:
    """Gaussian sketch with independent N(0,1) entries (unscaled, as in Corollary 1)."""
    return DenseSketch(rng.standard_normal((s, length)))
