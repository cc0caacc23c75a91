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

Two generated dense sketches (s x len, entries regenerated from the seed, never
stored by the solver; readings of the transform and Gaussian sketches that
Section 2.7 names):

  * SRHT, a subsampled randomized Hadamard transform
    S = sqrt(M/s) R (H_M / sqrt(M)) D, M = 2^b the smallest power of two >= len
    (v padded with zeros), H_M the Sylvester-Hadamard matrix
    (H[i, j] = (-1)^popcount(i & j)), D = diag(d_c) random signs, R the s rows
    rho(0), ..., rho(s-1) of a seeded bijection of [0, M): entries
    S[r, c] = (-1)^(popcount(rho(r) & c) + d_c) / sqrt(s).
    With k = h(seed ^ TAG_SRHT, 0, 0) (the SplitMix64 hash above): x0 = low 32
    bits of k, K = (high 32 bits of k) | 1, h = max(1, b // 2), mask = M - 1;
    rho(r) = f(f((r ^ x0) & mask)) followed by x ^= x >> h, where
    f(x) = ((x ^ (x >> h)) * K) mod 2^32 & mask (xor-shift and odd multiplier:
    bijections of [0, M)).  d_c = bit 63 of the SplitMix64 output of state
    (seed ^ TAG_SIGN) ^ c.
  * Gaussian: S[r, c] = g / sqrt(s) with g = sqrt(-2 ln u1) cos(2 pi u2)
    (Box-Muller), u1 = (hi53(h1) + 1) 2^-53, u2 = hi53(h2) 2^-53, h1 and h2 the
    SplitMix64 outputs of states (seed ^ TAG_GAUSS) ^ (2 key) and ^ (2 key + 1),
    key = r * len + c, hi53 the top 53 bits.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

MASK64 = (1 << 64) - 1
TAG_SRHT = 0x5352485400000000
TAG_SIGN = 0x5352485400000001
TAG_GAUSS = 0x4741555353000000
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


# ---------------------------------------------------------------- generated dense sketches

def _mix_vec(state: np.ndarray) -> np.ndarray:
    """First SplitMix64 output of every uint64 state (numpy wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = state + np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def _popcount32(x: np.ndarray) -> np.ndarray:
    """Bits set in every uint32 entry (SWAR, no library popcount)."""
    x = x.astype(np.uint32)
    x = x - ((x >> np.uint32(1)) & np.uint32(0x55555555))
    x = (x & np.uint32(0x33333333)) + ((x >> np.uint32(2)) & np.uint32(0x33333333))
    x = (x + (x >> np.uint32(4))) & np.uint32(0x0F0F0F0F)
    with np.errstate(over="ignore"):
        return ((x * np.uint32(0x01010101)) >> np.uint32(24)).astype(np.int64)


def srht_order(length: int) -> int:
    """b with M = 2^b the smallest power of two >= length."""
    b = 0
    while (1 << b) < length:
        b += 1
    return b


def srht_rows(seed: int, s: int, length: int) -> np.ndarray:
    """rho(0), ..., rho(s-1): the sampled rows of H_M (distinct; s <= M)."""
    b = srht_order(length)
    M = 1 << b
    if not (1 <= s <= M):
        raise ValueError("need 1 <= s <= M")
    k = splitmix64_mix((seed ^ TAG_SRHT) + GOLDEN_GAMMA)
    x0, K = k & 0xFFFFFFFF, ((k >> 32) | 1) & 0xFFFFFFFF
    h, mask = max(1, b // 2), M - 1
    out = np.empty(s, dtype=np.int64)
    for r in range(s):
        x = (r ^ x0) & mask
        for _ in range(2):
            x ^= x >> h
            x = ((x * K) & 0xFFFFFFFF) & mask
        x ^= x >> h
        out[r] = x
    return out


def srht_signs(seed: int, length: int) -> np.ndarray:
    """d_c in {0, 1} (the sign is (-1)^d_c) for c < length."""
    st = np.uint64((seed ^ TAG_SIGN) & MASK64) ^ np.arange(length, dtype=np.uint64)
    return (_mix_vec(st) >> np.uint64(63)).astype(np.int64)


def srht_dense(seed: int, s: int, length: int) -> np.ndarray:
    """The s x length SRHT sketch (entries +-1/sqrt(s))."""
    rho = srht_rows(seed, s, length).astype(np.uint32)
    c = np.arange(length, dtype=np.uint32)
    par = (_popcount32(rho[:, None] & c[None, :]) + srht_signs(seed, length)[None, :]) & 1
    return (1.0 - 2.0 * par) / math.sqrt(s)


def gaussian_hash_dense(seed: int, s: int, length: int) -> np.ndarray:
    """The s x length Gaussian sketch drawn from the hash (entries N(0, 1/s))."""
    key = (np.arange(s, dtype=np.uint64)[:, None] * np.uint64(length) + np.arange(length, dtype=np.uint64)[None, :])
    base = np.uint64((seed ^ TAG_GAUSS) & MASK64)
    with np.errstate(over="ignore"):
        h1 = _mix_vec(base ^ (key * np.uint64(2)))
        h2 = _mix_vec(base ^ (key * np.uint64(2) + np.uint64(1)))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)
    return g / math.sqrt(s)


class SRHT(DenseSketch):
    """Subsampled randomized Hadamard transform drawn from the seed (dense here; the GPU regenerates it)."""

    def __init__(self, seed: int, s: int, length: int):
        super().__init__(srht_dense(seed, s, length))


class GaussianHash(DenseSketch):
    """Gaussian sketch drawn from the seed by Box-Muller (dense here; the GPU regenerates it)."""

    def __init__(self, seed: int, s: int, length: int):
        super().__init__(gaussian_hash_dense(seed, s, length))
