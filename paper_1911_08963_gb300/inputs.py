"""Seeded synthetic inputs: random binary codes G = [I_k | R] and workload traces.

This module is shared by the GPU library's tests/benchmark and by the CPU oracle's
tests.  It draws random bits and packs them; it holds none of the minimum-distance
arithmetic (no elimination, no weights, no enumeration).

Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the
output mix z = (z ^ z>>30) * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) * 0x94D049BB133111EB;
z ^ z>>31.

Packing: a matrix of k rows and n columns is a numpy uint64 array of shape
(k, ceil(n/64)); bit t of word w of row i is entry (i, 64w + t); padding bits are zero.

The paper's own test matrices (its codes "mat015", "mat023", Section 4) are not
available; the workloads below are random linear codes of comparable length and
dimension, which is the class of codes the paper targets.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, bound: int) -> int:
        """An integer in [0, bound) (modulo reduction; the bias is below 2^-50 here)."""
        return self.next() % bound

    def uniform(self) -> float:
        """A double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


def words(n: int) -> int:
    return (n + 63) // 64


def draw_R(rng: SplitMix64, k: int, r: int) -> np.ndarray:
    """k rows of r i.i.d. Bernoulli(1/2) bits: one 64-bit draw per 64 columns of a row."""
    R = np.zeros((k, words(r)), dtype=np.uint64)
    for i in range(k):
        for w in range(words(r)):
            bits = rng.next()
            width = min(64, r - 64 * w)
            if width < 64:
                bits &= (1 << width) - 1
            R[i, w] = bits
    return R


def systematic(R: np.ndarray, n: int, k: int) -> np.ndarray:
    """G = [I_k | R] packed: row i has column i set and R's row i in columns k..n-1."""
    r = n - k
    G = np.zeros((k, words(n)), dtype=np.uint64)
    for i in range(k):
        row = 1 << i
        for w in range(words(r)):
            row |= int(R[i, w]) << (k + 64 * w)
        for w in range(words(n)):
            G[i, w] = (row >> (64 * w)) & MASK64
    return G


def random_code(n: int, k: int, seed: int, skip: int = 0) -> np.ndarray:
    """G = [I_k | R] with R drawn from SplitMix64(seed), after `skip` whole R draws."""
    rng = SplitMix64(seed)
    for _ in range(skip):
        draw_R(rng, k, n - k)
    return systematic(draw_R(rng, k, n - k), n, k)


# Single-code workloads.  `skip` is the number of leading R draws of the seed's stream
# that were singular over F2: each code uses the first draw whose R is invertible, so
# that G has two disjoint full-rank information sets (the identity columns and the R
# columns).  The values were found by tests/golden/make_single_codes.py, which calls
# only the CPU oracle, and tests/test_inputs.py re-checks them.
SINGLE = {
    "rand64x32": dict(n=64, k=32, seed=1, skip=1),
    "rand128x64": dict(n=128, k=64, seed=2, skip=2),
    "rand200x100": dict(n=200, k=100, seed=3, skip=0),
}


def single_code(name: str) -> tuple[np.ndarray, int, int]:
    c = SINGLE[name]
    return random_code(c["n"], c["k"], c["seed"], c["skip"]), c["n"], c["k"]


def batch_codes(count: int = 2048, seed: int = 4, n_lo: int = 48, n_hi: int = 160):
    """Uneven batch: n ~ U{n_lo..n_hi}, k ~ U{ceil(n/3)..floor(n/2)}, G = [I_k | R].
    R is not conditioned, so some codes have a rank-deficient last information set."""
    rng = SplitMix64(seed)
    codes = []
    for _ in range(count):
        n = n_lo + rng.below(n_hi - n_lo + 1)
        klo, khi = -(-n // 3), n // 2
        k = klo + rng.below(khi - klo + 1)
        codes.append((systematic(draw_R(rng, k, n - k), n, k), n, k))
    return codes


def serving_trace(count: int, seed: int = 5, rate: float = 200.0, n_lo: int = 64, n_hi: int = 200,
                  spread: int = 8):
    """Poisson arrivals (exponential gaps of mean 1/rate seconds) of random codes with
    n ~ U{n_lo..n_hi} and k = floor(n/2) + delta, delta ~ U{-spread..spread}.
    Returns a list of (arrival_time_s, G, n, k)."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        n = n_lo + rng.below(n_hi - n_lo + 1)
        k = n // 2 + rng.below(2 * spread + 1) - spread
        k = max(1, min(n - 1, k))
        out.append((t, systematic(draw_R(rng, k, n - k), n, k), n, k))
    return out
