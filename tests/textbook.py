"""Codes whose minimum distance is fixed by their definition, and small GF(2) helpers.

Everything here is written for the tests, independently of both the oracle and the GPU
library: rows are Python integers (bit c = column c), elimination is done with them, and
combinations come from itertools.

Weight enumerators quoted are textbook facts (MacWilliams and Sloane, "The Theory of
Error-Correcting Codes": Ch. 1 for Hamming, simplex and Reed-Muller first order codes,
Ch. 2 Sec. 6 for the extended Golay code).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def pack(rows, n):
    """List of Python-int rows -> packed uint64 array (k, ceil(n/64))."""
    nw = (n + 63) // 64
    G = np.zeros((len(rows), nw), dtype=np.uint64)
    for i, r in enumerate(rows):
        for w in range(nw):
            G[i, w] = (r >> (64 * w)) & ((1 << 64) - 1)
    return G


def unpack(G):
    """Packed uint64 array -> list of Python-int rows."""
    G = np.asarray(G, dtype=np.uint64)
    out = []
    for row in G:
        v = 0
        for w, x in enumerate(row):
            v |= int(x) << (64 * w)
        out.append(v)
    return out


def wt(x: int) -> int:
    return bin(x).count("1")


def gf2_rank(rows) -> int:
    basis = {}  # leading bit -> row
    r = 0
    for v in rows:
        while v:
            h = v.bit_length() - 1
            if h in basis:
                v ^= basis[h]
            else:
                basis[h] = v
                r += 1
                break
    return r


def in_rowspace(rows, x: int) -> bool:
    return gf2_rank(list(rows) + [x]) == gf2_rank(rows)


def solve_message(rows, x: int):
    """A message m (bit i = row i) with sum_i m_i rows[i] == x, or None."""
    # track combinations alongside the basis
    basis = {}
    for i, v in enumerate(rows):
        comb = 1 << i
        while v:
            h = v.bit_length() - 1
            if h in basis:
                v ^= basis[h][0]
                comb ^= basis[h][1]
            else:
                basis[h] = (v, comb)
                break
    comb = 0
    while x:
        h = x.bit_length() - 1
        if h not in basis:
            return None
        x ^= basis[h][0]
        comb ^= basis[h][1]
    return comb


def column(rows, c) -> int:
    """Column c of the matrix as an integer (bit i = row i)."""
    return sum(((r >> c) & 1) << i for i, r in enumerate(rows))


def all_codewords(rows):
    """Every codeword xG, x over all 2^k messages."""
    k = len(rows)
    out = []
    for x in range(1 << k):
        v = 0
        for i in range(k):
            if (x >> i) & 1:
                v ^= rows[i]
        out.append(v)
    return out


def weight_distribution(rows, n):
    dist = [0] * (n + 1)
    for v in all_codewords(rows):
        dist[wt(v)] += 1
    return dist


def colex_rank_formula(c) -> int:
    """sum_i C(c_i, i) with 1-based positions i."""
    return sum(math.comb(ci, i + 1) for i, ci in enumerate(c))


def level_scan(rows, g):
    """(least weight, first colex rank) over all g-subsets of the rows, via itertools."""
    best = None
    for c in itertools.combinations(range(len(rows)), g):
        v = 0
        for i in c:
            v ^= rows[i]
        key = (wt(v), colex_rank_formula(c))
        if best is None or key < best:
            best = key
    return best


# ----------------------------------------------------------------- constructions ---

def hamming(m: int):
    """Hamming code [2^m - 1, 2^m - 1 - m, 3]: the null space of the m x (2^m - 1) matrix
    whose columns are all nonzero m-bit vectors."""
    n = (1 << m) - 1
    H_cols = list(range(1, n + 1))           # column c of H is the integer c + 1
    rows = []
    for x in range(1 << n):
        s = 0
        for c in range(n):
            if (x >> c) & 1:
                s ^= H_cols[c]
        if s == 0 and x and gf2_rank(rows + [x]) > len(rows):
            rows.append(x)
        if len(rows) == n - m:
            break
    return rows, n, n - m


def golay24():
    """Extended Golay code [24, 12, 8]: shifts of the generator polynomial
    g(x) = 1 + x^2 + x^4 + x^5 + x^6 + x^10 + x^11 of the cyclic [23, 12, 7] Golay code,
    each extended by an overall parity bit at column 23."""
    gpoly = sum(1 << e for e in (0, 2, 4, 5, 6, 10, 11))
    rows = []
    for s in range(12):
        r = gpoly << s
        if wt(r) % 2:
            r |= 1 << 23
        rows.append(r)
    return rows, 24, 12


def reed_muller1(m: int):
    """First-order Reed-Muller RM(1, m) [2^m, m + 1, 2^(m-1)]: the all-ones word and the m
    coordinate functions evaluated at the points 0..2^m - 1."""
    n = 1 << m
    rows = [(1 << n) - 1]
    for i in range(m):
        rows.append(sum(((p >> i) & 1) << p for p in range(n)))
    return rows, n, m + 1


def simplex(m: int):
    """Simplex code [2^m - 1, m, 2^(m-1)]: columns are all nonzero m-bit vectors."""
    n = (1 << m) - 1
    rows = [sum((((c + 1) >> i) & 1) << c for c in range(n)) for i in range(m)]
    return rows, n, m


def repetition(n: int):
    return [(1 << n) - 1], n, 1


def single_parity(n: int):
    """[n, n-1, 2]: rows e_i + e_{n-1}."""
    return [(1 << i) | (1 << (n - 1)) for i in range(n - 1)], n, n - 1


def trivial(n: int):
    return [1 << i for i in range(n)], n, n


def scramble(rows, n, seed):
    """Same code, other generator: random invertible row operations and a column
    permutation are NOT applied (the column order fixes the information sets); only row
    operations, so the code is unchanged."""
    rng = np.random.default_rng(seed)
    rows = list(rows)
    k = len(rows)
    for _ in range(4 * k):
        a, b = rng.integers(0, k, size=2)
        if a != b:
            rows[a] ^= rows[b]
    return rows


def permute_columns(rows, n, seed):
    """An equivalent code (same weight distribution) with the columns permuted."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    out = []
    for r in rows:
        v = 0
        for c in range(n):
            if (r >> c) & 1:
                v |= 1 << int(perm[c])
        out.append(v)
    return out


def random_rows(n, k, seed, full_rank=True):
    rng = np.random.default_rng(seed)
    while True:
        rows = [int.from_bytes(rng.bytes((n + 7) // 8), "little") & ((1 << n) - 1) for _ in range(k)]
        if not full_rank or gf2_rank(rows) == k:
            return rows


TEXTBOOK = {
    # name: (constructor, d, {weight: count} for the nonzero codewords that pin A_w)
    "hamming7": (lambda: hamming(3), 3, {3: 7, 4: 7, 7: 1}),
    "hamming15": (lambda: hamming(4), 3, {3: 35}),
    "golay24": (golay24, 8, {8: 759, 12: 2576, 16: 759, 24: 1}),
    "rm1_4": (lambda: reed_muller1(4), 8, {8: 30, 16: 1}),
    "rm1_5": (lambda: reed_muller1(5), 16, {16: 62, 32: 1}),
    "simplex4": (lambda: simplex(4), 8, {8: 15}),
    "simplex5": (lambda: simplex(5), 16, {16: 31}),
    "repetition9": (lambda: repetition(9), 9, {9: 1}),
    "parity10": (lambda: single_parity(10), 2, {2: 45}),
    "trivial6": (lambda: trivial(6), 1, {1: 6}),
}
