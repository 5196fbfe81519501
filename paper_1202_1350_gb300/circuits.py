"""Layer descriptions of the paper's benchmark circuits (Sec. 6.2.1), in the
form vc_circuit_create takes: log widths from the output layer (index 0) to the
input layer, and the wiring kind of each layer.

  F2       sum of squares: a squaring layer, then a binary addition tree.
  F0       distinct elements by Fermat's little theorem: per input the pair
           (x^2, 2x), then 59 pair layers that square the first entry and
           multiply the second by it, then a layer squaring the second entry,
           giving 4 x^(p-1) = 4 [x != 0]; then an addition tree.  Output 4 F0.
  MatMult  C = A B: n^3 products A[i][k] B[k][j], then an addition tree over k
           (the n^2 entries of C are the outputs).
  pattern_match, matmult_check: the paper's pattern-matching circuit and its
           single-output MatMult check, both ending in the F0 subcircuit; their
           lowest layers have explicit wiring.
"""
from __future__ import annotations

import numpy as np

from .vc import EXPLICIT, F0_FINAL, F0_FIRST, F0_PAIR, MATMULT, SQUARE, TREE


def f2(logn: int):
    return [*range(logn + 1), logn], [TREE] * logn + [SQUARE]


def f0(logn: int):
    # layers: tree (logn), final power layer, 59 pair layers, first power layer
    widths = [*range(logn + 1)] + [logn + 1] * 60 + [logn]
    kinds = [TREE] * logn + [F0_FINAL] + [F0_PAIR] * 59 + [F0_FIRST]
    return widths, kinds


def matmult(logn: int):
    L = logn
    widths = [2 * L + j for j in range(L + 1)] + [2 * L + 1]
    kinds = [TREE] * L + [MATMULT]
    return widths, kinds


def _f0_top(a: int):
    """Layers 0.. of an F0 subcircuit over 2^a values: log widths and kinds of
    the a addition layers, the final power layer, 59 pair layers and the
    first power layer (whose input has width 2^a)."""
    return [*range(a + 1)] + [a + 1] * 60, [TREE] * a + [F0_FINAL] + [F0_PAIR] * 59 + [F0_FIRST]


def pattern_match(log_n: int, log_q: int):
    """Pattern matching over a text of 2^log_n symbols and a pattern of
    2^log_q symbols: per location i, v_i = sum_j (t_{i+j} - p_j)^2, then
    4 [v_i != 0] and a sum, so the output is 4 (n - occurrences).  Locations
    past n - q get v_i = q (never an occurrence).  Input layout: text,
    pattern, p - 1, 1, zeros (2n entries).  Returns (log widths, kinds,
    explicit layers: None or (type, in1, in2) with type 0 = ADD, 1 = MUL)."""
    a, b = log_n, log_q
    if a < 2 or not 0 <= b < a:
        raise ValueError("need 2 <= log_n and log_q < log_n")
    n, q = 1 << a, 1 << b
    neg, one = n + q, n + q + 1
    # A: text * 1, pattern * (p - 1), and 1 * 1 everywhere else
    k = np.arange(2 * n, dtype=np.uint32)
    a_in1 = np.where(k < n + q, k, one).astype(np.uint32)
    a_in2 = np.where((k >= n) & (k < n + q), neg, one).astype(np.uint32)
    layer_a = (np.ones(2 * n, np.uint8), a_in1, a_in2)
    # B: gate i q + j = t_{i+j} + (-p_j) where the pattern fits, else 1 * 1
    loc, j = np.divmod(np.arange(n * q, dtype=np.int64), q)
    fits = loc + q <= n
    b_ty = np.where(fits, 0, 1).astype(np.uint8)
    b_in1 = np.where(fits, loc + j, neg).astype(np.uint32)  # entry n + q of A is 1
    b_in2 = np.where(fits, n + j, neg).astype(np.uint32)
    w, kinds = _f0_top(a)
    w += [*range(a, a + b)] + [a + b, a + b, a + 1, a + 1]
    kinds += [TREE] * b + [SQUARE, EXPLICIT, EXPLICIT]
    return w, kinds, [None] * (len(kinds) - 2) + [(b_ty, b_in1, b_in2), layer_a]


def matmult_check(logm: int):
    """Single-output MatMult check C = A B for m x m matrices, m = 2^logm: one
    explicit layer of, per entry (i, j), the m products A_ik B_kj, C_ij (p - 1)
    and m - 1 zero products; logm + 1 addition layers give (A B - C)_ij; then
    F0, so the output is 4 #{(i, j) : (A B)_ij != C_ij}.  Input layout: A, B,
    C row-major, p - 1, zeros (4 m^2 entries)."""
    L = logm
    if L < 1:
        raise ValueError("need logm >= 1")
    m = 1 << L
    m2 = m * m
    neg, zero = 3 * m2, 3 * m2 + 1
    ij, kk = np.divmod(np.arange(2 * m * m2, dtype=np.int64), 2 * m)
    i, j = np.divmod(ij, m)
    prod = kk < m
    in1 = np.where(prod, i * m + kk, np.where(kk == m, 2 * m2 + ij, zero)).astype(np.uint32)
    in2 = np.where(prod, m2 + kk * m + j, np.where(kk == m, neg, zero)).astype(np.uint32)
    w, kinds = _f0_top(2 * L)
    w += [*range(2 * L, 3 * L + 1)] + [3 * L + 1, 2 * L + 2]
    kinds += [TREE] * (L + 1) + [EXPLICIT]
    return w, kinds, [None] * (len(kinds) - 1) + [(np.ones(2 * m * m2, np.uint8), in1, in2)]


def by_name(family: str, logn: int):
    return {"f2": f2, "f0": f0, "matmult": matmult}[family](logn)


def non_input_gates(log_width) -> int:
    """Gates outside the input layer (the count behind gates/s)."""
    return sum(1 << s for s in log_width[:-1])


def transcript_len(log_width) -> int:
    """u64 entries of a proof transcript: the outputs, three values per
    sum-check round and s_{i+1} + 1 line values per layer."""
    s = [int(v) for v in log_width]
    n = 1 << s[0]
    for i in range(len(s) - 1):
        n += 3 * (s[i] + 2 * s[i + 1]) + s[i + 1] + 1
    return n
