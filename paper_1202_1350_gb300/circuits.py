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
"""
from __future__ import annotations

from .vc import F0_FINAL, F0_FIRST, F0_PAIR, MATMULT, SQUARE, TREE


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
