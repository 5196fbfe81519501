"""Transcript parity of the CUDA prover with the CPU oracle (bit-exact: every
transcript entry is an exact field element).

Sizes sweep every tiling boundary of the device plan: product-weighted
sum-check CTAs fold 2^13 entries and general ones 2^10; line-reduction waves
fold 13 coordinates, then 8 per later wave, and a single-chunk wave runs as the
tail of the wave before it.  Widths 2^0..2^13, 2^16, 2^20, 2^21 and 2^22 cover
single-CTA, multi-CTA, tail and two-launch-plus-tail shapes; each benchmark
workload runs at its full size with its own input recipe."""
import random

import numpy as np
import pytest

from gpu_util import ensure_built, first_mismatch, gpu_prove, oracle_prove
from paper_1202_1350_gb300 import circuits
from paper_1202_1350_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
P = (1 << 61) - 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def check(widths, kinds, x, seeds, explicit=None):
    for seed in seeds:
        g = gpu_prove(widths, kinds, x, seed, explicit)
        o = oracle_prove(widths, kinds, x, seed, explicit)
        assert len(g) == len(o)
        assert first_mismatch(g, o) is None, f"seed {seed}: first mismatch at {first_mismatch(g, o)}"


@pytest.mark.parametrize("logn", list(range(0, 14)) + [16])
def test_f2_sizes(logn):
    x = I.f2_inputs(logn, 1 << 16, 1000 + logn)
    check(*circuits.f2(logn), x, seeds=(1, 0xDEADBEEF))


def test_f2_edge_values():
    x = np.array([0, P - 1, 1, P - 2, 1 << 60, 0, 5, P - 1] * 4, dtype=np.uint64)
    check(*circuits.f2(5), x, seeds=(3,))


@pytest.mark.parametrize("logn", [1, 2, 3, 4, 6, 8, 9, 10, 12])
def test_f0_sizes(logn):
    x = I.f0_inputs(logn, 2000 + logn)
    check(*circuits.f0(logn), x, seeds=(7,))


@pytest.mark.parametrize("logn", [0, 1, 2, 3, 4, 5])
def test_matmult_sizes(logn):
    x = I.matmult_inputs(logn, 1 << 10, 3000 + logn)
    check(*circuits.matmult(logn), x, seeds=(11,))


def random_explicit(rng, widths):
    layers = []
    for i in range(len(widths) - 1):
        S, Sn = 1 << widths[i], 1 << widths[i + 1]
        layers.append((np.array([rng.randrange(2) for _ in range(S)], np.uint8),
                       np.array([rng.randrange(Sn) for _ in range(S)], np.uint32),
                       np.array([rng.randrange(Sn) for _ in range(S)], np.uint32)))
    return layers


@pytest.mark.parametrize("widths", [[0, 0], [0, 1], [1, 0], [2, 3, 1], [3, 3, 3], [5, 4, 6],
                                    [12, 13], [13, 12], [11, 11, 12], [4, 0, 3]])
def test_explicit_random_circuits(widths):
    rng = random.Random(sum(widths) * 31 + len(widths))
    ex = random_explicit(rng, widths)
    x = np.array([rng.randrange(P) for _ in range(1 << widths[-1])], np.uint64)
    check(widths, [6] * (len(widths) - 1), x, seeds=(5, 99), explicit=ex)


def test_mixed_structured_and_explicit():
    rng = random.Random(4)
    widths = [0, 1, 2, 3, 3]
    kinds = [1, 1, 6, 0]
    ex = [None, None, random_explicit(rng, [2, 3])[0], None]
    x = np.array([rng.randrange(1 << 20) for _ in range(8)], np.uint64)
    check(widths, kinds, x, seeds=(8,), explicit=ex)


# --- the benchmark workloads at full size ------------------------------------------

def test_workload_f2_2e10():
    fam, logn, gen, seed = I.WORKLOADS["f2_2^10"]
    check(*circuits.f2(logn), gen(seed), seeds=(1, 2))


def test_workload_f2_2e20():
    fam, logn, gen, seed = I.WORKLOADS["f2_2^20"]
    check(*circuits.f2(logn), gen(seed), seeds=(1,))


def test_f2_2e21_line_tail():
    x = I.f2_inputs(21, 1 << 16, 77)
    check(*circuits.f2(21), x, seeds=(5,))


def test_f2_2e22_second_line_wave_and_tail():
    """n = 22: line waves of 13, 8 (two chunks) and 1 coordinate (tail)."""
    x = I.f2_inputs(22, 1 << 16, 78)
    check(*circuits.f2(22), x, seeds=(6,))


def test_workload_f0_2e16():
    fam, logn, gen, seed = I.WORKLOADS["f0_2^16"]
    check(*circuits.f0(logn), gen(seed), seeds=(1,))


def test_workload_matmult_128():
    fam, logn, gen, seed = I.WORKLOADS["matmult_128"]
    check(*circuits.matmult(logn), gen(seed), seeds=(1,))


# the paper's pattern-matching circuit and its single-output MatMult check: two
# explicit layers (one) under a squaring layer / addition trees and the F0 layers

@pytest.mark.parametrize("a,b", [(2, 0), (3, 1), (5, 2), (7, 3), (9, 2)])
def test_pattern_match(a, b):
    w, k, ex = circuits.pattern_match(a, b)
    check(w, k, I.pm_inputs(a, b, 40 + a), seeds=(3, 0xFEED), explicit=ex)


@pytest.mark.parametrize("logm,errors", [(1, 0), (2, 0), (2, 2), (3, 0), (3, 4), (4, 1)])
def test_matmult_check(logm, errors):
    w, k, ex = circuits.matmult_check(logm)
    check(w, k, I.mm1_inputs(logm, 50 + logm, errors=errors), seeds=(5,), explicit=ex)
