"""Seeded synthetic inputs for the benchmark circuits.

This module holds no protocol arithmetic: it only produces input vectors (and
job mixes) from a counter-based splitmix64 stream, so that the CUDA path and the
CPU oracle can be fed identical data.  The paper's own workloads are randomly
generated frequency vectors (Sec. 6.2.4, F2 discussion), so synthetic inputs of
the same shape stand in for them; no dataset is involved.

Recipes (input seed = 0xC0FFEE + workload index):
  F2, n = 2^10          x uniform in [0, 1000]
  F2, n = 2^20          x uniform in [0, 2^16]
  F0, universe 2^16     x ~ Poisson(1), capped at 2^10 (about 63.2 % nonzero)
  MatMult, n = 128      A, B uniform in [0, 2^10]
  batch                 512 F2 with log2 n uniform in {8..18} + 64 MatMult, n in {16, 32, 64}
  serving               70 % F2 with log2 n uniform in {10..22}, 30 % MatMult, n in {32, 64, 128}
  pattern matching      text and pattern uniform over 4 symbols, 3 planted occurrences
  MatMult check         A, B uniform in [0, 2^10], C = A B with seeded off-by-one entries
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
SEED_BASE = 0xC0FFEE


def splitmix64_stream(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of splitmix64 started at `seed` (vectorised)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_ints(seed: int, n: int, hi: int) -> np.ndarray:
    """n integers in [0, hi] (inclusive); modulo bias below 2^-40 for hi < 2^13."""
    z = splitmix64_stream(seed, n) >> np.uint64(11)
    return (z % np.uint64(hi + 1)).astype(np.uint64)


def poisson1_capped(seed: int, n: int, cap: int = 1 << 10) -> np.ndarray:
    """n draws of Poisson(1) by inverse CDF on 53-bit uniforms, capped at `cap`."""
    u = (splitmix64_stream(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    cdf = []
    acc, term = 0.0, math.exp(-1.0)
    for k in range(0, 40):
        acc += term
        cdf.append(acc)
        term /= (k + 1)
    x = np.searchsorted(np.array(cdf), u, side="right").astype(np.uint64)
    return np.minimum(x, np.uint64(cap))


def f2_inputs(logn: int, hi: int, seed: int) -> np.ndarray:
    return uniform_ints(seed, 1 << logn, hi)


def f0_inputs(logn: int, seed: int) -> np.ndarray:
    return poisson1_capped(seed, 1 << logn)


def matmult_inputs(logn: int, hi: int, seed: int) -> np.ndarray:
    """Inputs of the MatMult circuit: A row-major, then B row-major (2 n^2 values)."""
    n = 1 << logn
    return uniform_ints(seed, 2 * n * n, hi)


P61 = (1 << 61) - 1


def pm_inputs(log_n: int, log_q: int, seed: int, alphabet: int = 4, planted: int = 3) -> np.ndarray:
    """Inputs of the pattern-matching circuit: a text of n symbols and a
    pattern of q symbols, both uniform over `alphabet` symbols, with the
    pattern copied into the text at `planted` seeded locations; then the
    constants p - 1 and 1 and zeros (2n entries)."""
    n, q = 1 << log_n, 1 << log_q
    text = uniform_ints(seed, n, alphabet - 1)
    pat = uniform_ints(seed + 1, q, alphabet - 1)
    locs = splitmix64_stream(seed + 2, planted) % np.uint64(n - q + 1)
    for i in locs:
        text[int(i):int(i) + q] = pat
    x = np.zeros(2 * n, np.uint64)
    x[:n] = text
    x[n:n + q] = pat
    x[n + q] = P61 - 1
    x[n + q + 1] = 1
    return x


def mm1_inputs(logm: int, seed: int, hi: int = 1 << 10, errors: int = 0) -> np.ndarray:
    """Inputs of the single-output MatMult check: A, B uniform in [0, hi], the
    claimed product C = A B (exact integers, far below p) with `errors` seeded
    entries off by one, the constant p - 1 and zeros (4 m^2 entries)."""
    m = 1 << logm
    ab = uniform_ints(seed, 2 * m * m, hi).astype(np.int64)
    A, B = ab[:m * m].reshape(m, m), ab[m * m:].reshape(m, m)
    C = (A @ B).astype(np.uint64).ravel()
    if errors:
        pos = splitmix64_stream(seed + 1, errors) % np.uint64(m * m)
        for k in pos:
            C[int(k)] += np.uint64(1)
    x = np.zeros(4 * m * m, np.uint64)
    x[:2 * m * m] = ab.astype(np.uint64)
    x[2 * m * m:3 * m * m] = C
    x[3 * m * m] = P61 - 1
    return x


# Workload table: name -> (circuit family, log size, input recipe)
WORKLOADS = {
    "f2_2^10": ("f2", 10, lambda s: f2_inputs(10, 1000, s), SEED_BASE + 0),
    "f2_2^20": ("f2", 20, lambda s: f2_inputs(20, 1 << 16, s), SEED_BASE + 1),
    "f0_2^16": ("f0", 16, lambda s: f0_inputs(16, s), SEED_BASE + 1),
    "matmult_128": ("matmult", 7, lambda s: matmult_inputs(7, 1 << 10, s), SEED_BASE + 2),
}


def batch_mix(seed: int = SEED_BASE + 3, n_f2: int = 512, n_mm: int = 64):
    """Job list of the batched workload: (family, log size, input seed)."""
    z = splitmix64_stream(seed, n_f2 + n_mm)
    jobs = []
    for j in range(n_f2):
        jobs.append(("f2", 8 + int(z[j] % np.uint64(11)), seed * 1000003 + j))
    for j in range(n_mm):
        jobs.append(("matmult", 4 + int(z[n_f2 + j] % np.uint64(3)), seed * 1000003 + n_f2 + j))
    return jobs


def job_inputs(family: str, logn: int, seed: int) -> np.ndarray:
    if family == "f2":
        return f2_inputs(logn, 1 << 16, seed)
    if family == "f0":
        return f0_inputs(logn, seed)
    if family == "matmult":
        return matmult_inputs(logn, 1 << 10, seed)
    raise ValueError(family)


def serving_mix(seed: int, n_jobs: int):
    """Job list of the serving workload, in arrival order: (family, log size, input seed)."""
    z = splitmix64_stream(seed, 2 * n_jobs)
    jobs = []
    for j in range(n_jobs):
        if int(z[2 * j] % np.uint64(10)) < 7:
            jobs.append(("f2", 10 + int(z[2 * j + 1] % np.uint64(13)), seed * 1000003 + j))
        else:
            jobs.append(("matmult", 5 + int(z[2 * j + 1] % np.uint64(3)), seed * 1000003 + j))
    return jobs


def poisson_arrivals(seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    u = (splitmix64_stream(seed ^ 0x5EED, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)
