"""Brute-force sum-check in Python big integers, for tiny circuits only.

This is a second, independent definition of the prover's messages, used to pin
the oracle.  It does not use the gate-centric formula nor table folding: every
round polynomial is the literal sum of the layer polynomial

    f(p, w1, w2) = eq(z, p) [ add~(p,w1,w2) (V~(w1) + V~(w2)) + mult~(p,w1,w2) V~(w1) V~(w2) ]

over all Boolean settings of the unbound variables, where add~ and mult~ are
the multilinear extensions of the gate-triple indicator functions and V~ is the
multilinear extension of the next layer (GKR iteration, Sec. 3.1 of the paper).
"""
from __future__ import annotations

import itertools

P = (1 << 61) - 1


def eq1(x, b):
    return (x * b + (1 - x) * (1 - b)) % P


def eq(xs, ys):
    r = 1
    for x, y in zip(xs, ys):
        r = r * eq1(x, y) % P
    return r


def bits(v, n):
    return [(v >> k) & 1 for k in range(n)]


def mle(V, x):
    n = len(x)
    acc = 0
    for b in range(1 << n):
        acc = (acc + eq(x, bits(b, n)) * V[b]) % P
    return acc


def wiring(gates, si, sn, p, w1, w2):
    """(add~, mult~) at (p, w1, w2) from the gate list [(type, in1, in2)]."""
    add = mult = 0
    for g, (ty, a, b) in enumerate(gates):
        w = eq(p, bits(g, si)) * eq(w1, bits(a, sn)) % P * eq(w2, bits(b, sn)) % P
        if ty:
            mult = (mult + w) % P
        else:
            add = (add + w) % P
    return add, mult


def layer_poly(gates, si, sn, Vn, z, x):
    p, w1, w2 = x[:si], x[si:si + sn], x[si + sn:]
    add, mult = wiring(gates, si, sn, p, w1, w2)
    a, b = mle(Vn, w1), mle(Vn, w2)
    return eq(z, p) * ((add * (a + b) + mult * a * b) % P) % P


def inv(a):
    return pow(a, P - 2, P)


def lagrange(q, x):
    n = len(q) - 1
    acc = 0
    for t in range(n + 1):
        num = den = 1
        for u in range(n + 1):
            if u != t:
                num = num * (x - u) % P
                den = den * (t - u) % P
        acc = (acc + q[t] * num * inv(den)) % P
    return acc


def prove(gates_by_layer, log_width, layer_values, challenges):
    """Whole transcript by brute force.  challenges: the field elements the
    verifier draws, in protocol order (output point, then per layer the round
    challenges and tau)."""
    d = len(gates_by_layer)
    ch = iter(int(c) for c in challenges)
    out = [int(v) for v in layer_values[0]]
    z = [next(ch) for _ in range(log_width[0])]
    for i in range(d):
        si, sn = log_width[i], log_width[i + 1]
        n = si + 2 * sn
        Vn = [int(v) for v in layer_values[i + 1]]
        gates = gates_by_layer[i]
        r = []
        for j in range(n):
            for t in (0, 1, 2):
                acc = 0
                for suffix in itertools.product((0, 1), repeat=n - j - 1):
                    acc = (acc + layer_poly(gates, si, sn, Vn, z, r + [t] + list(suffix))) % P
                out.append(acc)
            r.append(next(ch))
        r1, r2 = r[si:si + sn], r[si + sn:]
        for t in range(sn + 1):
            out.append(mle(Vn, [(a + t * (b - a)) % P for a, b in zip(r1, r2)]))
        tau = next(ch)
        z = [(a + tau * (b - a)) % P for a, b in zip(r1, r2)]
    return out
