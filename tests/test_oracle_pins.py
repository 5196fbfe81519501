"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with a retyped copy of itself:
  * field operations against Python big integers (Sec. 6.1, p = 2^61 - 1);
  * multilinear extensions against Boolean-point values and multilinearity;
  * interpolation against polynomials evaluated directly;
  * round messages and line values against a brute-force sum over the Boolean
    hypercube of the layer polynomial built from add~/mult~ (tests/brute.py),
    an independent definition of the GKR iteration (Sec. 3.1);
  * the sum-check invariant g_j(0) + g_j(1) = running claim in every round;
  * closed forms of the benchmark circuits' outputs (Sec. 6.2.1);
  * completeness and soundness of the verifier (Sec. 2.1).
"""
import random

import numpy as np
import pytest

import brute
import oracle

P = oracle.P


# --- field ---------------------------------------------------------------------

EDGE = [0, 1, 2, P - 1, P - 2, (1 << 60), (1 << 61) - 2, 12345678901234567]


def test_field_ops_match_bigint():
    rng = random.Random(1)
    vals = EDGE + [rng.randrange(P) for _ in range(300)]
    for a in vals:
        for b in vals[:40]:
            assert oracle.fe_add(a, b) == (a + b) % P
            assert oracle.fe_sub(a, b) == (a - b) % P
            assert oracle.fe_mul(a, b) == (a * b) % P


def test_field_inverse_and_pow():
    rng = random.Random(2)
    for a in [1, 2, P - 1] + [rng.randrange(1, P) for _ in range(50)]:
        ai = oracle.fe_inv(a)
        assert a * ai % P == 1
        e = rng.randrange(1 << 64)
        assert oracle.fe_pow(a, e) == pow(a, e, P)
    # Fermat: a^(p-1) = 1 for a != 0 (the identity the F0 circuit relies on)
    assert oracle.fe_pow(0, P - 1) == 0
    assert oracle.fe_pow(7, P - 1) == 1


# --- multilinear extensions ------------------------------------------------------

def test_mle_boolean_points_and_multilinearity():
    rng = random.Random(3)
    for n in range(0, 6):
        V = [rng.randrange(P) for _ in range(1 << n)]
        for b in range(1 << n):
            assert oracle.mle(V, brute.bits(b, n)) == V[b]
        for _ in range(4):
            x = [rng.randrange(P) for _ in range(n)]
            assert oracle.mle(V, x) == brute.mle(V, x)
            for k in range(n):
                # degree 1 in each coordinate: value at 2 = 2 * value(1) - value(0)
                x0, x1, x2 = list(x), list(x), list(x)
                x0[k], x1[k], x2[k] = 0, 1, 2
                v0, v1, v2 = (oracle.mle(V, y) for y in (x0, x1, x2))
                assert v2 == (2 * v1 - v0) % P


def test_eq_definition():
    rng = random.Random(4)
    for n in range(0, 6):
        x = [rng.randrange(P) for _ in range(n)]
        y = [rng.randrange(P) for _ in range(n)]
        assert oracle.eq(x, y) == brute.eq(x, y)
        # eq(x, .) sums to 1 over the hypercube
        assert sum(oracle.eq(x, brute.bits(b, n)) for b in range(1 << n)) % P == 1


def test_interpolation_against_polynomials():
    rng = random.Random(5)
    for _ in range(20):
        c = [rng.randrange(P) for _ in range(3)]
        poly = lambda t: (c[0] + c[1] * t + c[2] * t * t) % P
        r = rng.randrange(P)
        assert oracle.interp3(poly(0), poly(1), poly(2), r) == poly(r)
    for deg in range(0, 9):
        c = [rng.randrange(P) for _ in range(deg + 1)]
        poly = lambda t: sum(ci * pow(t, k, P) for k, ci in enumerate(c)) % P
        x = rng.randrange(P)
        assert oracle.lagrange([poly(t) for t in range(deg + 1)], x) == poly(x)


# --- challenge generator (convention: restated from its published definition) ----

def test_splitmix64_restatement_and_range():
    def ref(seed, n):
        s, out = seed, []
        M = (1 << 64) - 1
        for _ in range(n):
            s = (s + 0x9E3779B97F4A7C15) & M
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
            out.append(z ^ (z >> 31))
        return out
    for seed in (0, 1, 0xC0FFEE, (1 << 64) - 1):
        assert [int(v) for v in oracle.splitmix64(seed, 16)] == ref(seed, 16)
    ch = oracle.draw_challenges(9, 1000)
    assert (ch < P).all()
    assert [int(v) for v in ch[:8]] == [v >> 3 for v in ref(9, 8)]


def test_splitmix64_published_values():
    """The oracle's stream against splitmix64's published known-answer values
    (tests/golden/splitmix64_kat.txt), not against a restatement."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2
    for row in rows:
        seed, want = int(row[0]), [int(v) for v in row[1:]]
        assert [int(v) for v in oracle.splitmix64(seed, len(want))] == want


# --- circuit expansions -------------------------------------------------------------

def expand_kind(kind, si, sn):
    """Gate lists of the structured wiring kinds, written from their definitions."""
    S = 1 << si
    if kind == oracle.SQUARE:
        return [(1, g, g) for g in range(S)]
    if kind == oracle.TREE:
        return [(0, 2 * g, 2 * g + 1) for g in range(S)]
    if kind == oracle.MATMULT:
        L = si // 3
        n = 1 << L
        gates = []
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    gates.append(None)
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    gates[i * n * n + j * n + k] = (1, i * n + k, n * n + k * n + j)
        return gates
    if kind == oracle.F0_FIRST:
        return [(1, g // 2, g // 2) if g % 2 == 0 else (0, g // 2, g // 2) for g in range(S)]
    if kind == oracle.F0_PAIR:
        return [(1, g, g) if g % 2 == 0 else (1, g, g - 1) for g in range(S)]
    if kind == oracle.F0_FINAL:
        return [(1, 2 * g + 1, 2 * g + 1) for g in range(S)]
    raise ValueError(kind)


@pytest.mark.parametrize("family,logn", [("f2", 3), ("f0", 2), ("matmult", 2), ("matmult", 1)])
def test_structured_expansion(family, logn):
    lw, kinds = getattr(oracle, f"{family}_layers")(logn)
    c = oracle.Circuit(lw, kinds)
    for i, k in enumerate(kinds):
        ty, a, b = c.layer_gates(i)
        ref = expand_kind(k, lw[i], lw[i + 1])
        assert [(int(t), int(x), int(y)) for t, x, y in zip(ty, a, b)] == ref


def test_bad_shapes_rejected():
    with pytest.raises(ValueError):
        oracle.Circuit([2, 2], [oracle.TREE])
    with pytest.raises(ValueError):
        oracle.Circuit([1, 3], [oracle.SQUARE])
    with pytest.raises(ValueError):
        oracle.Circuit([1, 1], [oracle.EXPLICIT],
                       explicit=[(np.array([0, 1]), np.array([0, 2]), np.array([1, 1]))])


# --- the protocol against brute force -----------------------------------------------

def random_explicit(rng, log_width):
    d = len(log_width) - 1
    layers = []
    for i in range(d):
        S, Sn = 1 << log_width[i], 1 << log_width[i + 1]
        ty = np.array([rng.randrange(2) for _ in range(S)], np.uint8)
        a = np.array([rng.randrange(Sn) for _ in range(S)], np.uint32)
        b = np.array([rng.randrange(Sn) for _ in range(S)], np.uint32)
        layers.append((ty, a, b))
    return layers


TINY_SHAPES = [[0, 1], [1, 1], [1, 2], [2, 1], [0, 0], [1, 0], [2, 2, 1], [0, 2, 2], [1, 2, 2, 1]]


def brute_case(c, gates_by_layer, inputs, seed):
    vals = c.evaluate(inputs)
    ch = oracle.draw_challenges(seed, c.num_challenges())
    return brute.prove(gates_by_layer, c.log_width, vals, ch)


@pytest.mark.parametrize("shape", TINY_SHAPES)
def test_explicit_circuit_matches_brute_force(shape):
    rng = random.Random(hash(tuple(shape)) & 0xFFFF)
    layers = random_explicit(rng, shape)
    c = oracle.Circuit(shape, [oracle.EXPLICIT] * (len(shape) - 1), explicit=layers)
    x = [rng.randrange(P) for _ in range(1 << shape[-1])]
    gates = [[(int(t), int(a), int(b)) for t, a, b in zip(*L)] for L in layers]
    for seed in (1, 77):
        ref = brute_case(c, gates, x, seed)
        t1 = c.prove(x, seed, form=1)
        t2 = c.prove(x, seed, form=2)
        assert [int(v) for v in t1] == ref
        assert [int(v) for v in t2] == ref
        assert c.verify(x, seed, t2) == (True, -1)


@pytest.mark.parametrize("family,logn", [("f2", 1), ("f2", 2), ("matmult", 1)])
def test_structured_circuits_match_brute_force(family, logn):
    lw, kinds = getattr(oracle, f"{family}_layers")(logn)
    c = oracle.Circuit(lw, kinds)
    gates = [expand_kind(k, lw[i], lw[i + 1]) for i, k in enumerate(kinds)]
    rng = random.Random(logn)
    x = [rng.randrange(1000) for _ in range(c.n_inputs)]
    ref = brute_case(c, gates, x, 5)
    assert [int(v) for v in c.prove(x, 5, form=1)] == ref
    assert [int(v) for v in c.prove(x, 5, form=2)] == ref


def test_f0_power_layers_match_brute_force():
    """The F0 power layers (first, pair, final) against brute force, on a short
    circuit that uses each kind once: input -> first -> pair -> final -> tree."""
    lw = [0, 1, 2, 2, 1]
    kinds = [oracle.TREE, oracle.F0_FINAL, oracle.F0_PAIR, oracle.F0_FIRST]
    c = oracle.Circuit(lw, kinds)
    gates = [expand_kind(k, lw[i], lw[i + 1]) for i, k in enumerate(kinds)]
    x = [3, 0]
    ref = brute_case(c, gates, x, 21)
    assert [int(v) for v in c.prove(x, 21, form=1)] == ref
    assert [int(v) for v in c.prove(x, 21, form=2)] == ref


def replay(c, transcript, seed):
    """Replay the verifier's claims in Python; returns per-round (g0+g1, claim)
    pairs and per-layer line data, using only big-integer arithmetic."""
    ch = [int(v) for v in oracle.draw_challenges(seed, c.num_challenges())]
    t = [int(v) for v in transcript]
    lw = c.log_width
    pos = 1 << lw[0]
    k = lw[0]
    z = ch[:k]
    claim = brute.mle(t[:pos], z)
    rounds, lines = [], []
    for i in range(c.d):
        si, sn = lw[i], lw[i + 1]
        r = []
        for j in range(si + 2 * sn):
            g0, g1, g2 = t[pos:pos + 3]
            pos += 3
            rounds.append(((g0 + g1) % P, claim))
            rj = ch[k]
            k += 1
            r.append(rj)
            # degree-2 interpolation through (0,g0),(1,g1),(2,g2)
            claim = brute.lagrange([g0, g1, g2], rj)
        q = t[pos:pos + sn + 1]
        pos += sn + 1
        tau = ch[k]
        k += 1
        lines.append((i, r[si:si + sn], r[si + sn:], q, tau))
        z = [(a + tau * (b - a)) % P for a, b in zip(r[si:si + sn], r[si + sn:])]
        claim = brute.lagrange(q, tau)
    return rounds, lines


@pytest.mark.parametrize("family,logn", [("f2", 5), ("f0", 2), ("matmult", 2)])
def test_round_invariant_and_line_values(family, logn):
    lw, kinds = getattr(oracle, f"{family}_layers")(logn)
    c = oracle.Circuit(lw, kinds)
    rng = random.Random(9)
    x = [rng.randrange(50) for _ in range(c.n_inputs)]
    vals = c.evaluate(x)
    t = c.prove(x, 3)
    rounds, lines = replay(c, t, 3)
    for s, claim in rounds:
        assert s == claim
    for i, r1, r2, q, tau in lines:
        Vn = [int(v) for v in vals[i + 1]]
        assert q[0] == brute.mle(Vn, r1)
        assert q[1] == brute.mle(Vn, r2)
        # degree <= s_{i+1}: the interpolant through q(0..s) predicts V~ on the line
        s = len(r1)
        for tt in (s + 1, 12345):
            pt = [(a + tt * (b - a)) % P for a, b in zip(r1, r2)]
            assert brute.lagrange(q, tt) == brute.mle(Vn, pt)


# --- closed forms (Sec. 6.2.1) --------------------------------------------------------

def test_f2_output_is_sum_of_squares():
    rng = random.Random(11)
    for logn in (0, 1, 4, 8):
        lw, kinds = oracle.f2_layers(logn)
        c = oracle.Circuit(lw, kinds)
        x = [rng.randrange(1 << 16) for _ in range(1 << logn)]
        assert int(c.evaluate(x)[0][0]) == sum(v * v for v in x) % P
    # large values wrap mod p
    c = oracle.Circuit(*oracle.f2_layers(2))
    x = [P - 1, P - 2, 1 << 60, 5]
    assert int(c.evaluate(x)[0][0]) == sum(v * v for v in x) % P


def test_f0_output_is_four_times_distinct_count():
    rng = random.Random(12)
    for logn in (1, 3, 6):
        c = oracle.Circuit(*oracle.f0_layers(logn))
        x = [rng.choice([0, 0, 1, 2, 1000, P - 1]) for _ in range(1 << logn)]
        nz = sum(1 for v in x if v)
        assert int(c.evaluate(x)[0][0]) == 4 * nz % P


def test_matmult_output_is_product():
    rng = np.random.default_rng(13)
    for logn in (0, 1, 3):
        n = 1 << logn
        A = rng.integers(0, 1 << 10, (n, n))
        B = rng.integers(0, 1 << 10, (n, n))
        c = oracle.Circuit(*oracle.matmult_layers(logn))
        out = c.evaluate(np.concatenate([A.reshape(-1), B.reshape(-1)]))[0]
        assert (out.reshape(n, n).astype(np.int64) == A @ B).all()


# --- wiring predicates: generic sum vs closed-form products ------------------------------

def eq3(a, b, c):
    return (a * b % P * c + (1 - a) * (1 - b) % P * (1 - c)) % P


def closed_form(kind, si, sn, p, w1, w2):
    """add~, mult~ of the structured kinds as products of per-coordinate factors."""
    prod = lambda xs: __import__("functools").reduce(lambda u, v: u * v % P, xs, 1)
    if kind == oracle.SQUARE:
        return 0, prod(eq3(p[k], w1[k], w2[k]) for k in range(si))
    if kind == oracle.TREE:
        v = (1 - w1[0]) * w2[0] % P * prod(eq3(p[k], w1[k + 1], w2[k + 1]) for k in range(si))
        return v % P, 0
    if kind == oracle.F0_FIRST:
        base = prod(eq3(p[k + 1], w1[k], w2[k]) for k in range(sn))
        return p[0] * base % P, (1 - p[0]) * base % P
    if kind == oracle.F0_PAIR:
        v = brute.eq1(p[0], w1[0]) * (1 - w2[0]) % P * prod(eq3(p[k], w1[k], w2[k]) for k in range(1, si))
        return 0, v % P
    if kind == oracle.F0_FINAL:
        v = w1[0] * w2[0] % P * prod(eq3(p[k], w1[k + 1], w2[k + 1]) for k in range(si))
        return 0, v % P
    if kind == oracle.MATMULT:
        L = si // 3
        v = prod(eq3(p[b], w1[b], w2[L + b]) for b in range(L))
        v = v * prod(brute.eq1(p[L + b], w2[b]) for b in range(L)) % P
        v = v * prod(brute.eq1(p[2 * L + b], w1[L + b]) for b in range(L)) % P
        v = v * (1 - w1[2 * L]) % P * w2[2 * L] % P
        return 0, v
    raise ValueError(kind)


@pytest.mark.parametrize("kind,si,sn", [
    (oracle.SQUARE, 3, 3), (oracle.TREE, 2, 3), (oracle.TREE, 0, 1), (oracle.F0_FIRST, 3, 2),
    (oracle.F0_PAIR, 3, 3), (oracle.F0_FINAL, 2, 3), (oracle.MATMULT, 3, 3), (oracle.MATMULT, 6, 5)])
def test_wiring_closed_forms(kind, si, sn):
    c = oracle.Circuit([si, sn], [kind])
    rng = random.Random(kind * 100 + si)
    for _ in range(3):
        p = [rng.randrange(P) for _ in range(si)]
        w1 = [rng.randrange(P) for _ in range(sn)]
        w2 = [rng.randrange(P) for _ in range(sn)]
        assert c.wiring_eval(0, p, w1, w2) == closed_form(kind, si, sn, p, w1, w2)


# --- completeness and soundness ----------------------------------------------------------

@pytest.mark.parametrize("family,logn", [("f2", 6), ("f0", 3), ("matmult", 2)])
def test_honest_prover_accepted(family, logn):
    c = oracle.Circuit(*getattr(oracle, f"{family}_layers")(logn))
    rng = random.Random(14)
    x = [rng.randrange(1 << 16) for _ in range(c.n_inputs)]
    for seed in range(1, 9):
        assert c.verify(x, seed, c.prove(x, seed)) == (True, -1)


def test_tampering_rejected():
    c = oracle.Circuit(*oracle.f2_layers(5))
    rng = random.Random(15)
    x = [rng.randrange(1 << 16) for _ in range(c.n_inputs)]
    seed = 4
    t = c.prove(x, seed)
    L = len(t)
    # every single-element change of the transcript is caught
    for k in range(L):
        bad = t.copy()
        bad[k] = (int(bad[k]) + 1 + rng.randrange(P - 1)) % P
        assert c.verify(x, seed, bad)[0] is False, k
    # non-canonical transcript values are rejected
    bad = t.copy()
    bad[3] = P
    assert c.verify(x, seed, bad) == (False, -2)
    # a claim about different inputs is rejected
    y = list(x)
    y[7] = (y[7] + 1) % P
    assert c.verify(y, seed, t)[0] is False


def test_wrong_gate_value_rejected():
    """A prover whose evaluation has one wrong gate (at every layer in turn),
    with the layers above recomputed from it, is rejected at that layer."""
    c = oracle.Circuit(*oracle.f2_layers(4))
    rng = random.Random(16)
    x = [rng.randrange(1 << 16) for _ in range(c.n_inputs)]
    ty_all = [c.layer_gates(i) for i in range(c.d)]
    for layer in range(1, c.d):
        vals = [v.astype(object) for v in c.evaluate(x)]
        g = rng.randrange(len(vals[layer]))
        vals[layer][g] = (int(vals[layer][g]) + 1) % P
        for i in range(layer - 1, -1, -1):
            ty, a, b = ty_all[i]
            vals[i] = np.array([(int(vals[i + 1][a[k]]) * int(vals[i + 1][b[k]])) % P if ty[k]
                                else (int(vals[i + 1][a[k]]) + int(vals[i + 1][b[k]])) % P
                                for k in range(len(ty))], dtype=object)
        t = c.prove_values([np.array(v, dtype=np.uint64) for v in vals], seed=8)
        ok, where = c.verify(x, 8, t)
        assert not ok
        assert where == layer


def test_noncanonical_input_rejected_by_evaluate():
    c = oracle.Circuit(*oracle.f2_layers(2))
    with pytest.raises(ValueError):
        c.evaluate([1, 2, P, 3])


def test_f2_circuit_size_matches_the_paper_table():
    """The paper's results table prints the F2 circuit at 8.4 million input
    entries as 25.2 million gates (inputs counted).  The oracle's F2 layering
    (a squaring layer, then a binary addition tree) at n = 2^23 inputs has
    n + n + (n - 1) gates, which rounds to the printed figures."""
    import os
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_circuit_sizes.txt")):
        if line.strip() and not line.startswith("#"):
            name, inputs, gates = line.split()
            rows[name] = (float(inputs), float(gates))
    inputs, gates = rows["F2"]
    widths, kinds = oracle.f2_layers(23)
    assert round((1 << widths[-1]) / 1e5) == round(inputs / 1e5)
    assert round(sum(1 << s for s in widths) / 1e5) == round(gates / 1e5)


# --- pattern matching and the single-output MatMult check (Sec. 6.2.1) -----------

def _occurrences(text, pat):
    n, q = len(text), len(pat)
    return sum(all(int(text[i + j]) == int(pat[j]) for j in range(q)) for i in range(n - q + 1))


@pytest.mark.parametrize("a,b,seed", [(2, 0, 1), (2, 1, 2), (3, 1, 3), (5, 2, 4), (6, 3, 5), (7, 1, 6)])
def test_pattern_match_output_counts_occurrences(a, b, seed):
    """The circuit's output is 4 (n - occurrences), occurrences counted by
    brute force over every location of the text."""
    from paper_1202_1350_gb300 import inputs as I
    w, k, ex = oracle.pm_layers(a, b)
    c = oracle.Circuit(w, k, explicit=ex)
    n, q = 1 << a, 1 << b
    x = I.pm_inputs(a, b, seed)
    occ = _occurrences(x[:n], x[n:n + q])
    assert occ >= 1  # the planted copies
    assert int(c.evaluate(x)[0][0]) == 4 * (n - occ)
    # a text without the pattern anywhere: no occurrence
    y = x.copy()
    y[n:n + q] = 7  # a symbol outside the text's alphabet
    assert int(c.evaluate(y)[0][0]) == 4 * n


@pytest.mark.parametrize("logm,errors", [(1, 0), (2, 0), (2, 1), (2, 3), (3, 0), (3, 5)])
def test_matmult_check_output_counts_wrong_entries(logm, errors):
    """Output 4 #{(i, j) : (A B)_ij != C_ij}: zero exactly when C = A B."""
    from paper_1202_1350_gb300 import inputs as I
    w, k, ex = oracle.mm1_layers(logm)
    c = oracle.Circuit(w, k, explicit=ex)
    m = 1 << logm
    x = I.mm1_inputs(logm, 70 + logm, errors=errors)
    A = x[:m * m].astype(object).reshape(m, m)
    B = x[m * m:2 * m * m].astype(object).reshape(m, m)
    C = x[2 * m * m:3 * m * m].astype(object).reshape(m, m)
    wrong = int(((A.dot(B) - C) % P != 0).sum())
    assert wrong <= errors and (wrong > 0) == (errors > 0)
    assert int(c.evaluate(x)[0][0]) == 4 * wrong


@pytest.mark.parametrize("which", ["pm", "mm1"])
def test_pm_and_mm1_proofs_accepted_and_tampering_rejected(which):
    from paper_1202_1350_gb300 import inputs as I
    if which == "pm":
        w, k, ex = oracle.pm_layers(4, 2)
        x = I.pm_inputs(4, 2, 11)
    else:
        w, k, ex = oracle.mm1_layers(2)
        x = I.mm1_inputs(2, 12, errors=1)
    c = oracle.Circuit(w, k, explicit=ex)
    t = c.prove(x, 99)
    assert c.verify(x, 99, t)[0]
    bad = t.copy()
    bad[len(bad) // 2] = (int(bad[len(bad) // 2]) + 1) % P
    assert not c.verify(x, 99, bad)[0]


def test_pm_and_mm1_wiring_equals_the_packages_description():
    """The package describes these circuits with its own code; both
    descriptions must be the same circuit."""
    from paper_1202_1350_gb300 import circuits as C
    pairs = [(oracle.pm_layers(a, b), C.pattern_match(a, b)) for a, b in [(2, 0), (3, 2), (6, 3)]]
    pairs += [(oracle.mm1_layers(L), C.matmult_check(L)) for L in (1, 2, 3)]
    for (w1, k1, e1), (w2, k2, e2) in pairs:
        assert list(w1) == list(w2) and list(k1) == list(k2)
        for x, y in zip(e1, e2):
            assert (x is None) == (y is None)
            if x is not None:
                for u, v in zip(x, y):
                    assert np.array_equal(np.asarray(u, np.int64), np.asarray(v, np.int64))


# --- the special-purpose non-interactive F2 protocol (Sec. 3.2, 4.2, 6.3) ----------

def _sympy_coefficients(row, nodes):
    """Coefficients of the degree < h polynomial through (nodes[y], row[y]) by
    solving the Vandermonde system mod p with sympy's modular matrix inverse:
    an independent method (no Lagrange products)."""
    sympy = pytest.importorskip("sympy")
    h = len(row)
    V = sympy.Matrix(h, h, lambda y, j: pow(int(nodes[int(y)]), int(j), P))
    c = V.inv_mod(P) * sympy.Matrix([int(t) for t in row])
    return [int(t) % P for t in c]


def test_f2sp_nodes_form_subgroups():
    """37 generates F_p^* (sympy); u = 37^((p-1)/(2h)) has order exactly 2h,
    so the nodes u^(2y) are the h distinct elements of the subgroup of order h
    and the proof points u^k those of the subgroup of order 2h; an h that does
    not divide (p - 1) / 2 is refused."""
    sympy = pytest.importorskip("sympy")
    assert sympy.is_primitive_root(oracle.F2SP_GENERATOR, P)
    for h in (1, 3, 5, 7, 9, 15, 21, 45, 1001, 5005):
        u = oracle.f2sp_root(h)
        assert pow(u, 2 * h, P) == 1 and pow(u, h, P) == P - 1
        assert sympy.n_order(u, P) == 2 * h
    for h in (2, 4, 8, 1024, 17):
        with pytest.raises(ValueError):
            oracle.f2sp_prove(np.zeros(h, np.uint64), 1, h)


@pytest.mark.parametrize("v,h,seed", [(1, 1, 1), (1, 3, 2), (2, 3, 3), (4, 5, 4), (3, 7, 5), (2, 9, 6), (2, 15, 7)])
def test_f2sp_proof_against_sympy_interpolation(v, h, seed):
    """s(u^k) = sum_x f_x(u^k)^2 with f_x's coefficients from a modular
    Vandermonde solve (sympy); at the nodes (k even) s is the column's sum of
    squares, and the even points sum to F2."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 1000, v * h).astype(np.uint64)
    proof = oracle.f2sp_prove(a, v, h)
    assert len(proof) == 2 * h
    u = oracle.f2sp_root(h)
    nodes = [pow(u, 2 * y, P) for y in range(h)]
    coeffs = [_sympy_coefficients(a[x * h:(x + 1) * h], nodes) for x in range(v)]
    for k in range(2 * h):
        pt = pow(u, k, P)
        want = sum(sum(c * pow(pt, j, P) for j, c in enumerate(cs)) ** 2 for cs in coeffs) % P
        assert int(proof[k]) == want
    grid = a.astype(object).reshape(v, h)
    for y in range(h):
        assert int(proof[2 * y]) == int((grid[:, y] ** 2).sum()) % P
    assert sum(int(t) for t in proof[0::2]) % P == int((grid ** 2).sum()) % P


@pytest.mark.parametrize("v,h", [(1, 1), (5, 3), (16, 15), (10, 33)])
def test_f2sp_complete_and_sound(v, h):
    rng = np.random.default_rng(v * 100 + h)
    a = rng.integers(0, 1 << 16, v * h).astype(np.uint64)
    proof = oracle.f2sp_prove(a, v, h)
    f2 = int((a.astype(object) ** 2).sum()) % P
    for seed in range(1, 9):
        assert oracle.f2sp_verify(a, v, h, seed, proof) == (True, f2)
    for m in range(len(proof)):  # every single-entry change
        bad = proof.copy()
        bad[m] = (int(bad[m]) + 1 + m) % P
        assert not oracle.f2sp_verify(a, v, h, 3, bad)[0]
    bad = proof.copy()
    bad[0] = P  # a non-canonical entry is a rejection
    assert not oracle.f2sp_verify(a, v, h, 3, bad)[0]
    # a different input is caught by the verifier's secret point
    b = a.copy()
    b[len(b) // 2] += np.uint64(1)
    assert not oracle.f2sp_verify(b, v, h, 3, proof)[0]
