/*
 * vc_oracle.c -- plain CPU oracle for the GKR/CMT interactive proof for layered
 * arithmetic circuits over F_p, p = 2^61 - 1.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this library.  It shares no source, header, table or
 * helper with the CUDA path, and the CUDA path never calls it.
 *
 * Everything here is deliberately slow and written to be checked against the
 * paper by eye: field products use a 128-bit product and the C `%` operator,
 * eq() and multilinear extensions are direct products and sums, and there is no
 * blocking, fusion or reordering.
 *
 * Paper: Thaler, Roberts, Mitzenmacher, Pfister, "Verifiable Computation with
 * Massively Parallel Interactive Proofs".
 *   Sec. 3.1   GKR protocol: layered fan-in-2 ADD/MULT circuit, one iteration
 *              per layer, each iteration touches two adjacent layers, prover
 *              messages are polynomials given by evaluations, challenges are
 *              random field elements.
 *   Sec. 4.1.1 each gate contributes independently to every prover message;
 *              the message is the field sum of the contributions.
 *   Sec. 4.1.2 / Sec. 2.2  the verifier's secret is one symbol of the
 *              low-degree-extension encoding of the input (the input's
 *              multilinear extension at a random point).
 *   Sec. 5.1.4 contribution of gate g depends on g, its in-neighbour indices and
 *              in-neighbour values; binary-tree wiring in1 = 2g, in2 = 2g+1.
 *   Sec. 6.1   field F_p with p = 2^61 - 1.
 *   Sec. 6.2.1 benchmark circuits F2, F0 (Fermat: a^(p-1) = 1 iff a != 0),
 *              MatMult.
 *
 * The paper defers the protocol's exact definition to GKR and CMT.  Readings
 * taken here (each also listed in the design notes):
 *   - layer 0 is the output layer, layer d the input layer; layer i has
 *     S_i = 2^{s_i} gates;
 *   - multilinear coordinate x_k corresponds to bit (k-1) of a gate index;
 *   - the identity proved at layer i is
 *       V~_i(z) = sum_{p, w1, w2} eq(z,p) [ add~_i(p,w1,w2) (V~_{i+1}(w1) + V~_{i+1}(w2))
 *                                         + mult~_i(p,w1,w2) V~_{i+1}(w1) V~_{i+1}(w2) ]
 *     with the sum-check variables bound in the order p_1..p_{s_i},
 *     w1_1..w1_{s_{i+1}}, w2_1..w2_{s_{i+1}};
 *   - each round message is a degree-2 polynomial sent as its values at 0,1,2;
 *   - two claims about V~_{i+1} are reduced to one along the line
 *     l(t) = r1 + t (r2 - r1): the prover sends q(t) = V~_{i+1}(l(t)) at
 *     t = 0..s_{i+1}, the verifier draws tau and continues with z = l(tau);
 *   - challenges come from splitmix64 seeded with the proof seed: x = next()>>3,
 *     redrawn while x == p; order: s_0 output coordinates, then per layer the
 *     round challenges in round order, then tau;
 *   - transcript = [S_0 outputs] ++ per layer [3 values per round] ++ [q(0..s_{i+1})].
 *
 * The splitmix64 stream (a convention; the paper fixes no generator) is
 * pinned to the generator's published known-answer values.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t fe;
typedef unsigned __int128 u128;

#define OR_P ((((uint64_t)1) << 61) - 1)

/* ------------------------------------------------------------------------- */
/* Field F_p, p = 2^61 - 1 (Sec. 6.1).  Plain 128-bit arithmetic and `%`.     */
/* ------------------------------------------------------------------------- */

fe or_add(fe a, fe b) { return (fe)(((u128)a + (u128)b) % OR_P); }
fe or_sub(fe a, fe b) { return (fe)(((u128)a + (u128)OR_P - (u128)(b % OR_P)) % OR_P); }
fe or_mul(fe a, fe b) { return (fe)(((u128)a * (u128)b) % OR_P); }

fe or_pow(fe a, uint64_t e)
{
    fe r = 1, b = a % OR_P;
    while (e) {
        if (e & 1) r = or_mul(r, b);
        b = or_mul(b, b);
        e >>= 1;
    }
    return r;
}

/* Fermat inverse a^(p-2); a must be nonzero. */
fe or_inv(fe a) { return or_pow(a, OR_P - 2); }

/* ------------------------------------------------------------------------- */
/* Seeded challenges: splitmix64 (Steele, Lea, Flood 2014), published form.   */
/* Sec. 3.1: the verifier's challenges are random field elements.            */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t state; } or_prg;

static uint64_t splitmix64_next(or_prg *g)
{
    uint64_t z;
    g->state += 0x9E3779B97F4A7C15ULL;
    z = g->state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static fe draw_fe(or_prg *g)
{
    for (;;) {
        uint64_t x = splitmix64_next(g) >> 3;
        if (x != OR_P) return x;
    }
}

/* Raw access for tests of the generator itself. */
uint64_t or_splitmix64(uint64_t seed, uint64_t count, uint64_t *out)
{
    or_prg g = { seed };
    for (uint64_t i = 0; i < count; i++) out[i] = splitmix64_next(&g);
    return g.state;
}

void or_draw_challenges(uint64_t seed, uint64_t count, fe *out)
{
    or_prg g = { seed };
    for (uint64_t i = 0; i < count; i++) out[i] = draw_fe(&g);
}

/* ------------------------------------------------------------------------- */
/* eq and multilinear extensions, written out as their definitions.          */
/* ------------------------------------------------------------------------- */

/* eq(x, b) = prod_k (x_k b_k + (1 - x_k)(1 - b_k)) for field vectors x, y. */
static fe eq_pts(const fe *x, const fe *y, int n)
{
    fe r = 1;
    for (int k = 0; k < n; k++) {
        fe t = or_add(or_mul(x[k], y[k]),
                      or_mul(or_sub(1, x[k]), or_sub(1, y[k])));
        r = or_mul(r, t);
    }
    return r;
}

/* eq(x, bits of b) with coordinate k <-> bit k of the index. */
static fe eq_bits(const fe *x, uint64_t b, int n)
{
    fe r = 1;
    for (int k = 0; k < n; k++)
        r = or_mul(r, ((b >> k) & 1) ? x[k] : or_sub(1, x[k]));
    return r;
}

/* Multilinear extension V~(x) = sum_b eq(x, b) V[b] over {0,1}^n (direct sum). */
fe or_mle(const fe *V, int n, const fe *x)
{
    fe acc = 0;
    uint64_t S = (uint64_t)1 << n;
    for (uint64_t b = 0; b < S; b++)
        acc = or_add(acc, or_mul(eq_bits(x, b, n), V[b]));
    return acc;
}

fe or_eq(const fe *x, const fe *y, int n) { return eq_pts(x, y, n); }

/* ------------------------------------------------------------------------- */
/* Layered arithmetic circuits (Sec. 3.1, Sec. 5.1.4, Sec. 6.2.1).            */
/* ------------------------------------------------------------------------- */

enum {
    OR_SQUARE = 0,   /* gate g = MUL(g, g); s_i = s_{i+1}                     */
    OR_TREE = 1,     /* gate g = ADD(2g, 2g+1); s_{i+1} = s_i + 1 (Sec. 5.1.4)*/
    OR_MATMULT = 2,  /* gate (i,j,k) = A[i][k] * B[k][j]; s_i = 3L, s_{i+1} = 2L+1 */
    OR_F0_FIRST = 3, /* gate 2j = MUL(j,j), 2j+1 = ADD(j,j); s_i = s_{i+1} + 1 */
    OR_F0_PAIR = 4,  /* gate 2j = MUL(2j,2j), 2j+1 = MUL(2j+1,2j); s_i = s_{i+1} */
    OR_F0_FINAL = 5, /* gate j = MUL(2j+1, 2j+1); s_i = s_{i+1} - 1            */
    OR_EXPLICIT = 6  /* gate arrays given by the caller                      */
};

typedef struct {
    int d;            /* layers 0..d; 0 = output, d = input */
    int *s;           /* s[0..d] */
    uint8_t **type;   /* type[i][g] for i < d: 0 = ADD, 1 = MUL */
    uint32_t **in1;   /* in-neighbours of layer-i gates, in layer i+1 */
    uint32_t **in2;
} or_circuit;

void or_circuit_free(or_circuit *c)
{
    if (!c) return;
    for (int i = 0; i < c->d; i++) {
        free(c->type[i]);
        free(c->in1[i]);
        free(c->in2[i]);
    }
    free(c->type);
    free(c->in1);
    free(c->in2);
    free(c->s);
    free(c);
}

/*
 * Build an explicit circuit from a layer description.  kind[i] says how layer
 * i is wired to layer i+1; for OR_EXPLICIT, ex_type/ex_in1/ex_in2 give the gate
 * arrays of that layer (other entries may be NULL).  Returns NULL if a layer's
 * widths do not fit its kind or an explicit in-neighbour is out of range.
 */
or_circuit *or_circuit_new(int d, const uint32_t *log_width, const uint32_t *kind,
                           const uint8_t *const *ex_type,
                           const uint32_t *const *ex_in1,
                           const uint32_t *const *ex_in2)
{
    if (d < 1 || d > 4096) return NULL;
    for (int i = 0; i <= d; i++)
        if (log_width[i] > 30) return NULL;
    or_circuit *c = (or_circuit *)calloc(1, sizeof(or_circuit));
    c->d = d;
    c->s = (int *)malloc(sizeof(int) * (size_t)(d + 1));
    for (int i = 0; i <= d; i++) c->s[i] = (int)log_width[i];
    c->type = (uint8_t **)calloc((size_t)d, sizeof(uint8_t *));
    c->in1 = (uint32_t **)calloc((size_t)d, sizeof(uint32_t *));
    c->in2 = (uint32_t **)calloc((size_t)d, sizeof(uint32_t *));
    for (int i = 0; i < d; i++) {
        int si = c->s[i], sn = c->s[i + 1];
        uint64_t S = (uint64_t)1 << si, Sn = (uint64_t)1 << sn;
        c->type[i] = (uint8_t *)malloc(S);
        c->in1[i] = (uint32_t *)malloc(S * 4);
        c->in2[i] = (uint32_t *)malloc(S * 4);
        uint8_t *ty = c->type[i];
        uint32_t *a = c->in1[i], *b = c->in2[i];
        int ok = 1;
        switch (kind[i]) {
        case OR_SQUARE:
            ok = (si == sn);
            for (uint64_t g = 0; ok && g < S; g++) { ty[g] = 1; a[g] = (uint32_t)g; b[g] = (uint32_t)g; }
            break;
        case OR_TREE:
            ok = (sn == si + 1);
            for (uint64_t g = 0; ok && g < S; g++) { ty[g] = 0; a[g] = (uint32_t)(2 * g); b[g] = (uint32_t)(2 * g + 1); }
            break;
        case OR_MATMULT: {
            /* A[i][k] is input i*n + k, B[k][j] is input n^2 + k*n + j;
               gate index = k + n*j + n^2*i computes A[i][k] * B[k][j]. */
            int L = si / 3;
            ok = (si % 3 == 0) && (sn == 2 * L + 1);
            uint64_t n = (uint64_t)1 << L;
            for (uint64_t g = 0; ok && g < S; g++) {
                uint64_t k = g % n, j = (g / n) % n, ii = g / (n * n);
                ty[g] = 1;
                a[g] = (uint32_t)(ii * n + k);
                b[g] = (uint32_t)(n * n + k * n + j);
            }
            break;
        }
        case OR_F0_FIRST:
            ok = (si == sn + 1);
            for (uint64_t g = 0; ok && g < S; g++) {
                ty[g] = (g % 2 == 0) ? 1 : 0;
                a[g] = (uint32_t)(g / 2);
                b[g] = (uint32_t)(g / 2);
            }
            break;
        case OR_F0_PAIR:
            ok = (si == sn) && si >= 1;
            for (uint64_t g = 0; ok && g < S; g++) {
                ty[g] = 1;
                a[g] = (uint32_t)g;
                b[g] = (uint32_t)(g - (g % 2));
            }
            break;
        case OR_F0_FINAL:
            ok = (sn == si + 1);
            for (uint64_t g = 0; ok && g < S; g++) {
                ty[g] = 1;
                a[g] = (uint32_t)(2 * g + 1);
                b[g] = (uint32_t)(2 * g + 1);
            }
            break;
        case OR_EXPLICIT:
            ok = ex_type && ex_in1 && ex_in2 && ex_type[i] && ex_in1[i] && ex_in2[i];
            for (uint64_t g = 0; ok && g < S; g++) {
                ty[g] = ex_type[i][g];
                a[g] = ex_in1[i][g];
                b[g] = ex_in2[i][g];
                if (ty[g] > 1 || a[g] >= Sn || b[g] >= Sn) ok = 0;
            }
            break;
        default:
            ok = 0;
        }
        if (!ok) { or_circuit_free(c); return NULL; }
    }
    return c;
}

int or_circuit_depth(const or_circuit *c) { return c->d; }

/* Export the expanded gate arrays of layer i (for cross-checks in tests). */
void or_circuit_layer(const or_circuit *c, int i, uint8_t *type, uint32_t *in1, uint32_t *in2)
{
    uint64_t S = (uint64_t)1 << c->s[i];
    memcpy(type, c->type[i], S);
    memcpy(in1, c->in1[i], S * 4);
    memcpy(in2, c->in2[i], S * 4);
}

static uint64_t rounds_of(const or_circuit *c, int i) { return (uint64_t)c->s[i] + 2 * (uint64_t)c->s[i + 1]; }

uint64_t or_transcript_len(const or_circuit *c)
{
    uint64_t n = (uint64_t)1 << c->s[0];
    for (int i = 0; i < c->d; i++) n += 3 * rounds_of(c, i) + (uint64_t)c->s[i + 1] + 1;
    return n;
}

uint64_t or_num_challenges(const or_circuit *c)
{
    uint64_t n = (uint64_t)c->s[0];
    for (int i = 0; i < c->d; i++) n += rounds_of(c, i) + 1;
    return n;
}

/* Layer values live in one flat array: layer i starts at or_layer_offset(c, i). */
uint64_t or_layer_offset(const or_circuit *c, int i)
{
    uint64_t off = 0;
    for (int k = 0; k < i; k++) off += (uint64_t)1 << c->s[k];
    return off;
}

uint64_t or_total_values(const or_circuit *c) { return or_layer_offset(c, c->d + 1); }

/*
 * Layer-by-layer evaluation from the input layer d up to the output layer 0
 * (Sec. 6.2.4 "the very first step of the prover's computation").
 * values: flat array of or_total_values(c) entries; layer d is filled from
 * `inputs`.  Returns 0, or -1 if an input is not a canonical field element.
 */
int or_evaluate(const or_circuit *c, const fe *inputs, fe *values)
{
    uint64_t Sd = (uint64_t)1 << c->s[c->d];
    fe *Vd = values + or_layer_offset(c, c->d);
    for (uint64_t g = 0; g < Sd; g++) {
        if (inputs[g] >= OR_P) return -1;
        Vd[g] = inputs[g];
    }
    for (int i = c->d - 1; i >= 0; i--) {
        fe *Vi = values + or_layer_offset(c, i);
        const fe *Vn = values + or_layer_offset(c, i + 1);
        uint64_t S = (uint64_t)1 << c->s[i];
        for (uint64_t g = 0; g < S; g++) {
            fe x = Vn[c->in1[i][g]], y = Vn[c->in2[i][g]];
            Vi[g] = c->type[i][g] ? or_mul(x, y) : or_add(x, y);
        }
    }
    return 0;
}

/* Gate function Phi_g(a, b): a + b for ADD, a * b for MUL. */
static fe phi(uint8_t type, fe a, fe b) { return type ? or_mul(a, b) : or_add(a, b); }

/* Degree-2 polynomial from its values at 0, 1, 2, evaluated at r:
   g(r) = g0 (r-1)(r-2)/2 - g1 r (r-2) + g2 r (r-1)/2. */
static fe interp3(fe g0, fe g1, fe g2, fe r)
{
    fe half = or_inv(2);
    fe rm1 = or_sub(r, 1), rm2 = or_sub(r, 2);
    fe t0 = or_mul(or_mul(g0, or_mul(rm1, rm2)), half);
    fe t1 = or_mul(g1, or_mul(r, rm2));
    fe t2 = or_mul(or_mul(g2, or_mul(r, rm1)), half);
    return or_add(or_sub(t0, t1), t2);
}

/* Polynomial given by its values q[0..n] at 0..n, evaluated at x (Lagrange). */
static fe lagrange(const fe *q, int n, fe x)
{
    fe acc = 0;
    for (int t = 0; t <= n; t++) {
        fe num = 1, den = 1;
        for (int u = 0; u <= n; u++) {
            if (u == t) continue;
            num = or_mul(num, or_sub(x, (fe)u));
            den = or_mul(den, or_sub((fe)t, (fe)u));
        }
        acc = or_add(acc, or_mul(q[t], or_mul(num, or_inv(den))));
    }
    return acc;
}

fe or_interp3(fe g0, fe g1, fe g2, fe r) { return interp3(g0, g1, g2, r); }
fe or_lagrange(const fe *q, int n, fe x) { return lagrange(q, n, x); }

/* Point on the line l(t) = r1 + t (r2 - r1). */
static void line_point(const fe *r1, const fe *r2, int n, fe t, fe *out)
{
    for (int k = 0; k < n; k++) out[k] = or_add(r1[k], or_mul(t, or_sub(r2[k], r1[k])));
}

/*
 * Generic wiring predicates at a point: add~_i(rP, r1, r2) and mult~_i(rP, r1, r2)
 * as sums over the gates of layer i of eq(rP,g) eq(r1,in1(g)) eq(r2,in2(g)).
 */
void or_wiring_eval(const or_circuit *c, int i, const fe *rP, const fe *r1, const fe *r2,
                    fe *add_out, fe *mult_out)
{
    uint64_t S = (uint64_t)1 << c->s[i];
    int si = c->s[i], sn = c->s[i + 1];
    fe add = 0, mult = 0;
    for (uint64_t g = 0; g < S; g++) {
        fe w = or_mul(eq_bits(rP, g, si),
                      or_mul(eq_bits(r1, c->in1[i][g], sn), eq_bits(r2, c->in2[i][g], sn)));
        if (c->type[i][g]) mult = or_add(mult, w);
        else add = or_add(add, w);
    }
    *add_out = add;
    *mult_out = mult;
}

/* ------------------------------------------------------------------------- */
/* Prover, form 1: gate-centric, straight from the definition (Sec. 4.1.1).   */
/* ------------------------------------------------------------------------- */

/*
 * Round message g_j(t) of the layer-i sum-check, as the sum over gates g of
 * layer i of their single contribution (Sec. 4.1.1: every gate contributes to
 * exactly one term of the sum).  `r` holds the j challenges already bound in
 * this layer.  With P, W1, W2 the partially bound points (Boolean suffixes set
 * to the gate's own index bits, which is the only suffix with nonzero eq):
 *   phase 1 (j < s_i):           eq(z,P) eq(P,g) Phi_g(V[in1], V[in2])
 *   phase 2 (ω1 variables):      eq(z,rP) eq(rP,g) eq(W1,in1) Phi_g(V~(W1), V[in2])
 *   phase 3 (ω2 variables):      eq(z,rP) eq(rP,g) eq(r1,in1) eq(W2,in2) Phi_g(V~(r1), V~(W2))
 * V~ at a partially bound point is a direct multilinear-extension sum.
 */
static fe message_gate_centric(const or_circuit *c, int i, const fe *V_i1, const fe *z,
                               const fe *r, int j, fe t)
{
    int si = c->s[i], sn = c->s[i + 1];
    uint64_t S = (uint64_t)1 << si;
    fe *P = (fe *)malloc(sizeof(fe) * (size_t)(si + 1));
    fe *W = (fe *)malloc(sizeof(fe) * (size_t)(sn + 1));
    fe acc = 0;
    for (uint64_t g = 0; g < S; g++) {
        uint32_t a = c->in1[i][g], b = c->in2[i][g];
        fe contrib;
        if (j < si) {
            for (int k = 0; k < si; k++)
                P[k] = (k < j) ? r[k] : (k == j) ? t : (fe)((g >> k) & 1);
            contrib = or_mul(eq_pts(z, P, si), eq_bits(P, g, si));
            contrib = or_mul(contrib, phi(c->type[i][g], V_i1[a], V_i1[b]));
        } else if (j < si + sn) {
            int jj = j - si;
            const fe *rP = r;
            for (int k = 0; k < sn; k++)
                W[k] = (k < jj) ? r[si + k] : (k == jj) ? t : (fe)((a >> k) & 1);
            contrib = or_mul(eq_pts(z, rP, si), eq_bits(rP, g, si));
            contrib = or_mul(contrib, eq_bits(W, a, sn));
            contrib = or_mul(contrib, phi(c->type[i][g], or_mle(V_i1, sn, W), V_i1[b]));
        } else {
            int jj = j - si - sn;
            const fe *rP = r, *r1 = r + si;
            for (int k = 0; k < sn; k++)
                W[k] = (k < jj) ? r[si + sn + k] : (k == jj) ? t : (fe)((b >> k) & 1);
            contrib = or_mul(eq_pts(z, rP, si), eq_bits(rP, g, si));
            contrib = or_mul(contrib, or_mul(eq_bits(r1, a, sn), eq_bits(W, b, sn)));
            contrib = or_mul(contrib, phi(c->type[i][g], or_mle(V_i1, sn, r1), or_mle(V_i1, sn, W)));
        }
        acc = or_add(acc, contrib);
    }
    free(P);
    free(W);
    return acc;
}

/* ------------------------------------------------------------------------- */
/* Prover, form 2: the textbook table-folding sum-check, layer by layer.      */
/* ------------------------------------------------------------------------- */

/* Fold a table of 2m entries with challenge r: T'[k] = T[2k] + r (T[2k+1] - T[2k]). */
static void fold(fe *T, uint64_t m, fe r)
{
    for (uint64_t k = 0; k < m; k++) T[k] = or_add(T[2 * k], or_mul(r, or_sub(T[2 * k + 1], T[2 * k])));
}

/* T(t, k) = T[2k] + t (T[2k+1] - T[2k]): the table's value with the current
   variable set to t and the rest to the bits of k. */
static fe at_t(const fe *T, uint64_t k, fe t) { return or_add(T[2 * k], or_mul(t, or_sub(T[2 * k + 1], T[2 * k]))); }

/* Multilinear extension by successive folding (the same value as or_mle). */
static fe mle_by_folding(const fe *V, int n, const fe *x)
{
    uint64_t S = (uint64_t)1 << n;
    fe *T = (fe *)malloc(sizeof(fe) * S);
    memcpy(T, V, sizeof(fe) * S);
    for (int k = 0; k < n; k++) fold(T, S >> (k + 1), x[k]);
    fe v = T[0];
    free(T);
    return v;
}

/* eq(x, .) over {0,1}^n by doubling: E[b + 2^k c] = E[b] * (c ? x_k : 1 - x_k). */
static fe *eq_table(const fe *x, int n)
{
    uint64_t S = (uint64_t)1 << n;
    fe *E = (fe *)malloc(sizeof(fe) * S);
    E[0] = 1;
    for (int k = 0; k < n; k++) {
        uint64_t h = (uint64_t)1 << k;
        for (uint64_t b = 0; b < h; b++) {
            E[b + h] = or_mul(E[b], x[k]);
            E[b] = or_mul(E[b], or_sub(1, x[k]));
        }
    }
    return E;
}

/*
 * One layer of the folding prover.  Writes 3 (s_i + 2 s_{i+1}) round values and
 * s_{i+1} + 1 line values to `out`, consumes challenges from g, and on return
 * z_next holds l(tau).  V_i1 is layer i+1.
 */
static void prove_layer_folding(const or_circuit *c, int i, const fe *V_i1, const fe *z,
                                or_prg *g, fe *out, fe *z_next)
{
    int si = c->s[i], sn = c->s[i + 1];
    uint64_t S = (uint64_t)1 << si, Sn = (uint64_t)1 << sn;
    fe *r = (fe *)malloc(sizeof(fe) * (size_t)(si + 2 * sn + 1));
    int pos = 0, j = 0;

    /* Phase 1: sum_p eq(z,p) C[p], C[p] = Phi_p(V[in1(p)], V[in2(p)]). */
    fe *E = eq_table(z, si);
    fe *C = (fe *)malloc(sizeof(fe) * S);
    for (uint64_t p = 0; p < S; p++) C[p] = phi(c->type[i][p], V_i1[c->in1[i][p]], V_i1[c->in2[i][p]]);
    for (int k = 0; k < si; k++, j++) {
        uint64_t m = S >> (k + 1);
        for (fe t = 0; t < 3; t++) {
            fe acc = 0;
            for (uint64_t q = 0; q < m; q++) acc = or_add(acc, or_mul(at_t(E, q, t), at_t(C, q, t)));
            out[pos++] = acc;
        }
        r[j] = draw_fe(g);
        fold(E, m, r[j]);
        fold(C, m, r[j]);
    }
    fe eq_z_rP = E[0]; /* eq(z, rP) */
    free(E);
    free(C);
    const fe *rP = r;

    /* Phase 2: weights w_g = eq(z,rP) eq(rP,g); tables over w1 (layer i+1):
       A1[w] = sum_{ADD g, in1=w} w_g, B1[w] = sum_{ADD g, in1=w} w_g V[in2],
       M1[w] = sum_{MUL g, in1=w} w_g V[in2]; message sum A1 V + B1 + M1 V. */
    fe *eqP = eq_table(rP, si);
    fe *w = (fe *)malloc(sizeof(fe) * S);
    for (uint64_t q = 0; q < S; q++) w[q] = or_mul(eq_z_rP, eqP[q]);
    free(eqP);
    fe *A1 = (fe *)calloc(Sn, sizeof(fe));
    fe *B1 = (fe *)calloc(Sn, sizeof(fe));
    fe *M1 = (fe *)calloc(Sn, sizeof(fe));
    for (uint64_t q = 0; q < S; q++) {
        uint32_t a = c->in1[i][q], b = c->in2[i][q];
        if (c->type[i][q]) {
            M1[a] = or_add(M1[a], or_mul(w[q], V_i1[b]));
        } else {
            A1[a] = or_add(A1[a], w[q]);
            B1[a] = or_add(B1[a], or_mul(w[q], V_i1[b]));
        }
    }
    fe *Vt = (fe *)malloc(sizeof(fe) * Sn);
    memcpy(Vt, V_i1, sizeof(fe) * Sn);
    for (int k = 0; k < sn; k++, j++) {
        uint64_t m = Sn >> (k + 1);
        for (fe t = 0; t < 3; t++) {
            fe acc = 0;
            for (uint64_t q = 0; q < m; q++) {
                fe v = at_t(Vt, q, t);
                acc = or_add(acc, or_mul(at_t(A1, q, t), v));
                acc = or_add(acc, at_t(B1, q, t));
                acc = or_add(acc, or_mul(at_t(M1, q, t), v));
            }
            out[pos++] = acc;
        }
        r[j] = draw_fe(g);
        fold(A1, m, r[j]);
        fold(B1, m, r[j]);
        fold(M1, m, r[j]);
        fold(Vt, m, r[j]);
    }
    fe v1 = Vt[0]; /* V~_{i+1}(r1) */
    free(A1);
    free(B1);
    free(M1);
    const fe *r1 = r + si;

    /* Phase 3: u_g = w_g eq(r1, in1(g)); A2[w] = sum_{ADD g, in2=w} u_g,
       M2[w] = sum_{MUL g, in2=w} u_g; message sum A2 (v1 + V) + M2 v1 V. */
    fe *eq1 = eq_table(r1, sn);
    fe *A2 = (fe *)calloc(Sn, sizeof(fe));
    fe *M2 = (fe *)calloc(Sn, sizeof(fe));
    for (uint64_t q = 0; q < S; q++) {
        uint32_t a = c->in1[i][q], b = c->in2[i][q];
        fe u = or_mul(w[q], eq1[a]);
        if (c->type[i][q]) M2[b] = or_add(M2[b], u);
        else A2[b] = or_add(A2[b], u);
    }
    free(eq1);
    free(w);
    memcpy(Vt, V_i1, sizeof(fe) * Sn);
    for (int k = 0; k < sn; k++, j++) {
        uint64_t m = Sn >> (k + 1);
        for (fe t = 0; t < 3; t++) {
            fe acc = 0;
            for (uint64_t q = 0; q < m; q++) {
                fe v = at_t(Vt, q, t);
                acc = or_add(acc, or_mul(at_t(A2, q, t), or_add(v1, v)));
                acc = or_add(acc, or_mul(at_t(M2, q, t), or_mul(v1, v)));
            }
            out[pos++] = acc;
        }
        r[j] = draw_fe(g);
        fold(A2, m, r[j]);
        fold(M2, m, r[j]);
        fold(Vt, m, r[j]);
    }
    free(A2);
    free(M2);
    free(Vt);
    const fe *r2 = r + si + sn;

    /* Line reduction: q(t) = V~_{i+1}(l(t)) for t = 0..s_{i+1}. */
    fe *pt = (fe *)malloc(sizeof(fe) * (size_t)(sn + 1));
    for (int t = 0; t <= sn; t++) {
        line_point(r1, r2, sn, (fe)t, pt);
        out[pos++] = mle_by_folding(V_i1, sn, pt);
    }
    fe tau = draw_fe(g);
    line_point(r1, r2, sn, tau, z_next);
    free(pt);
    free(r);
}

/* Same layer, gate-centric form (form 1): identical output by definition. */
static void prove_layer_gate_centric(const or_circuit *c, int i, const fe *V_i1, const fe *z,
                                     or_prg *g, fe *out, fe *z_next)
{
    int si = c->s[i], sn = c->s[i + 1];
    int n = si + 2 * sn;
    fe *r = (fe *)malloc(sizeof(fe) * (size_t)(n + 1));
    int pos = 0;
    for (int j = 0; j < n; j++) {
        for (fe t = 0; t < 3; t++) out[pos++] = message_gate_centric(c, i, V_i1, z, r, j, t);
        r[j] = draw_fe(g);
    }
    const fe *r1 = r + si, *r2 = r + si + sn;
    fe *pt = (fe *)malloc(sizeof(fe) * (size_t)(sn + 1));
    for (int t = 0; t <= sn; t++) {
        line_point(r1, r2, sn, (fe)t, pt);
        out[pos++] = or_mle(V_i1, sn, pt);
    }
    fe tau = draw_fe(g);
    line_point(r1, r2, sn, tau, z_next);
    free(pt);
    free(r);
}

/*
 * Prove from given layer values (flat, as or_evaluate writes them).  Taking the
 * values as an argument lets tests run a prover whose evaluation is wrong.
 * form = 1: gate-centric definition; form = 2: table folding.
 */
int or_prove_values(const or_circuit *c, const fe *values, uint64_t seed, int form, fe *transcript)
{
    or_prg g = { seed };
    uint64_t S0 = (uint64_t)1 << c->s[0];
    int smax = 0;
    for (int i = 0; i <= c->d; i++) if (c->s[i] > smax) smax = c->s[i];
    fe *z = (fe *)malloc(sizeof(fe) * (size_t)(smax + 1));
    fe *zn = (fe *)malloc(sizeof(fe) * (size_t)(smax + 1));
    uint64_t pos = 0;
    for (uint64_t b = 0; b < S0; b++) transcript[pos++] = values[b];
    for (int k = 0; k < c->s[0]; k++) z[k] = draw_fe(&g);
    for (int i = 0; i < c->d; i++) {
        const fe *V_i1 = values + or_layer_offset(c, i + 1);
        if (form == 1) prove_layer_gate_centric(c, i, V_i1, z, &g, transcript + pos, zn);
        else prove_layer_folding(c, i, V_i1, z, &g, transcript + pos, zn);
        pos += 3 * rounds_of(c, i) + (uint64_t)c->s[i + 1] + 1;
        memcpy(z, zn, sizeof(fe) * (size_t)c->s[i + 1]);
    }
    free(z);
    free(zn);
    return 0;
}

/* Evaluate, then prove.  Returns -1 on a non-canonical input. */
int or_prove(const or_circuit *c, const fe *inputs, uint64_t seed, int form, fe *transcript)
{
    fe *values = (fe *)malloc(sizeof(fe) * or_total_values(c));
    if (or_evaluate(c, inputs, values) != 0) { free(values); return -1; }
    or_prove_values(c, values, seed, form, transcript);
    free(values);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Verifier (Sec. 2.2, Sec. 3.1, Sec. 4.1.2).                                 */
/* ------------------------------------------------------------------------- */

/*
 * Returns 1 (accept) or 0 (reject).  Per round: g(0) + g(1) must equal the
 * running claim, the claim becomes g(r).  End of layer i: the claim must equal
 * eq(z, rP) [add~(rP,r1,r2) (q(0) + q(1)) + mult~(rP,r1,r2) q(0) q(1)], then
 * z = l(tau) and the claim becomes q(tau).  Last: the claim must equal the
 * input's multilinear extension at z (the verifier's secret).
 * If fail_layer is not NULL it receives the layer whose check failed (-1 if
 * none, d for the final input check, -2 for a non-canonical value).
 */
int or_verify(const or_circuit *c, const fe *inputs, uint64_t seed, const fe *transcript,
              int *fail_layer)
{
    or_prg g = { seed };
    int smax = 0;
    for (int i = 0; i <= c->d; i++) if (c->s[i] > smax) smax = c->s[i];
    fe *z = (fe *)malloc(sizeof(fe) * (size_t)(smax + 1));
    fe *r = (fe *)malloc(sizeof(fe) * (size_t)(3 * smax + 1));
    int ok = 1, where = -1;
    uint64_t L = or_transcript_len(c);
    for (uint64_t k = 0; k < L; k++)
        if (transcript[k] >= OR_P) { ok = 0; where = -2; }
    uint64_t S0 = (uint64_t)1 << c->s[0], pos = S0;
    for (int k = 0; k < c->s[0]; k++) z[k] = draw_fe(&g);
    fe claim = ok ? or_mle(transcript, c->s[0], z) : 0;
    for (int i = 0; ok && i < c->d; i++) {
        int si = c->s[i], sn = c->s[i + 1], n = si + 2 * sn;
        for (int j = 0; j < n; j++) {
            fe g0 = transcript[pos], g1 = transcript[pos + 1], g2 = transcript[pos + 2];
            pos += 3;
            if (or_add(g0, g1) != claim) { ok = 0; where = i; }
            r[j] = draw_fe(&g);
            claim = interp3(g0, g1, g2, r[j]);
        }
        const fe *q = transcript + pos;
        pos += (uint64_t)sn + 1;
        const fe *rP = r, *r1 = r + si, *r2 = r + si + sn;
        fe add, mult;
        or_wiring_eval(c, i, rP, r1, r2, &add, &mult);
        /* q(0) = V~(r1), q(1) = V~(r2); with s_{i+1} = 0 the line is a single
           point and q has the one value q(0) = V~(r1) = V~(r2). */
        fe v1 = q[0], v2 = (sn >= 1) ? q[1] : q[0];
        fe expect = or_mul(eq_pts(z, rP, si),
                           or_add(or_mul(add, or_add(v1, v2)), or_mul(mult, or_mul(v1, v2))));
        if (ok && expect != claim) { ok = 0; where = i; }
        fe tau = draw_fe(&g);
        line_point(r1, r2, sn, tau, z);
        claim = lagrange(q, sn, tau);
    }
    if (ok) {
        for (uint64_t b = 0; b < ((uint64_t)1 << c->s[c->d]); b++)
            if (inputs[b] >= OR_P) { ok = 0; where = -2; }
    }
    if (ok && or_mle(inputs, c->s[c->d], z) != claim) { ok = 0; where = c->d; }
    free(z);
    free(r);
    if (fail_layer) *fail_layer = ok ? -1 : where;
    return ok;
}

/* ------------------------------------------------------------------------- */
/* Special-purpose non-interactive F2 protocol (Sec. 3.2 outline, Sec. 4.2,   */
/* Sec. 6.3; the protocol of Chakrabarti et al. as implemented by CMT).       */
/*                                                                           */
/* The frequency vector a (n = v h entries) is a v x h grid, a(x, y) at      */
/* x h + y.  Row x is extended by the polynomial f_x of degree < h that      */
/* takes the value a(x, y) at the node w^y, y = 0..h-1, where w generates    */
/* the subgroup of order h of F_p^*.  The proof is the polynomial            */
/* s(Y) = sum_x f_x(Y)^2 (degree <= 2h - 2) given by its values at the 2h    */
/* points u^k, k = 0..2h-1, where u generates the subgroup of order 2h and   */
/* u^2 = w (so the even points are the nodes).  The verifier keeps f_x(r)    */
/* for a secret random r (one value per row, v words), accepts iff           */
/* s(r) = sum_x f_x(r)^2, and reads F2 = sum_x sum_y a(x,y)^2 =              */
/* sum_{k even} s(u^k).  Readings: the nodes form a multiplicative subgroup  */
/* (the paper's prover runs the Prime Factor FFT on each row, which needs    */
/* points of smooth multiplicative order, Sec. 4.2 and 5.2), so h must       */
/* divide (p - 1) / 2; u = 37^((p-1)/(2h)) with 37 the least primitive root  */
/* of p; r is challenge 0 of the seed's stream (the coins of the GKR part).  */
/*                                                                           */
/* Everything below is the definition: Lagrange basis values as products    */
/* over the node sets, no FFT, no barycentric shortcut.                      */
/* ------------------------------------------------------------------------- */

#define OR_F2SP_GEN 37u

/* u = 37^((p-1)/(2h)), a generator of the subgroup of order 2h; 0 if 2h does
 * not divide p - 1. */
static fe f2sp_root(uint64_t h)
{
    if (h == 0 || (OR_P - 1) % (2 * h) != 0) return 0;
    return or_pow(OR_F2SP_GEN, (OR_P - 1) / (2 * h));
}

/* L_y(m) over the nodes pts[0..k-1]: prod_{j != y} (m - pts[j]) / (pts[y] - pts[j]). */
static fe lagrange_basis(const fe *pts, uint64_t k, uint64_t y, fe m)
{
    fe num = 1, den = 1;
    for (uint64_t j = 0; j < k; j++) {
        if (j == y) continue;
        num = or_mul(num, or_sub(m, pts[j]));
        den = or_mul(den, or_sub(pts[y], pts[j]));
    }
    return or_mul(num, or_inv(den));
}

/* Value at m of the polynomial through (pts[j], vals[j]), j = 0..k-1. */
static fe lagrange_eval(const fe *pts, const fe *vals, uint64_t k, fe m)
{
    fe s = 0;
    for (uint64_t y = 0; y < k; y++) s = or_add(s, or_mul(vals[y], lagrange_basis(pts, k, y, m)));
    return s;
}

/* nodes[y] = u^(2y), y < h; points[k] = u^k, k < 2h. */
static void f2sp_points(fe u, uint64_t h, fe *nodes, fe *points)
{
    fe t = 1;
    for (uint64_t k = 0; k < 2 * h; k++) {
        points[k] = t;
        if (k % 2 == 0) nodes[k / 2] = t;
        t = or_mul(t, u);
    }
}

/* Prover: proof[k] = s(u^k) for k = 0..2h-1.  Returns -1 for a non-canonical
 * entry of a, or for h = 0 or h not dividing (p - 1) / 2. */
int or_f2sp_prove(const fe *a, uint64_t v, uint64_t h, fe *proof)
{
    const fe u = f2sp_root(h);
    if (!u) return -1;
    for (uint64_t i = 0; i < v * h; i++)
        if (a[i] >= OR_P) return -1;
    const uint64_t np = 2 * h;
    fe *nodes = (fe *)malloc(sizeof(fe) * h), *points = (fe *)malloc(sizeof(fe) * np);
    f2sp_points(u, h, nodes, points);
    fe *L = (fe *)malloc(sizeof(fe) * h * np); /* L[k h + y] = L_y(u^k) */
    for (uint64_t k = 0; k < np; k++)
        for (uint64_t y = 0; y < h; y++) L[k * h + y] = lagrange_basis(nodes, h, y, points[k]);
    for (uint64_t k = 0; k < np; k++) proof[k] = 0;
    for (uint64_t x = 0; x < v; x++) {
        const fe *row = a + x * h;
        for (uint64_t k = 0; k < np; k++) {
            fe f = 0;
            for (uint64_t y = 0; y < h; y++) f = or_add(f, or_mul(row[y], L[k * h + y]));
            proof[k] = or_add(proof[k], or_mul(f, f));
        }
    }
    free(L);
    free(nodes);
    free(points);
    return 0;
}

/* Verifier: r from the seed; f_x(r) for every row; s(r) from the proof by
 * Lagrange interpolation over the 2h points.  Returns 1 (accept) or 0, and the
 * answer sum_{k even} proof[k] in *f2; -1 for a non-canonical entry of a, or
 * an h the prover rejects.  A proof entry >= p is a rejection. */
int or_f2sp_verify(const fe *a, uint64_t v, uint64_t h, uint64_t seed, const fe *proof, fe *f2)
{
    const fe u = f2sp_root(h);
    if (!u) return -1;
    for (uint64_t i = 0; i < v * h; i++)
        if (a[i] >= OR_P) return -1;
    const uint64_t np = 2 * h;
    for (uint64_t k = 0; k < np; k++)
        if (proof[k] >= OR_P) return 0;
    fe *nodes = (fe *)malloc(sizeof(fe) * h), *points = (fe *)malloc(sizeof(fe) * np);
    f2sp_points(u, h, nodes, points);
    fe r;
    or_draw_challenges(seed, 1, &r);
    fe lhs = 0;
    for (uint64_t x = 0; x < v; x++) {
        const fe fr = lagrange_eval(nodes, a + x * h, h, r);
        lhs = or_add(lhs, or_mul(fr, fr));
    }
    const fe rhs = lagrange_eval(points, proof, np, r);
    fe ans = 0;
    for (uint64_t k = 0; k < np; k += 2) ans = or_add(ans, proof[k]);
    *f2 = ans;
    free(nodes);
    free(points);
    return lhs == rhs ? 1 : 0;
}
