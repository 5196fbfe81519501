"""CPU oracle for the GKR/CMT prover and verifier over F_p, p = 2^61 - 1.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA path in ``paper_1202_1350_gb300`` and never imports it.

The arithmetic lives in ``vc_oracle.c`` (plain C, 128-bit products and ``%``),
compiled with gcc into ``oracle/_build/liboracle.so`` and called through ctypes.
The circuit descriptions below are this package's own restatement of the
paper's benchmark circuits (Sec. 6.2.1): F2 (a squaring layer then a binary
addition tree), F0 (Fermat power x^(p-1) then a tree), MatMult (one layer of
n^3 products then a tree over the summation index), pattern matching and the
single-output MatMult check (both with the F0 subcircuit); and the
special-purpose non-interactive F2 protocol (a v x h grid, rows extended as
polynomials, the proof s(Y) = sum of squared row extensions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

P = (1 << 61) - 1

SQUARE, TREE, MATMULT, F0_FIRST, F0_PAIR, F0_FINAL, EXPLICIT = range(7)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no GPU involved); returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            fe = ctypes.c_uint64
            for name in ("or_add", "or_sub", "or_mul", "or_pow"):
                getattr(L, name).restype = fe
                getattr(L, name).argtypes = [fe, fe]
            L.or_inv.restype = fe
            L.or_inv.argtypes = [fe]
            L.or_splitmix64.restype = fe
            L.or_splitmix64.argtypes = [fe, fe, _u64p]
            L.or_draw_challenges.restype = None
            L.or_draw_challenges.argtypes = [fe, fe, _u64p]
            L.or_mle.restype = fe
            L.or_mle.argtypes = [_u64p, ctypes.c_int, _u64p]
            L.or_eq.restype = fe
            L.or_eq.argtypes = [_u64p, _u64p, ctypes.c_int]
            L.or_interp3.restype = fe
            L.or_interp3.argtypes = [fe, fe, fe, fe]
            L.or_lagrange.restype = fe
            L.or_lagrange.argtypes = [_u64p, ctypes.c_int, fe]
            L.or_circuit_new.restype = ctypes.c_void_p
            L.or_circuit_new.argtypes = [ctypes.c_int, _u32p, _u32p,
                                         ctypes.POINTER(_u8p), ctypes.POINTER(_u32p),
                                         ctypes.POINTER(_u32p)]
            L.or_circuit_free.restype = None
            L.or_circuit_free.argtypes = [ctypes.c_void_p]
            L.or_circuit_layer.restype = None
            L.or_circuit_layer.argtypes = [ctypes.c_void_p, ctypes.c_int, _u8p, _u32p, _u32p]
            for name in ("or_transcript_len", "or_num_challenges", "or_total_values"):
                getattr(L, name).restype = fe
                getattr(L, name).argtypes = [ctypes.c_void_p]
            L.or_layer_offset.restype = fe
            L.or_layer_offset.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.or_evaluate.restype = ctypes.c_int
            L.or_evaluate.argtypes = [ctypes.c_void_p, _u64p, _u64p]
            L.or_prove.restype = ctypes.c_int
            L.or_prove.argtypes = [ctypes.c_void_p, _u64p, fe, ctypes.c_int, _u64p]
            L.or_prove_values.restype = ctypes.c_int
            L.or_prove_values.argtypes = [ctypes.c_void_p, _u64p, fe, ctypes.c_int, _u64p]
            L.or_verify.restype = ctypes.c_int
            L.or_verify.argtypes = [ctypes.c_void_p, _u64p, fe, _u64p,
                                    ctypes.POINTER(ctypes.c_int)]
            L.or_f2sp_prove.restype = ctypes.c_int
            L.or_f2sp_prove.argtypes = [_u64p, fe, fe, _u64p]
            L.or_f2sp_verify.restype = ctypes.c_int
            L.or_f2sp_verify.argtypes = [_u64p, fe, fe, fe, _u64p, _u64p]
            L.or_wiring_eval.restype = None
            L.or_wiring_eval.argtypes = [ctypes.c_void_p, ctypes.c_int, _u64p, _u64p, _u64p,
                                         _u64p, _u64p]
            _lib = L
    return _lib


def _p64(a: np.ndarray):
    return a.ctypes.data_as(_u64p)


def _arr(x) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    return a


# --- field (Sec. 6.1) ----------------------------------------------------------

def fe_add(a, b): return lib().or_add(a, b)
def fe_sub(a, b): return lib().or_sub(a, b)
def fe_mul(a, b): return lib().or_mul(a, b)
def fe_pow(a, e): return lib().or_pow(a, e)
def fe_inv(a): return lib().or_inv(a)


def splitmix64(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    lib().or_splitmix64(seed, n, _p64(out))
    return out


def draw_challenges(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    lib().or_draw_challenges(seed, n, _p64(out))
    return out


def mle(values, point) -> int:
    v = _arr(values)
    x = _arr(point)
    n = len(x)
    assert len(v) == (1 << n)
    return lib().or_mle(_p64(v), n, _p64(x) if n else _p64(np.zeros(1, np.uint64)))


def eq(x, y) -> int:
    a, b = _arr(x), _arr(y)
    dummy = np.zeros(1, np.uint64)
    return lib().or_eq(_p64(a) if len(a) else _p64(dummy), _p64(b) if len(b) else _p64(dummy), len(a))


def interp3(g0, g1, g2, r) -> int:
    return lib().or_interp3(g0, g1, g2, r)


def lagrange(q, x) -> int:
    a = _arr(q)
    return lib().or_lagrange(_p64(a), len(a) - 1, x)


# --- circuits (Sec. 6.2.1) -------------------------------------------------------

def f2_layers(logn: int):
    """F2 = sum x_i^2: a squaring layer over n inputs, then logn addition layers."""
    log_width = list(range(0, logn + 1)) + [logn]
    kinds = [TREE] * logn + [SQUARE]
    return log_width, kinds


def f0_layers(logn: int):
    """4 * F0 = sum 4 x^(p-1) over n inputs.

    Layer E1 (width 2n) holds x^2 and 2x; layers E2..E60 square the first of
    each pair and multiply the second by it, so after E_k the pair is
    (x^(2^k), 2 x^(2^k - 1)); the last power layer squares the second:
    4 x^(2^61 - 2) = 4 x^(p-1), which is 4 for x != 0 and 0 for x = 0 (Fermat,
    Sec. 6.2.1).  Then logn addition layers.
    """
    tree_w = list(range(0, logn + 1))
    log_width = tree_w + [logn + 1] * 60 + [logn]
    kinds = [TREE] * logn + [F0_FINAL] + [F0_PAIR] * 59 + [F0_FIRST]
    return log_width, kinds


def matmult_layers(logn: int):
    """C = A B for n x n matrices: n^3 products, then logn addition layers over k."""
    L = logn
    log_width = [2 * L + j for j in range(0, L + 1)] + [2 * L + 1]
    kinds = [TREE] * L + [MATMULT]
    return log_width, kinds


# --- special-purpose non-interactive F2 protocol (Sec. 3.2, 4.2, 6.3) ------------

F2SP_GENERATOR = 37  # the least primitive root of p


def f2sp_root(h: int) -> int:
    """u = 37^((p-1)/(2h)): a generator of the subgroup of order 2h (h must
    divide (p - 1) / 2); the nodes are u^(2y), the proof points u^k."""
    if h <= 0 or (P - 1) % (2 * h):
        raise ValueError("h must divide (p - 1) / 2")
    return pow(F2SP_GENERATOR, (P - 1) // (2 * h), P)


def f2sp_prove(a, v: int, h: int) -> np.ndarray:
    """The proof of the special-purpose F2 protocol for the v x h grid a (row
    x at a[x h : x h + h]): s(u^k) = sum_x f_x(u^k)^2 for k = 0..2h-1, f_x the
    degree < h polynomial with f_x(u^(2y)) = a(x, y)."""
    x = _arr(a)
    assert len(x) == v * h
    out = np.zeros(2 * h, np.uint64)
    if lib().or_f2sp_prove(_p64(x), v, h, _p64(out)) != 0:
        raise ValueError("non-canonical input or h not dividing (p - 1) / 2")
    return out


def f2sp_verify(a, v: int, h: int, seed: int, proof):
    """(accept, F2 answer) of the verifier with the secret point r drawn from seed."""
    x = _arr(a)
    pr = _arr(proof)
    assert len(x) == v * h and len(pr) == 2 * h
    f2 = np.zeros(1, np.uint64)
    rc = lib().or_f2sp_verify(_p64(x), v, h, seed, _p64(pr), _p64(f2))
    if rc < 0:
        raise ValueError("non-canonical input")
    return bool(rc), int(f2[0])


def pm_layers(log_n: int, log_q: int):
    """Pattern matching (Sec. 6.2.1): for every location i of a text of n = 2^log_n
    symbols, v_i = sum_j (t_{i+j} - p_j)^2 over a pattern of q = 2^log_q symbols
    (zero exactly at an occurrence, for symbols far below p), then the F0
    subcircuit 4 [v_i != 0] and a sum: the output is 4 (n - occurrences).

    Input layout (2n entries): text, pattern, the constant p - 1 at n + q, the
    constant 1 at n + q + 1, zeros.  The two lowest layers are explicit:
      A: entry k <- text (times 1), -pattern (times p - 1), or 1 (1 times 1);
      B: gate i q + j <- t_{i+j} + (-p_j) for locations with i + q <= n, and
         1 = 1 * 1 at the q - 1 locations past the end (never an occurrence).
    Then a squaring layer, log_q addition layers over j, the F0 layers and
    log_n addition layers.  Returns (log_width, kinds, explicit)."""
    a, b = log_n, log_q
    assert a >= 2 and 0 <= b <= a - 1
    n, q = 1 << a, 1 << b
    m1, one = n + q, n + q + 1
    W = 2 * n
    ty_a = np.ones(W, np.uint8)
    a1 = np.full(W, one, np.uint32)
    a2 = np.full(W, one, np.uint32)
    for k in range(n):
        a1[k] = k
    for k in range(n, n + q):
        a1[k], a2[k] = k, m1
    Sb = n * q
    ty_b = np.zeros(Sb, np.uint8)
    b1 = np.zeros(Sb, np.uint32)
    b2 = np.zeros(Sb, np.uint32)
    for i in range(n):
        for j in range(q):
            g = i * q + j
            if i + q <= n:
                b1[g], b2[g] = i + j, n + j
            else:
                ty_b[g], b1[g], b2[g] = 1, m1, m1  # A[n + q] = 1
    log_width = list(range(0, a + 1)) + [a + 1] * 60 + list(range(a, a + b)) + [a + b, a + b, a + 1, a + 1]
    kinds = [TREE] * a + [F0_FINAL] + [F0_PAIR] * 59 + [F0_FIRST] + [TREE] * b + [SQUARE, EXPLICIT, EXPLICIT]
    explicit = [None] * (len(kinds) - 2) + [(ty_b, b1, b2), (ty_a, a1, a2)]
    return log_width, kinds, explicit


def mm1_layers(logm: int):
    """Single-output MatMult (Sec. 6.2.1): for m x m matrices A, B and the
    prover-supplied C, the output is 4 #{(i, j) : (A B)_ij != C_ij} (zero
    exactly when C = A B).  One explicit layer holds, for each (i, j), the m
    products A_ik B_kj, the entry C_ij (p - 1) and m - 1 zeros (0 0); log m + 1
    addition layers give (A B - C)_ij; then the F0 layers and 2 log m addition
    layers.  Input layout (4 m^2 entries): A row-major, B row-major, C
    row-major, p - 1 at 3 m^2, zeros.  Returns (log_width, kinds, explicit)."""
    L = logm
    m = 1 << L
    assert L >= 1
    m2 = m * m
    m1, zero = 3 * m2, 3 * m2 + 1
    S = m2 * 2 * m
    ty = np.ones(S, np.uint8)
    i1 = np.full(S, zero, np.uint32)
    i2 = np.full(S, zero, np.uint32)
    for i in range(m):
        for j in range(m):
            base = (i * m + j) * 2 * m
            for k in range(m):
                i1[base + k] = i * m + k
                i2[base + k] = m2 + k * m + j
            i1[base + m] = 2 * m2 + i * m + j
            i2[base + m] = m1
    log_width = list(range(0, 2 * L + 1)) + [2 * L + 1] * 60 + list(range(2 * L, 3 * L + 1)) + [3 * L + 1, 2 * L + 2]
    kinds = [TREE] * (2 * L) + [F0_FINAL] + [F0_PAIR] * 59 + [F0_FIRST] + [TREE] * (L + 1) + [EXPLICIT]
    explicit = [None] * (len(kinds) - 1) + [(ty, i1, i2)]
    return log_width, kinds, explicit


class Circuit:
    """Oracle-side layered circuit; layer 0 is the output, the last is the input."""

    def __init__(self, log_width, kinds, explicit=None):
        self.log_width = [int(x) for x in log_width]
        self.kinds = [int(k) for k in kinds]
        self.d = len(self.kinds)
        assert len(self.log_width) == self.d + 1
        L = lib()
        lw = (ctypes.c_uint32 * (self.d + 1))(*self.log_width)
        kd = (ctypes.c_uint32 * self.d)(*self.kinds)
        self._keep = []
        if explicit is not None:
            tys = (_u8p * self.d)()
            i1s = (_u32p * self.d)()
            i2s = (_u32p * self.d)()
            for i, layer in enumerate(explicit):
                if layer is None:
                    continue
                ty = np.ascontiguousarray(layer[0], dtype=np.uint8)
                a = np.ascontiguousarray(layer[1], dtype=np.uint32)
                b = np.ascontiguousarray(layer[2], dtype=np.uint32)
                self._keep += [ty, a, b]
                tys[i] = ty.ctypes.data_as(_u8p)
                i1s[i] = a.ctypes.data_as(_u32p)
                i2s[i] = b.ctypes.data_as(_u32p)
            h = L.or_circuit_new(self.d, lw, kd, tys, i1s, i2s)
        else:
            h = L.or_circuit_new(self.d, lw, kd, None, None, None)
        if not h:
            raise ValueError("layer widths do not fit the wiring kinds")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_circuit_free(h)
            self._h = None

    @property
    def n_inputs(self) -> int:
        return 1 << self.log_width[-1]

    def transcript_len(self) -> int:
        return lib().or_transcript_len(self._h)

    def num_challenges(self) -> int:
        return lib().or_num_challenges(self._h)

    def layer_offset(self, i: int) -> int:
        return lib().or_layer_offset(self._h, i)

    def layer_gates(self, i: int):
        S = 1 << self.log_width[i]
        ty = np.zeros(S, np.uint8)
        a = np.zeros(S, np.uint32)
        b = np.zeros(S, np.uint32)
        lib().or_circuit_layer(self._h, i, ty.ctypes.data_as(_u8p),
                               a.ctypes.data_as(_u32p), b.ctypes.data_as(_u32p))
        return ty, a, b

    def evaluate(self, inputs) -> list:
        """All layer values, list index = layer number (0 = output)."""
        x = _arr(inputs)
        assert len(x) == self.n_inputs
        vals = np.zeros(lib().or_total_values(self._h), dtype=np.uint64)
        if lib().or_evaluate(self._h, _p64(x), _p64(vals)) != 0:
            raise ValueError("non-canonical input")
        return [vals[self.layer_offset(i):self.layer_offset(i) + (1 << self.log_width[i])].copy()
                for i in range(self.d + 1)]

    def prove(self, inputs, seed: int, form: int = 2) -> np.ndarray:
        x = _arr(inputs)
        assert len(x) == self.n_inputs
        t = np.zeros(self.transcript_len(), dtype=np.uint64)
        if lib().or_prove(self._h, _p64(x), seed, form, _p64(t)) != 0:
            raise ValueError("non-canonical input")
        return t

    def prove_values(self, layers, seed: int, form: int = 2) -> np.ndarray:
        flat = np.ascontiguousarray(np.concatenate([_arr(v) for v in layers]))
        t = np.zeros(self.transcript_len(), dtype=np.uint64)
        lib().or_prove_values(self._h, _p64(flat), seed, form, _p64(t))
        return t

    def verify(self, inputs, seed: int, transcript):
        x = _arr(inputs)
        t = _arr(transcript)
        assert len(t) == self.transcript_len()
        where = ctypes.c_int(0)
        ok = lib().or_verify(self._h, _p64(x), seed, _p64(t), ctypes.byref(where))
        return bool(ok), where.value

    def wiring_eval(self, i, rP, r1, r2):
        add = np.zeros(1, np.uint64)
        mult = np.zeros(1, np.uint64)
        pad = lambda v: _arr(list(v) + [0])
        a, b, c = pad(rP), pad(r1), pad(r2)
        lib().or_wiring_eval(self._h, i, _p64(a), _p64(b), _p64(c), _p64(add), _p64(mult))
        return int(add[0]), int(mult[0])
