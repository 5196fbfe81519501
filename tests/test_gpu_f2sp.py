"""The special-purpose non-interactive F2 protocol on the GPU: the proof
equals the oracle's bit for bit, the streaming verifier's accept bits and
answers equal the oracle verifier's, and at the bench size the answer is the
closed form sum a_i^2 and the honest proof is accepted."""
import numpy as np
import pytest

import oracle
from gpu_util import ensure_built, to_np
from paper_1202_1350_gb300 import inputs as I
from paper_1202_1350_gb300 import vc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
P = (1 << 61) - 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.uint64)).view(np.int64).copy()).cuda()


def gpu_proof(s, a, h, host=False):
    if host:
        out = np.zeros(2 * h, np.uint64)
        vc.vc_f2sp_prove(s, np.ascontiguousarray(a), out)
        return out
    out = torch.empty(2 * h, dtype=torch.int64, device="cuda")
    vc.vc_f2sp_prove(s, dev(a), out)
    return to_np(out)


def gpu_verify(s, a, v, h, seed, proof, chunk=None):
    vc.vc_f2sp_verify_begin(s, seed)
    chunk = chunk or v
    for x0 in range(0, v, chunk):
        n = min(chunk, v - x0)
        vc.vc_f2sp_verify_absorb(s, dev(a[x0 * h:(x0 + n) * h]), x0, n)
    return vc.vc_f2sp_verify_end(s, dev(proof))


# h: one and several transform dimensions, every allowed prime power
SHAPES = [(1, 1), (1, 3), (3, 5), (8, 9), (5, 31), (64, 63), (17, 143), (2, 315), (300, 3), (7, 25), (3, 41 * 3),
          (2, 61 * 5), (4, 1001)]


@pytest.mark.parametrize("v,h", SHAPES)
def test_proof_equals_oracle(v, h):
    a = I.uniform_ints(1000 + v + h, v * h, 1 << 16)
    s = vc.vc_f2sp_create(v, h)
    try:
        want = oracle.f2sp_prove(a, v, h)
        assert (gpu_proof(s, a, h) == want).all()
        assert (gpu_proof(s, a, h, host=True) == want).all()
    finally:
        vc.vc_f2sp_destroy(s)


@pytest.mark.parametrize("v,h", [(1, 1), (3, 5), (8, 9), (64, 63), (17, 143)])
def test_verifier_equals_oracle(v, h):
    a = I.uniform_ints(2000 + v + h, v * h, 1 << 16)
    s = vc.vc_f2sp_create(v, h)
    try:
        proof = oracle.f2sp_prove(a, v, h)
        for seed in (1, 2, 0xDEADBEEF):
            got = gpu_verify(s, a, v, h, seed, proof, chunk=max(1, v // 3))
            assert got == oracle.f2sp_verify(a, v, h, seed, proof)
            assert got[0]
        for m in (0, 1, h - 1, 2 * h - 1):
            bad = proof.copy()
            bad[m] = (int(bad[m]) + 5) % P
            got = gpu_verify(s, a, v, h, 7, bad)
            assert got == oracle.f2sp_verify(a, v, h, 7, bad)
            assert not got[0]
    finally:
        vc.vc_f2sp_destroy(s)


def _odd_point_direct(a, v, h, y):
    """s(u w^y) from f_x(u w^y) = sum_j a(x, j) L_j(u w^y) with the subgroup's
    Lagrange basis L_j(X) = w^j (X^h - 1) / (h (X - w^j)) (big integers): a
    check independent of the prover's transform."""
    u = oracle.f2sp_root(h)
    w = u * u % P
    X = u * pow(w, y, P) % P
    c = (pow(X, h, P) - 1) * pow(h, -1, P) % P
    basis = [pow(w, j, P) * c * pow((X - pow(w, j, P)) % P, -1, P) % P for j in range(h)]
    total = 0
    for x in range(v):
        f = sum(int(a[x * h + j]) * basis[j] for j in range(h)) % P
        total += f * f
    return total % P


def test_bench_size_closed_form():
    """n ~ 2^20 as a 1048 x 1001 grid (1001 = 7 11 13): the answer is sum a_i^2
    (big integers), the even points are the columns' sums of squares, sampled
    odd points equal a direct evaluation, the honest proof is accepted at
    several secret points and a changed entry anywhere is rejected."""
    v, h = 1048, 1001
    a = I.uniform_ints(5, v * h, 1 << 16)
    s = vc.vc_f2sp_create(v, h)
    try:
        proof = gpu_proof(s, a, h)
        f2 = int((a.astype(object) ** 2).sum()) % P
        grid = a.astype(object).reshape(v, h)
        assert [int(t) for t in proof[0::2]] == [int(c) % P for c in (grid ** 2).sum(axis=0)]
        for y in (0, 500, h - 1):
            assert int(proof[2 * y + 1]) == _odd_point_direct(a, v, h, y)
        for seed in (3, 4, 5):
            assert gpu_verify(s, a, v, h, seed, proof, chunk=300) == (True, f2)
        for m in (5, h + 8, 2 * h - 1):
            bad = proof.copy()
            bad[m] = (int(bad[m]) + 1) % P
            assert not gpu_verify(s, a, v, h, 3, bad)[0]
    finally:
        vc.vc_f2sp_destroy(s)


def test_paper_row_length():
    """h = 5005 = 5 7 11 13 (the paper's 25-million-entry rows of about 5000
    entries; the oracle is too slow here): even points are the columns' sums
    of squares, sampled odd points equal a direct evaluation, the verifier
    (equal to the oracle's at small sizes) accepts at several secret points
    and rejects a changed extension value."""
    v, h = 3, 5005
    a = I.uniform_ints(31, v * h, 1 << 16)
    s = vc.vc_f2sp_create(v, h)
    try:
        proof = gpu_proof(s, a, h)
        grid = a.astype(object).reshape(v, h)
        assert [int(t) for t in proof[0::2]] == [int(c) % P for c in (grid ** 2).sum(axis=0)]
        for y in (0, 1, 1234, h - 1):
            assert int(proof[2 * y + 1]) == _odd_point_direct(a, v, h, y)
        for seed in (1, 2, 3):
            assert gpu_verify(s, a, v, h, seed, proof)[0]
        bad = proof.copy()
        bad[2 * 1500 + 1] = (int(bad[2 * 1500 + 1]) + 1) % P
        assert not gpu_verify(s, a, v, h, 1, bad)[0]
    finally:
        vc.vc_f2sp_destroy(s)


def _absorb_split(s, rows, h, splits):
    """Absorb rows [0, v) in calls of the given row counts (host memory)."""
    x0 = 0
    for n in splits:
        vc.vc_f2sp_verify_absorb(s, rows[x0 * h:(x0 + n) * h], x0, n)
        x0 += n


# the library streams host rows in chunks of about 2^21 entries (16 MB):
# these grids span at least three
@pytest.mark.parametrize("v,h,uneven", [(2_200_000, 3, [1, 300_001, 1_000_000]),
                                        (450_000, 15, [1, 60_001, 200_000])])
def test_streaming_host_rows_double_buffered(v, h, uneven):
    """Host rows stream through the verifier's two device buffers, so these
    grids span several chunks: one absorb call over all rows, calls that
    split chunks unevenly (1 row, then sizes that are no multiple of a
    chunk, the rest), page-locked and pageable rows, and host calls mixed
    with device rows all give the oracle verifier's accept bit and answer,
    for the honest proof and a changed one."""
    chunk = (1 << 21) // h
    a = I.uniform_ints(4000 + h, v * h, 1 << 16)
    proof = oracle.f2sp_prove(a, v, h)
    bad = proof.copy()
    bad[2 * (h // 2) + 1] = (int(bad[2 * (h // 2) + 1]) + 3) % P
    pinned = torch.from_numpy(a.view(np.int64).copy()).pin_memory()
    pageable = np.ascontiguousarray(a)
    uneven = uneven + [v - sum(uneven)]
    s = vc.vc_f2sp_create(v, h)
    try:
        for pr, seed in ((proof, 11), (bad, 12)):
            want = oracle.f2sp_verify(a, v, h, seed, pr)
            assert want[0] == (pr is proof)
            for rows, splits in ((pinned, [v]), (pinned, uneven), (pageable, [v]), (pageable, uneven)):
                vc.vc_f2sp_verify_begin(s, seed)
                _absorb_split(s, rows, h, splits)
                assert vc.vc_f2sp_verify_end(s, dev(pr)) == want, (len(splits), type(rows))
            # host chunks, then the rest from the device
            vc.vc_f2sp_verify_begin(s, seed)
            _absorb_split(s, pinned, h, [chunk + 5])
            x0 = chunk + 5
            vc.vc_f2sp_verify_absorb(s, dev(a[x0 * h:]), x0, v - x0)
            assert vc.vc_f2sp_verify_end(s, pr) == want
    finally:
        vc.vc_f2sp_destroy(s)


def test_streaming_reuses_one_host_buffer():
    """The caller streams every row through one page-locked buffer, refilling
    it as soon as each absorb call returns (the rows have been copied by
    then, while the absorbs still run): the verdict equals the oracle's."""
    v, h = 600_000, 5
    part = 50_000
    a = I.uniform_ints(4100, v * h, 1 << 16)
    proof = oracle.f2sp_prove(a, v, h)
    want = oracle.f2sp_verify(a, v, h, 21, proof)
    assert want[0]
    buf = torch.empty(part * h, dtype=torch.int64).pin_memory()
    s = vc.vc_f2sp_create(v, h)
    try:
        vc.vc_f2sp_verify_begin(s, 21)
        for x0 in range(0, v, part):
            buf.copy_(torch.from_numpy(a[x0 * h:(x0 + part) * h].view(np.int64)))
            vc.vc_f2sp_verify_absorb(s, buf, x0, part)
        assert vc.vc_f2sp_verify_end(s, proof) == want
    finally:
        vc.vc_f2sp_destroy(s)


def test_async_streaming_two_buffers():
    """The asynchronous absorb returns before its own rows are copied (once
    the previous call's are), so the caller alternates two page-locked
    buffers, refilling the one it passed two calls ago: the verdict equals the
    oracle's, for chunks smaller and larger than the device buffers."""
    v, h = 600_000, 5
    a = I.uniform_ints(4200, v * h, 1 << 16)
    proof = oracle.f2sp_prove(a, v, h)
    want = oracle.f2sp_verify(a, v, h, 22, proof)
    assert want[0]
    s = vc.vc_f2sp_create(v, h)
    try:
        for part in (30_000, 250_000):
            bufs = [torch.empty(part * h, dtype=torch.int64).pin_memory() for _ in range(2)]
            vc.vc_f2sp_verify_begin(s, 22)
            for k, x0 in enumerate(range(0, v, part)):
                n = min(part, v - x0)
                b = bufs[k & 1]
                b[:n * h].copy_(torch.from_numpy(a[x0 * h:(x0 + n) * h].view(np.int64)))
                vc.vc_f2sp_verify_absorb_async(s, b[:n * h], x0, n)
            assert vc.vc_f2sp_verify_end(s, proof) == want, part
    finally:
        vc.vc_f2sp_destroy(s)


def test_bad_inputs():
    s = vc.vc_f2sp_create(4, 5)
    try:
        a = I.uniform_ints(9, 20, 100)
        a[3] = P
        with pytest.raises(vc.VcError) as e:
            gpu_proof(s, a, 5)
        assert e.value.status == vc.VC_EINVAL
        with pytest.raises(vc.VcError) as e:
            gpu_verify(s, a, 4, 5, 1, oracle.f2sp_prove(I.uniform_ints(9, 20, 100), 4, 5))
        assert e.value.status == vc.VC_EINVAL
        good = I.uniform_ints(10, 20, 100)
        proof = gpu_proof(s, good, 5)  # the context is usable again
        assert (proof == oracle.f2sp_prove(good, 4, 5)).all()
    finally:
        vc.vc_f2sp_destroy(s)
    # h must be a product of distinct members of {3|9, 5|25, 7, 11, 13, 31, 41, 61}, at most 7000
    for h in (0, 2, 4, 27, 125, 151, 9009, 7007 * 3):
        assert not vc.f2sp_valid_h(h)
        with pytest.raises(vc.VcError):
            vc.vc_f2sp_create(4, h)
