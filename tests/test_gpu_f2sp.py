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
        out = np.zeros(2 * h - 1, np.uint64)
        vc.vc_f2sp_prove(s, np.ascontiguousarray(a), out)
        return out
    out = torch.empty(2 * h - 1, dtype=torch.int64, device="cuda")
    vc.vc_f2sp_prove(s, dev(a), out)
    return to_np(out)


def gpu_verify(s, a, v, h, seed, proof, chunk=None):
    vc.vc_f2sp_verify_begin(s, seed)
    chunk = chunk or v
    for x0 in range(0, v, chunk):
        n = min(chunk, v - x0)
        vc.vc_f2sp_verify_absorb(s, dev(a[x0 * h:(x0 + n) * h]), x0, n)
    return vc.vc_f2sp_verify_end(s, dev(proof))


SHAPES = [(1, 1), (1, 2), (3, 4), (8, 8), (5, 31), (64, 64), (17, 130), (2, 300), (300, 3)]


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


@pytest.mark.parametrize("v,h", [(1, 1), (3, 4), (8, 8), (64, 64), (17, 130)])
def test_verifier_equals_oracle(v, h):
    a = I.uniform_ints(2000 + v + h, v * h, 1 << 16)
    s = vc.vc_f2sp_create(v, h)
    try:
        proof = oracle.f2sp_prove(a, v, h)
        for seed in (1, 2, 0xDEADBEEF):
            got = gpu_verify(s, a, v, h, seed, proof, chunk=max(1, v // 3))
            assert got == oracle.f2sp_verify(a, v, h, seed, proof)
            assert got[0]
        for m in (0, h - 1, 2 * h - 2):
            bad = proof.copy()
            bad[m] = (int(bad[m]) + 5) % P
            got = gpu_verify(s, a, v, h, 7, bad)
            assert got == oracle.f2sp_verify(a, v, h, 7, bad)
            assert not got[0]
    finally:
        vc.vc_f2sp_destroy(s)


def test_bench_size_closed_form():
    """n = 2^20 as a 1024 x 1024 grid: the answer is sum a_i^2 (big integers)
    and the honest proof is accepted at several secret points; a changed
    entry anywhere is rejected."""
    v = h = 1024
    a = I.f2_inputs(20, 1 << 16, 5)
    s = vc.vc_f2sp_create(v, h)
    try:
        proof = gpu_proof(s, a, h)
        f2 = int((a.astype(object) ** 2).sum()) % P
        grid = a.astype(object).reshape(v, h)
        assert [int(t) for t in proof[:h]] == [int(c) % P for c in (grid ** 2).sum(axis=0)]
        for seed in (3, 4, 5):
            assert gpu_verify(s, a, v, h, seed, proof, chunk=300) == (True, f2)
        for m in (5, h + 7, 2 * h - 2):
            bad = proof.copy()
            bad[m] = (int(bad[m]) + 1) % P
            assert not gpu_verify(s, a, v, h, 3, bad)[0]
    finally:
        vc.vc_f2sp_destroy(s)


def test_rows_longer_than_one_tile():
    """h above the prover's 1024-entry shared-memory tile (the oracle is too
    slow here): the first h proof entries are the columns' sums of squares and
    the verifier, equal to the oracle's at small sizes, accepts the proof at
    several secret points and rejects a changed extension value."""
    v, h = 3, 2100
    a = I.uniform_ints(31, v * h, 1 << 16)
    s = vc.vc_f2sp_create(v, h)
    try:
        proof = gpu_proof(s, a, h)
        grid = a.astype(object).reshape(v, h)
        assert [int(t) for t in proof[:h]] == [int(c) % P for c in (grid ** 2).sum(axis=0)]
        for seed in (1, 2, 3):
            assert gpu_verify(s, a, v, h, seed, proof)[0]
        bad = proof.copy()
        bad[h + 1500] = (int(bad[h + 1500]) + 1) % P
        assert not gpu_verify(s, a, v, h, 1, bad)[0]
    finally:
        vc.vc_f2sp_destroy(s)


def test_bad_inputs():
    s = vc.vc_f2sp_create(4, 4)
    try:
        a = I.uniform_ints(9, 16, 100)
        a[3] = P
        with pytest.raises(vc.VcError) as e:
            gpu_proof(s, a, 4)
        assert e.value.status == vc.VC_EINVAL
        with pytest.raises(vc.VcError) as e:
            gpu_verify(s, a, 4, 4, 1, oracle.f2sp_prove(I.uniform_ints(9, 16, 100), 4, 4))
        assert e.value.status == vc.VC_EINVAL
        good = I.uniform_ints(10, 16, 100)
        proof = gpu_proof(s, good, 4)  # the context is usable again
        assert (proof == oracle.f2sp_prove(good, 4, 4)).all()
    finally:
        vc.vc_f2sp_destroy(s)
    with pytest.raises(vc.VcError):
        vc.vc_f2sp_create(4, 0)
    with pytest.raises(vc.VcError):
        vc.vc_f2sp_create(4, 9000)
