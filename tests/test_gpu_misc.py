"""Device field arithmetic, evaluation, error reporting, batching and
determinism of the CUDA path."""
import random

import numpy as np
import pytest

import oracle
from gpu_util import ensure_built, gpu_prove, oracle_prove, to_np
from paper_1202_1350_gb300 import circuits, vc
from paper_1202_1350_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
P = (1 << 61) - 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.uint64)).view(np.int64).copy()).cuda()


def test_field_mul_matches_bigint():
    rng = random.Random(0)
    edge = [0, 1, 2, P - 1, P - 2, 1 << 60, (1 << 32) - 1, 1 << 32, (1 << 61) - 2, 0x1FFFFFFF00000000]
    a = edge * len(edge) + [rng.randrange(P) for _ in range(20000)]
    b = [e for e in edge for _ in edge] + [rng.randrange(P) for _ in range(20000)]
    out = torch.empty(len(a), dtype=torch.int64, device="cuda")
    vc.vc_field_mul(dev(a), dev(b), out)
    torch.cuda.synchronize()
    got = to_np(out)
    want = np.array([(x * y) % P for x, y in zip(a, b)], dtype=np.uint64)
    assert (got == want).all()


def test_field_mul_rate_runs():
    rates = [vc.vc_field_mul_rate(0, variant, 1 << 10) for variant in range(5)]
    assert all(r > 1e10 for r in rates), rates
    # a 32-bit multiply-add is cheaper than any field product
    assert rates[3] > max(rates[0], rates[1], rates[2])
    with pytest.raises(vc.VcError):
        vc.vc_field_mul_rate(0, 5, 1 << 10)


@pytest.mark.parametrize("family,logn", [("f2", 12), ("f0", 5), ("matmult", 4)])
def test_evaluate_outputs(family, logn):
    widths, kinds = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 55)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        out = torch.empty(1 << widths[0], dtype=torch.int64, device="cuda")
        vc.vc_evaluate(h, dev(x), out)
        got = to_np(out)
    finally:
        vc.vc_circuit_destroy(h)
    assert (got == oracle.Circuit(widths, kinds).evaluate(x)[0]).all()
    if family == "f2":
        assert int(got[0]) == sum(int(v) ** 2 for v in x) % P
    if family == "f0":
        assert int(got[0]) == 4 * int((x != 0).sum()) % P
    if family == "matmult":
        n = 1 << logn
        A = x[:n * n].astype(np.int64).reshape(n, n)
        B = x[n * n:].astype(np.int64).reshape(n, n)
        assert (got.astype(np.int64).reshape(n, n) == A @ B).all()


def test_noncanonical_input_reported():
    widths, kinds = circuits.f2(6)
    x = I.f2_inputs(6, 1 << 16, 1)
    x[10] = P
    h = vc.vc_circuit_create(widths, kinds)
    try:
        tr = np.zeros(vc.vc_transcript_len(h), np.uint64)
        with pytest.raises(vc.VcError) as e:
            vc.vc_prove(h, np.ascontiguousarray(x), 1, tr)
        assert e.value.status == vc.VC_EINVAL
        # asynchronous form: latched, reported by vc_circuit_sync, then cleared
        trd = torch.empty(len(tr), dtype=torch.int64, device="cuda")
        vc.vc_prove(h, dev(x), 1, trd)
        with pytest.raises(vc.VcError):
            vc.vc_circuit_sync(h)
        vc.vc_circuit_sync(h)
        out = torch.empty(1, dtype=torch.int64, device="cuda")
        with pytest.raises(vc.VcError):
            vc.vc_evaluate(h, dev(x), out)
    finally:
        vc.vc_circuit_destroy(h)


@pytest.mark.parametrize("family,logn", [("f2", 11), ("matmult", 3), ("f0", 3)])
def test_input_memory_kinds_agree(family, logn):
    """Device inputs and page-locked host inputs are read in place by the first
    evaluation launch where it runs over the input layer; pageable host inputs
    are copied.  All give the oracle's transcript, which the verifier accepts
    from each kind of input memory (and a forged last entry it rejects); a
    later evaluation on the handle reads its own inputs, not the earlier
    proof's buffer."""
    widths, kinds = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 21)
    want = oracle_prove(widths, kinds, x, 77)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        n = vc.vc_transcript_len(h)
        xd = dev(x)
        xp = torch.from_numpy(np.ascontiguousarray(x).view(np.int64).copy()).pin_memory()
        for src in (xd, xp, np.ascontiguousarray(x)):
            tr = torch.empty(n, dtype=torch.int64, device="cuda")
            vc.vc_prove(h, src, 77, tr)
            vc.vc_circuit_sync(h)
            assert (to_np(tr) == want).all()
            # the verifier's input MLE reads the same three kinds of input memory
            assert vc.vc_verify(h, src, 77, tr)
            assert vc.vc_verify(h, src, 77, to_np(tr))
            forged = tr.clone()
            forged[-1] = (int(forged[-1]) + 1) % P
            assert not vc.vc_verify(h, src, 77, forged)
        # the last proof read xd in place: overwrite it, then evaluate other inputs
        vc.vc_prove(h, xd, 78, tr)
        vc.vc_circuit_sync(h)
        xd.fill_(1)
        y = I.job_inputs(family, logn, 22)
        out = torch.empty(1 << widths[0], dtype=torch.int64, device="cuda")
        vc.vc_evaluate(h, dev(y), out)
        assert (to_np(out) == oracle.Circuit(widths, kinds).evaluate(y)[0]).all()
        # a non-canonical page-locked input is reported: by the call itself
        # with a host transcript; with a device transcript by the call where
        # the inputs are copied, else (read in place: asynchronous) latched
        # for vc_circuit_sync
        bad = xp.clone().pin_memory()
        bad[3] = P
        with pytest.raises(vc.VcError) as e:
            vc.vc_prove(h, bad, 1, np.zeros(n, np.uint64))
        assert e.value.status == vc.VC_EINVAL
        with pytest.raises(vc.VcError) as e:
            vc.vc_prove(h, bad, 1, tr)
            vc.vc_circuit_sync(h)
        assert e.value.status == vc.VC_EINVAL
        vc.vc_circuit_sync(h)  # the latch is cleared
    finally:
        vc.vc_circuit_destroy(h)


def test_deterministic_and_seed_dependent():
    widths, kinds = circuits.f2(9)
    x = I.f2_inputs(9, 1 << 16, 2)
    a = gpu_prove(widths, kinds, x, 5)
    b = gpu_prove(widths, kinds, x, 5)
    c = gpu_prove(widths, kinds, x, 6)
    assert (a == b).all()
    assert (a[:1] == c[:1]).all() and not (a == c).all()


def test_repeated_proofs_on_one_handle():
    widths, kinds = circuits.matmult(3)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        for seed in range(1, 5):
            x = I.matmult_inputs(3, 1 << 10, seed)
            tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
            vc.vc_prove(h, dev(x), seed, tr)
            vc.vc_circuit_sync(h)
            assert (to_np(tr) == oracle_prove(widths, kinds, x, seed)).all()
    finally:
        vc.vc_circuit_destroy(h)


def test_batch_equals_individual():
    jobs = [("f2", 6, 1), ("f2", 11, 2), ("matmult", 3, 3), ("f2", 0, 4), ("f0", 2, 5)]
    hs, xs, trs, seeds = [], [], [], []
    try:
        for fam, logn, s in jobs:
            w, k = circuits.by_name(fam, logn)
            h = vc.vc_circuit_create(w, k)
            hs.append(h)
            xs.append(dev(I.job_inputs(fam, logn, s)))
            trs.append(torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda"))
            seeds.append(100 + s)
        vc.vc_prove_batch(hs, xs, seeds, trs)
        torch.cuda.synchronize()
        for (fam, logn, s), tr, seed in zip(jobs, trs, seeds):
            w, k = circuits.by_name(fam, logn)
            assert (to_np(tr) == oracle_prove(w, k, I.job_inputs(fam, logn, s), seed)).all()
    finally:
        for h in hs:
            vc.vc_circuit_destroy(h)
