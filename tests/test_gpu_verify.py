"""The CUDA verifier: accepts honest transcripts, rejects tampered ones, and
agrees with the oracle verifier on every case (Sec. 2.1: completeness and
soundness)."""
import random

import numpy as np
import pytest

import oracle
from gpu_util import ensure_built, gpu_prove, to_np
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


CASES = [("f2", 10), ("f2", 1), ("f0", 3), ("matmult", 2), ("matmult", 0)]


@pytest.mark.parametrize("family,logn", CASES)
def test_honest_accepted(family, logn):
    widths, kinds = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 17)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        for seed in (1, 2, 3, 1 << 63):
            tr = gpu_prove(widths, kinds, x, seed)
            assert vc.vc_verify(h, dev(x), seed, dev(tr))
            assert oracle.Circuit(widths, kinds).verify(x, seed, tr) == (True, -1)
    finally:
        vc.vc_circuit_destroy(h)


def test_every_single_change_rejected():
    widths, kinds = circuits.f2(5)
    x = I.f2_inputs(5, 1 << 16, 5)
    seed = 9
    tr = gpu_prove(widths, kinds, x, seed)
    h = vc.vc_circuit_create(widths, kinds)
    rng = random.Random(1)
    try:
        xd = dev(x)
        for k in range(len(tr)):
            bad = tr.copy()
            bad[k] = (int(bad[k]) + 1 + rng.randrange(P - 1)) % P
            assert not vc.vc_verify(h, xd, seed, dev(bad)), k
    finally:
        vc.vc_circuit_destroy(h)


@pytest.mark.parametrize("family,logn", CASES + [("explicit", 0)])
def test_agrees_with_oracle_on_random_tampering(family, logn):
    rng = random.Random(hash((family, logn)) & 0xFFFF)
    if family == "explicit":
        widths, kinds = [3, 4, 2], [6, 6]
        ex = []
        for i in range(2):
            S, Sn = 1 << widths[i], 1 << widths[i + 1]
            ex.append((np.array([rng.randrange(2) for _ in range(S)], np.uint8),
                       np.array([rng.randrange(Sn) for _ in range(S)], np.uint32),
                       np.array([rng.randrange(Sn) for _ in range(S)], np.uint32)))
        x = np.array([rng.randrange(P) for _ in range(4)], np.uint64)
    else:
        widths, kinds = circuits.by_name(family, logn)
        ex = None
        x = I.job_inputs(family, logn, 23)
    seed = 31
    tr = gpu_prove(widths, kinds, x, seed, ex)
    oc = oracle.Circuit(widths, kinds, explicit=ex)
    h = vc.vc_circuit_create(widths, kinds, ex)
    try:
        xd = dev(x)
        assert vc.vc_verify(h, xd, seed, dev(tr))
        for _ in range(40):
            bad = tr.copy()
            k = rng.randrange(len(tr))
            bad[k] = rng.randrange(P)
            want = oc.verify(x, seed, bad)[0]
            assert vc.vc_verify(h, xd, seed, dev(bad)) == want
        # the right transcript for other inputs or another seed is rejected
        y = x.copy()
        y[0] = (int(y[0]) + 1) % P
        assert not vc.vc_verify(h, dev(y), seed, dev(tr))
        assert not vc.vc_verify(h, xd, seed + 1, dev(tr))
    finally:
        vc.vc_circuit_destroy(h)


def test_wrong_evaluation_rejected():
    """An oracle prover whose layer values carry one wrong gate (layers above
    recomputed) is rejected by the CUDA verifier, as by the oracle's."""
    widths, kinds = circuits.f2(6)
    x = I.f2_inputs(6, 1 << 16, 41)
    oc = oracle.Circuit(widths, kinds)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        for layer in (1, 3, 6):
            vals = [v.astype(object) for v in oc.evaluate(x)]
            g = min(2, len(vals[layer]) - 1)
            vals[layer][g] = (int(vals[layer][g]) + 1) % P
            for i in range(layer - 1, -1, -1):
                ty, a, b = oc.layer_gates(i)
                vals[i] = np.array([(int(vals[i + 1][a[k]]) * int(vals[i + 1][b[k]])) % P if ty[k]
                                    else (int(vals[i + 1][a[k]]) + int(vals[i + 1][b[k]])) % P
                                    for k in range(len(ty))], dtype=object)
            tr = oc.prove_values([np.array(v, dtype=np.uint64) for v in vals], 12)
            assert not vc.vc_verify(h, dev(x), 12, dev(tr))
    finally:
        vc.vc_circuit_destroy(h)


def test_noncanonical_values():
    widths, kinds = circuits.f2(4)
    x = I.f2_inputs(4, 1 << 16, 3)
    tr = gpu_prove(widths, kinds, x, 4)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        bad = tr.copy()
        bad[5] = P
        assert not vc.vc_verify(h, dev(x), 4, dev(bad))
        y = x.copy()
        y[1] = P
        with pytest.raises(vc.VcError) as e:
            vc.vc_verify(h, dev(y), 4, dev(tr))
        assert e.value.status == vc.VC_EINVAL
    finally:
        vc.vc_circuit_destroy(h)


def test_host_pointers():
    widths, kinds = circuits.f2(8)
    x = I.f2_inputs(8, 1 << 16, 8)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        tr = np.zeros(vc.vc_transcript_len(h), np.uint64)
        vc.vc_prove(h, np.ascontiguousarray(x), 6, tr)
        assert (tr == gpu_prove(widths, kinds, x, 6)).all()
        assert vc.vc_verify(h, np.ascontiguousarray(x), 6, tr)
        assert vc.vc_verify(h, dev(x), 6, tr)
    finally:
        vc.vc_circuit_destroy(h)


@pytest.mark.parametrize("which", ["pm", "mm1"])
def test_pm_and_mm1_verified(which):
    """Explicit-wiring circuits: the CUDA verifier (wiring predicates summed
    over the gates) accepts the honest proof and rejects a changed message."""
    if which == "pm":
        widths, kinds, ex = circuits.pattern_match(6, 2)
        x = I.pm_inputs(6, 2, 21)
    else:
        widths, kinds, ex = circuits.matmult_check(3)
        x = I.mm1_inputs(3, 22, errors=2)
    h = vc.vc_circuit_create(widths, kinds, ex)
    try:
        tr = gpu_prove(widths, kinds, x, 41, ex)
        assert vc.vc_verify(h, dev(x), 41, dev(tr))
        for pos in (0, len(tr) // 3, len(tr) - 1):
            bad = tr.copy()
            bad[pos] = (int(bad[pos]) + 1) % P
            assert not vc.vc_verify(h, dev(x), 41, dev(bad))
    finally:
        vc.vc_circuit_destroy(h)


# ---- the verifier in two passes: input pass (beside the proof), transcript pass

def two_pass(h, x, seed, tr, stream=None):
    vc.vc_verify_input(h, x, seed, stream=stream)
    return vc.vc_verify_transcript(h, seed, tr, stream=stream)


@pytest.mark.parametrize("family,logn", CASES + [("matmult", 4), ("matmult", 5), ("pm", 0), ("mm1", 0)])
def test_two_pass_agrees_with_one_pass(family, logn):
    """Honest transcripts accepted, changed ones rejected, exactly as vc_verify
    decides, for structured and explicitly wired circuits (MatMult n = 32:
    2^10 outputs, whose MLE comes from partial sums; up to 256 outputs, as for
    n = 16: formed in the check launch)."""
    ex = None
    if family == "pm":
        widths, kinds, ex = circuits.pattern_match(5, 2)
        x = I.pm_inputs(5, 2, 23)
    elif family == "mm1":
        widths, kinds, ex = circuits.matmult_check(2)
        x = I.mm1_inputs(2, 24, errors=1)
    else:
        widths, kinds = circuits.by_name(family, logn)
        x = I.job_inputs(family, logn, 19)
    h = vc.vc_circuit_create(widths, kinds, ex)
    rng = random.Random(7)
    try:
        xd = dev(x)
        for seed in (3, 1 << 62):
            tr = gpu_prove(widths, kinds, x, seed, ex)
            assert two_pass(h, xd, seed, dev(tr))
            assert two_pass(h, xd, seed, tr)  # host transcript: returns after the bit is read
            for _ in range(4):
                bad = tr.copy()
                k = rng.randrange(len(tr))
                bad[k] = (int(bad[k]) + 1 + rng.randrange(P - 1)) % P
                assert not two_pass(h, xd, seed, dev(bad))
                assert not vc.vc_verify(h, xd, seed, dev(bad))
    finally:
        vc.vc_circuit_destroy(h)


def test_input_pass_beside_the_proof():
    """The input pass runs on a second stream while the proof runs on the
    first, on one handle; the transcript pass then accepts the proof."""
    widths, kinds = circuits.f2(16)
    h = vc.vc_circuit_create(widths, kinds)
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    try:
        n = vc.vc_transcript_len(h)
        acc = torch.zeros(1, dtype=torch.int32, device="cuda")
        for seed in (5, 6, 7):
            x = I.f2_inputs(16, 1 << 16, seed)
            xd, tr = dev(x), torch.empty(n, dtype=torch.int64, device="cuda")
            start, done = torch.cuda.Event(), torch.cuda.Event()
            start.record(main)
            side.wait_event(start)
            vc.vc_verify_input(h, xd, seed, stream=side)
            done.record(side)
            vc.vc_prove(h, xd, seed, tr)
            main.wait_event(done)
            acc.zero_()
            vc.vc_verify_transcript(h, seed, tr, accept=acc)
            vc.vc_circuit_sync(h)
            assert int(acc.item()) == 1
            if seed == 5:
                assert (to_np(tr) == oracle.Circuit(widths, kinds).prove(x, seed)).all()
    finally:
        torch.cuda.synchronize()
        vc.vc_circuit_destroy(h)


def test_two_pass_misuse_and_bad_inputs():
    widths, kinds = circuits.f2(6)
    x = I.f2_inputs(6, 1 << 16, 4)
    tr = gpu_prove(widths, kinds, x, 8)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        def einval(f, *a, **k):
            with pytest.raises(vc.VcError) as e:
                f(*a, **k)
            assert e.value.status == vc.VC_EINVAL

        einval(vc.vc_verify_transcript, h, 8, tr)           # no input pass
        vc.vc_verify_input(h, dev(x), 8)
        einval(vc.vc_verify_transcript, h, 9, tr)           # another seed
        assert vc.vc_verify_transcript(h, 8, tr)
        einval(vc.vc_verify_transcript, h, 8, tr)           # the pass was consumed
        vc.vc_verify_input(h, dev(x), 8)
        assert vc.vc_verify(h, dev(x), 8, dev(tr))          # a one-pass call in between
        einval(vc.vc_verify_transcript, h, 8, tr)
        einval(vc.vc_verify_input, h, np.ascontiguousarray(x), 8)  # pageable host inputs
        # page-locked host inputs are read in place
        xp = torch.from_numpy(np.ascontiguousarray(x).view(np.int64).copy()).pin_memory()
        vc.vc_verify_input(h, xp, 8)
        assert vc.vc_verify_transcript(h, 8, dev(tr))
        # a non-canonical input: reported by the synchronous transcript pass,
        # or latched for vc_circuit_sync by the asynchronous one
        bad = xp.clone().pin_memory()
        bad[2] = P
        vc.vc_verify_input(h, bad, 8)
        einval(vc.vc_verify_transcript, h, 8, dev(tr))
        yd = dev(x)
        yd[2] = P
        acc = torch.zeros(1, dtype=torch.int32, device="cuda")
        vc.vc_verify_input(h, yd, 8)
        vc.vc_verify_transcript(h, 8, dev(tr), accept=acc)
        einval(vc.vc_circuit_sync, h)
        vc.vc_circuit_sync(h)
    finally:
        vc.vc_circuit_destroy(h)


def test_two_pass_at_the_bench_size():
    """F2 n = 2^20 (the bench workload): the input pass beside the proof, the
    transcript pass accepts; changed round values, line values and the output
    are rejected."""
    widths, kinds = circuits.f2(20)
    h = vc.vc_circuit_create(widths, kinds)
    side = torch.cuda.Stream()
    main = torch.cuda.current_stream()
    try:
        x = dev(I.f2_inputs(20, 1 << 16, 77))
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        start = torch.cuda.Event()
        start.record(main)
        vc.vc_prove(h, x, 123, tr)
        side.wait_event(start)
        vc.vc_verify_input(h, x, 123, stream=side)
        main.wait_stream(side)
        assert vc.vc_verify_transcript(h, 123, tr)
        n = len(tr)
        for pos in (0, 1, 2, n // 2, n - 1):
            bad = tr.clone()
            bad[pos] = (int(bad[pos]) + 1) % P
            vc.vc_verify_input(h, x, 123)
            assert not vc.vc_verify_transcript(h, 123, bad), pos
    finally:
        torch.cuda.synchronize()
        vc.vc_circuit_destroy(h)


def _oracle_transcript(w, k, x, seed, explicit=None):
    return oracle.Circuit(w, k, explicit=explicit).prove(np.asarray(x, np.uint64), seed)


@pytest.mark.parametrize("family,logn", [("f2", 0), ("f2", 5), ("f2", 12), ("f0", 6), ("matmult", 3)])
def test_prove_verify_one_call(family, logn):
    """vc_prove_verify (the proof, the verifier's input pass beside it and its
    checks after it, one graph): the transcript equals the oracle's and the
    accept bit is set, with device buffers (asynchronous), with host buffers
    (synchronous), with page-locked inputs read in place, and twice in a row
    on one handle; the same handle then verifies with vc_verify."""
    w, k = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 40 + logn)
    h = vc.vc_circuit_create(w, k)
    try:
        n = vc.vc_transcript_len(h)
        tr = torch.empty(n, dtype=torch.int64, device="cuda")
        acc = torch.zeros(1, dtype=torch.int32, device="cuda")
        for seed in (9, 10, 9):
            acc.zero_()
            vc.vc_prove_verify(h, dev(x), seed, tr, accept=acc)
            vc.vc_circuit_sync(h)
            assert (to_np(tr) == _oracle_transcript(w, k, x, seed)).all()
            assert int(acc.item()) == 1
        trh = np.zeros(n, np.uint64)
        assert vc.vc_prove_verify(h, np.ascontiguousarray(x, np.uint64), 11, trh) is True
        assert (trh == _oracle_transcript(w, k, x, 11)).all()
        xp = torch.from_numpy(np.ascontiguousarray(x, np.uint64).view(np.int64).copy()).pin_memory()
        acc.zero_()
        vc.vc_prove_verify(h, xp, 12, tr, accept=acc)
        vc.vc_circuit_sync(h)
        assert (to_np(tr) == _oracle_transcript(w, k, x, 12)).all() and int(acc.item()) == 1
        assert vc.vc_verify(h, dev(x), 12, tr)
        bad = tr.clone()
        bad[n - 1] = (int(bad[n - 1]) + 1) % P
        assert not vc.vc_verify(h, dev(x), 12, bad)
    finally:
        torch.cuda.synchronize()
        vc.vc_circuit_destroy(h)


@pytest.mark.parametrize("mode", ["upload", "host_values", "staged"])
def test_prove_verify_modes(mode):
    """The one-call form with uploaded inputs (the verifier reads the input
    layer the library's copy filled) and with layer values in mapped host
    memory equals the oracle; circuits whose values pass through device slots
    are refused; a non-canonical input is reported."""
    w, k = circuits.f2(11)
    x = I.f2_inputs(11, 1 << 16, 31)
    h = vc.vc_circuit_create(w, k, **{mode: True})
    try:
        n = vc.vc_transcript_len(h)
        tr = torch.empty(n, dtype=torch.int64, device="cuda")
        acc = torch.zeros(1, dtype=torch.int32, device="cuda")
        xp = torch.from_numpy(np.ascontiguousarray(x, np.uint64).view(np.int64).copy()).pin_memory()
        if mode == "staged":
            with pytest.raises(vc.VcError) as e:
                vc.vc_prove_verify(h, xp, 3, tr, accept=acc)
            assert e.value.status == vc.VC_EINVAL
            return
        vc.vc_prove_verify(h, xp, 3, tr, accept=acc)
        vc.vc_circuit_sync(h)
        assert (to_np(tr) == _oracle_transcript(w, k, x, 3)).all() and int(acc.item()) == 1
        xp[5] = P  # not a field element
        with pytest.raises(vc.VcError) as e:
            vc.vc_prove_verify(h, xp, 4, tr, accept=acc)
            vc.vc_circuit_sync(h)
        assert e.value.status == vc.VC_EINVAL
        vc.vc_circuit_sync(h)
    finally:
        torch.cuda.synchronize()
        vc.vc_circuit_destroy(h)
