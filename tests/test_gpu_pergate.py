"""The per-gate prover (the paper's method: one thread per gate per round)
gives the oracle's transcript on every circuit family, including explicit
wiring, and the same transcript as the folding prover."""
import numpy as np
import pytest

from gpu_util import ensure_built, first_mismatch, oracle_prove, to_np
from paper_1202_1350_gb300 import circuits, vc
from paper_1202_1350_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.uint64)).view(np.int64).copy()).cuda()


def both(widths, kinds, x, seed, explicit=None):
    h = vc.vc_circuit_create(widths, kinds, explicit)
    try:
        n = vc.vc_transcript_len(h)
        a = torch.empty(n, dtype=torch.int64, device="cuda")
        b = torch.empty(n, dtype=torch.int64, device="cuda")
        xd = dev(x)
        vc.vc_prove_pergate(h, xd, seed, a)
        vc.vc_prove(h, xd, seed, b)
        vc.vc_prove_pergate(h, xd, seed + 1, a)  # a second call replays the captured launches
        vc.vc_prove_pergate(h, xd, seed, a)
        vc.vc_circuit_sync(h)
        return to_np(a), to_np(b)
    finally:
        vc.vc_circuit_destroy(h)


CASES = [("f2", 0), ("f2", 1), ("f2", 5), ("f2", 11), ("f0", 3), ("matmult", 1), ("matmult", 3)]


@pytest.mark.parametrize("family,logn", CASES)
def test_pergate_equals_oracle(family, logn):
    w, k = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 60 + logn)
    pg, fold = both(w, k, x, 7)
    want = oracle_prove(w, k, x, 7)
    assert first_mismatch(pg, want) is None
    assert (fold == want).all()


@pytest.mark.parametrize("which", ["pm", "mm1"])
def test_pergate_explicit_circuits(which):
    if which == "pm":
        w, k, ex = circuits.pattern_match(5, 2)
        x = I.pm_inputs(5, 2, 3)
    else:
        w, k, ex = circuits.matmult_check(2)
        x = I.mm1_inputs(2, 4, errors=1)
    pg, fold = both(w, k, x, 11, ex)
    assert first_mismatch(pg, oracle_prove(w, k, x, 11, explicit=ex)) is None
    assert (pg == fold).all()


def test_pergate_f2_2e16_equals_folding():
    """Above the oracle's comfortable sizes: the two CUDA provers agree."""
    w, k = circuits.f2(16)
    pg, fold = both(w, k, I.f2_inputs(16, 1 << 16, 5), 21)
    assert first_mismatch(pg, fold) is None


def test_pergate_host_pointers_and_bad_input():
    w, k = circuits.f2(6)
    x = I.f2_inputs(6, 1 << 16, 8)
    h = vc.vc_circuit_create(w, k)
    try:
        tr = np.zeros(vc.vc_transcript_len(h), np.uint64)
        vc.vc_prove_pergate(h, np.ascontiguousarray(x), 3, tr)
        assert (tr == oracle_prove(w, k, x, 3)).all()
        y = x.copy()
        y[5] = (1 << 61) - 1
        with pytest.raises(vc.VcError) as e:
            vc.vc_prove_pergate(h, np.ascontiguousarray(y), 3, tr)
        assert e.value.status == vc.VC_EINVAL
    finally:
        vc.vc_circuit_destroy(h)
