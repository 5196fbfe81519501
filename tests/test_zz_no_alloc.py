"""vc_evaluate_noalloc: circuit evaluation for callers that cannot allocate
device memory (their memory belongs to another allocator, or the implicit
synchronisation of cudaMalloc/cudaFree is unacceptable to them).

Its outputs must equal vc_evaluate's and the CPU oracle's evaluation (exact
field elements, so bit for bit) on two calls in a row, since every call reuses
one fixed device array that keeps the previous call's contents.  This file is
collected last on purpose."""
import numpy as np
import pytest

import oracle
from gpu_util import ensure_built, to_np
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


def reference_outputs(widths, kinds, xd):
    h = vc.vc_circuit_create(widths, kinds)
    try:
        out = torch.empty(1 << widths[0], dtype=torch.int64, device="cuda")
        vc.vc_evaluate(h, xd, out)
        return to_np(out)
    finally:
        vc.vc_circuit_destroy(h)


def oracle_outputs(widths, kinds, x):
    """Layer 0 of the CPU oracle's evaluation (independent of the CUDA path)."""
    return oracle.Circuit(widths, kinds).evaluate(np.asarray(x, np.uint64))[0]


@pytest.mark.parametrize("family,logn", [("f2", 10), ("f2", 18), ("f0", 5), ("matmult", 4), ("matmult", 6)])
def test_matches_vc_evaluate_on_two_calls(family, logn):
    widths, kinds = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 71)
    want = reference_outputs(widths, kinds, dev(x))
    assert (want == oracle_outputs(widths, kinds, x)).all()
    for call in range(2):
        xd = dev(x)
        out = torch.full((1 << widths[0],), -1, dtype=torch.int64, device="cuda")
        vc.vc_evaluate_noalloc(widths, kinds, xd, out)
        assert (to_np(out) == want).all(), f"call {call}"


def test_different_circuits_back_to_back():
    """A call after a larger one must not see the earlier call's values."""
    big_w, big_k = circuits.f2(18)
    small_w, small_k = circuits.f2(3)
    xb = dev(I.f2_inputs(18, 1 << 16, 1))
    xs = dev(I.f2_inputs(3, 1 << 16, 2))
    ob = torch.empty(1, dtype=torch.int64, device="cuda")
    os_ = torch.empty(1, dtype=torch.int64, device="cuda")
    vc.vc_evaluate_noalloc(big_w, big_k, xb, ob)
    vc.vc_evaluate_noalloc(small_w, small_k, xs, os_)
    assert (to_np(os_) == reference_outputs(small_w, small_k, xs)).all()
    assert (to_np(ob) == reference_outputs(big_w, big_k, xb)).all()
    assert (to_np(os_) == oracle_outputs(small_w, small_k, to_np(xs))).all()
    assert (to_np(ob) == oracle_outputs(big_w, big_k, to_np(xb))).all()


def test_rejects_what_it_cannot_do():
    widths, kinds = circuits.f2(20)  # intermediate layers need 2^21 - 2 > 2^20 elements
    xd = dev(I.f2_inputs(20, 1 << 16, 3))
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    with pytest.raises(vc.VcError) as e:
        vc.vc_evaluate_noalloc(widths, kinds, xd, out)
    assert e.value.status == vc.VC_EINVAL
    small_w, small_k = circuits.f2(4)
    x = I.f2_inputs(4, 1 << 16, 4)
    with pytest.raises(vc.VcError):  # host memory is not accepted
        vc.vc_evaluate_noalloc(small_w, small_k, np.ascontiguousarray(x), np.zeros(1, np.uint64))
    bad = x.copy()
    bad[3] = P
    with pytest.raises(vc.VcError) as e:  # non-canonical input
        vc.vc_evaluate_noalloc(small_w, small_k, dev(bad), out)
    assert e.value.status == vc.VC_EINVAL
    # the array is still usable afterwards
    vc.vc_evaluate_noalloc(small_w, small_k, dev(x), out)
    assert int(to_np(out)[0]) == sum(int(v) ** 2 for v in x) % P
