"""Layer values in mapped host memory (VC_VALUES_IN_HOST_MEMORY) or in host
memory passing through device slots (VC_VALUES_STAGED, copy-once-per-layer):
the same transcripts, accept bits and outputs as with device-resident values,
and less device memory."""
import numpy as np
import pytest

from gpu_util import ensure_built, oracle_prove, to_np
from paper_1202_1350_gb300 import circuits, vc
from paper_1202_1350_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.uint64)).view(np.int64).copy()).cuda()


def prove(h, x, seed, host_tr=False):
    n = vc.vc_transcript_len(h)
    if host_tr:
        tr = np.zeros(n, np.uint64)
        vc.vc_prove(h, np.ascontiguousarray(x), seed, tr)
        return tr
    tr = torch.empty(n, dtype=torch.int64, device="cuda")
    vc.vc_prove(h, dev(x), seed, tr)
    vc.vc_circuit_sync(h)
    return to_np(tr)


CASES = [("f2", 0), ("f2", 5), ("f2", 12), ("f0", 3), ("matmult", 3)]


@pytest.mark.parametrize("family,logn", CASES)
def test_host_values_equal_oracle(family, logn):
    w, k = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 80 + logn)
    h = vc.vc_circuit_create(w, k, host_values=True)
    try:
        want = oracle_prove(w, k, x, 13)
        assert (prove(h, x, 13) == want).all()
        assert (prove(h, x, 13, host_tr=True) == want).all()
        assert vc.vc_verify(h, dev(x), 13, dev(want))
    finally:
        vc.vc_circuit_destroy(h)


def test_host_values_explicit_and_pergate():
    w, k, ex = circuits.pattern_match(5, 2)
    x = I.pm_inputs(5, 2, 9)
    h = vc.vc_circuit_create(w, k, ex, host_values=True)
    try:
        want = oracle_prove(w, k, x, 5, explicit=ex)
        assert (prove(h, x, 5) == want).all()
        tr = torch.empty(len(want), dtype=torch.int64, device="cuda")
        vc.vc_prove_pergate(h, dev(x), 5, tr)
        vc.vc_circuit_sync(h)
        assert (to_np(tr) == want).all()
    finally:
        vc.vc_circuit_destroy(h)


def test_host_values_large_equal_device_and_smaller_footprint():
    w, k = circuits.f2(18)
    x = I.f2_inputs(18, 1 << 16, 4)
    hd = vc.vc_circuit_create(w, k)
    hh = vc.vc_circuit_create(w, k, host_values=True)
    try:
        assert (prove(hh, x, 77) == prove(hd, x, 77)).all()
        assert vc.vc_circuit_bytes(hh) < vc.vc_circuit_bytes(hd) - 8 * (1 << 19)
    finally:
        vc.vc_circuit_destroy(hd)
        vc.vc_circuit_destroy(hh)


def test_host_values_in_a_batch():
    specs = [("f2", 9), ("matmult", 2), ("f2", 4)]
    hs, xs = [], []
    for j, (fam, n) in enumerate(specs):
        w, k = circuits.by_name(fam, n)
        hs.append(vc.vc_circuit_create(w, k, host_values=(j != 1)))
        xs.append(I.job_inputs(fam, n, 90 + j))
    b = vc.vc_batch_create(hs)
    try:
        trs = [torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda") for h in hs]
        vc.vc_batch_prove(b, [dev(x) for x in xs], [3, 4, 5], trs)
        vc.vc_batch_sync(b)
        for j, (fam, n) in enumerate(specs):
            w, k = circuits.by_name(fam, n)
            assert (to_np(trs[j]) == oracle_prove(w, k, xs[j], 3 + j)).all()
    finally:
        vc.vc_batch_destroy(b)
        for h in hs:
            vc.vc_circuit_destroy(h)


def test_bad_flags_rejected():
    import ctypes
    w, k = circuits.f2(3)
    desc, keep = vc._desc_struct(w, k)
    h = ctypes.c_void_p()
    for flags in (6, 3, 5, 32, 10, 17, 18, 20, 24):
        assert vc.lib().vc_circuit_create_ex(ctypes.byref(desc), 0, flags, ctypes.byref(h)) == vc.VC_EINVAL


@pytest.mark.parametrize("family,logn", [("f2", 4), ("f2", 12), ("f0", 6), ("matmult", 3)])
def test_uploaded_inputs_equal_oracle(family, logn):
    """VC_INPUTS_UPLOAD: page-locked host inputs are copied to the device by
    the prover and by the verifier's input pass (each into its own buffer);
    the transcript equals the oracle's, both verifiers accept it and reject a
    changed one, a refilled host buffer is picked up by the next proof, and a
    non-canonical input is still reported."""
    P = (1 << 61) - 1
    w, k = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 90 + logn)
    h = vc.vc_circuit_create(w, k, upload=True)
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    try:
        assert vc.vc_circuit_get_info(h)["residency"] == 0
        xh = torch.from_numpy(np.ascontiguousarray(x, np.uint64).view(np.int64).copy()).pin_memory()
        n = vc.vc_transcript_len(h)
        tr = torch.empty(n, dtype=torch.int64, device="cuda")
        acc = torch.zeros(1, dtype=torch.int32, device="cuda")
        start = torch.cuda.Event()
        start.record(main)
        vc.vc_prove(h, xh, 5, tr)
        side.wait_event(start)
        vc.vc_verify_input(h, xh, 5, stream=side)
        main.wait_stream(side)
        vc.vc_verify_transcript(h, 5, tr, accept=acc)
        torch.cuda.synchronize()
        vc.vc_circuit_sync(h)
        assert (to_np(tr) == oracle_prove(w, k, x, 5)).all()
        assert int(acc.item()) == 1
        assert vc.vc_verify(h, xh, 5, tr)
        bad = tr.clone()
        bad[n // 2] = (int(bad[n // 2]) + 1) % P
        assert not vc.vc_verify(h, xh, 5, bad)
        x2 = I.job_inputs(family, logn, 190 + logn)
        xh.copy_(torch.from_numpy(np.ascontiguousarray(x2, np.uint64).view(np.int64).copy()))
        vc.vc_prove(h, xh, 6, tr)
        vc.vc_circuit_sync(h)
        assert (to_np(tr) == oracle_prove(w, k, x2, 6)).all()
        assert vc.vc_verify(h, xh, 6, tr)
        xh[0] = -1  # 2^64 - 1: not a field element
        with pytest.raises(vc.VcError) as e:
            vc.vc_prove(h, xh, 7, tr)  # asynchronous: latched, reported by the sync
            vc.vc_circuit_sync(h)
        assert e.value.status == vc.VC_EINVAL
        vc.vc_circuit_sync(h)
    finally:
        torch.cuda.synchronize()
        vc.vc_circuit_destroy(h)


STAGED = [("f2", 0), ("f2", 1), ("f2", 2), ("f2", 5), ("f2", 13), ("f0", 3), ("f0", 6), ("matmult", 2),
          ("matmult", 4)]


@pytest.mark.parametrize("mode", ["staged", "windowed"])
@pytest.mark.parametrize("family,logn", STAGED)
def test_staged_values_equal_oracle(family, logn, mode):
    """Copy-once-per-layer (staged) and windowed values: every transcript
    entry equals the oracle's (device and host transcripts, two proofs in a
    row on one handle), the verifier accepts it and vc_evaluate gives the
    outputs."""
    w, k = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 70 + logn)
    h = vc.vc_circuit_create(w, k, **{mode: True})
    try:
        for seed in (13, 14):
            want = oracle_prove(w, k, x, seed)
            assert (prove(h, x, seed) == want).all(), seed
            assert (prove(h, x, seed, host_tr=True) == want).all(), seed
        assert vc.vc_verify(h, dev(x), 14, dev(want))
        out = torch.empty(1 << w[0], dtype=torch.int64, device="cuda")
        vc.vc_evaluate(h, dev(x), out)
        assert (to_np(out) == want[:1 << w[0]]).all()
    finally:
        vc.vc_circuit_destroy(h)


def test_staged_values_large_equal_device_and_device_bytes():
    """F2 2^18 and F0 2^12 with staged values equal the device-resident
    proofs; the deep F0 circuit needs far less device memory (eight slots
    instead of 62 layers of values) and F2 less too (two slots for its wide
    layers of 2^18, 2^18 and 2^17 values).  Host-link bytes: every wide layer
    crosses once on the way out; F2's input layer comes back in once (its
    slot held layer 17 meanwhile); F0's wide layers come back at most once.
    Windowed values: the same device bytes (up to launch lists), the same
    proofs, no host link."""
    for fam, n, seed in (("f2", 18, 5), ("f0", 12, 6)):
        w, k = circuits.by_name(fam, n)
        x = I.job_inputs(fam, n, 40 + n)
        hd = vc.vc_circuit_create(w, k)
        hs = vc.vc_circuit_create(w, k, staged=True)
        hw = vc.vc_circuit_create(w, k, windowed=True)
        try:
            assert (prove(hs, x, seed) == prove(hd, x, seed)).all(), fam
            assert (prove(hw, x, seed) == prove(hd, x, seed)).all(), fam
            # the same slots and narrow layers (the launch lists differ a little)
            assert abs(vc.vc_circuit_bytes(hw) - vc.vc_circuit_bytes(hs)) <= 65536
            info = vc.vc_circuit_get_info(hw)
            assert info["link_bytes"] == 0 and info["residency"] == vc.VC_VALUES_WINDOWED
            assert vc.vc_circuit_get_info(hd)["link_bytes"] == 0
            link = vc.vc_circuit_get_info(hs)["link_bytes"]
            wide = 8 * sum(1 << s for s in w if 4 * (1 << s) > (1 << max(w)))
            if fam == "f2":
                assert wide == 8 * (2 * (1 << 18) + (1 << 17))
                assert link == wide + 8 * (1 << 18)
                assert vc.vc_circuit_bytes(hs) < vc.vc_circuit_bytes(hd)
            else:
                values = 8 * sum(1 << s for s in w)
                assert vc.vc_circuit_bytes(hs) < vc.vc_circuit_bytes(hd) - values // 2
                assert wide < link < 2 * wide
        finally:
            vc.vc_circuit_destroy(hd)
            vc.vc_circuit_destroy(hs)
            vc.vc_circuit_destroy(hw)


@pytest.mark.parametrize("mode", ["staged", "windowed"])
def test_staged_rejected_where_layers_are_read_in_place(mode):
    w, k = circuits.f2(6)
    h = vc.vc_circuit_create(w, k, **{mode: True})
    h2 = vc.vc_circuit_create(w, k)
    try:
        with pytest.raises(vc.VcError):
            vc.vc_batch_create([h, h2])
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        with pytest.raises(vc.VcError):
            vc.vc_prove_pergate(h, dev(I.f2_inputs(6, 1 << 16, 1)), 3, tr)
    finally:
        vc.vc_circuit_destroy(h)
        vc.vc_circuit_destroy(h2)
    wp, kp, ex = circuits.pattern_match(5, 2)
    with pytest.raises(vc.VcError):
        vc.vc_circuit_create(wp, kp, ex, **{mode: True})


def test_auto_residency_follows_the_memory_cap():
    """VC_VALUES_AUTO under the library's device-memory cap: device-resident
    values when the whole circuit fits, windowed values when only they fit,
    mapped host memory when neither does, and VC_ENOMEM below that; every
    choice gives the oracle's transcript.  F0 with 2^10 inputs (62 layers of
    2^11 values), where windowed values need far less device memory."""
    w, k = circuits.f0(10)
    x = I.job_inputs("f0", 10, 5)
    want = oracle_prove(w, k, x, 3)
    sizes = {}
    for mode, kw in ((0, {}), (vc.VC_VALUES_WINDOWED, {"windowed": True}), (vc.VC_VALUES_IN_HOST_MEMORY,
                                                                              {"host_values": True})):
        h = vc.vc_circuit_create(w, k, **kw)
        sizes[mode] = vc.vc_circuit_bytes(h)
        vc.vc_circuit_destroy(h)
    dev, stg, hst = sizes[0], sizes[vc.VC_VALUES_WINDOWED], sizes[vc.VC_VALUES_IN_HOST_MEMORY]
    assert hst < stg < dev
    used = vc.vc_get_memory_usage()[0]
    try:
        for cap, mode in ((dev, 0), ((stg + dev) // 2, vc.VC_VALUES_WINDOWED),
                          ((hst + stg) // 2, vc.VC_VALUES_IN_HOST_MEMORY)):
            vc.vc_set_memory_limit(used + cap, 0)
            h = vc.vc_circuit_create(w, k, auto=True)
            try:
                assert vc.vc_circuit_get_info(h)["residency"] == mode
                assert (prove(h, x, 3) == want).all(), mode
            finally:
                vc.vc_circuit_destroy(h)
        vc.vc_set_memory_limit(used + hst // 2, 0)
        with pytest.raises(vc.VcError) as e:
            vc.vc_circuit_create(w, k, auto=True)
        assert e.value.status == vc.VC_ENOMEM
    finally:
        vc.vc_set_memory_limit(0, 0)
    # explicit wirings skip the windowed step
    wp, kp, ex = circuits.pattern_match(5, 2)
    h = vc.vc_circuit_create(wp, kp, ex)
    dev_p = vc.vc_circuit_bytes(h)
    vc.vc_circuit_destroy(h)
    used = vc.vc_get_memory_usage()[0]
    try:
        vc.vc_set_memory_limit(used + dev_p - 1, 0)
        h = vc.vc_circuit_create(wp, kp, ex, auto=True)
        try:
            assert vc.vc_circuit_get_info(h)["residency"] == vc.VC_VALUES_IN_HOST_MEMORY
        finally:
            vc.vc_circuit_destroy(h)
    finally:
        vc.vc_set_memory_limit(0, 0)
