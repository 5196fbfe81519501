"""The proof server: every job's transcript is the same in the mix as alone
(equal to the oracle's, or to a standalone vc_prove at sizes the oracle is
slow on), under admission by a device-memory cap and with launch sets in
flight concurrently."""
import numpy as np
import pytest

from gpu_util import ensure_built, oracle_prove, to_np
from paper_1202_1350_gb300 import Server, circuits, vc
from paper_1202_1350_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
P = (1 << 61) - 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.uint64)).view(np.int64).copy()).cuda()


def standalone(widths, kinds, x, seed):
    h = vc.vc_circuit_create(widths, kinds)
    try:
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        vc.vc_prove(h, dev(x), seed, tr)
        vc.vc_circuit_sync(h)
        return to_np(tr)
    finally:
        vc.vc_circuit_destroy(h)


MIX = [("f2", 5), ("f2", 10), ("matmult", 2), ("f2", 0), ("f0", 2), ("f2", 12), ("matmult", 4), ("f2", 7),
       ("f2", 10), ("f2", 5), ("matmult", 3), ("f2", 16)]


@pytest.mark.parametrize("split", [0, 13])
def test_server_mix_equals_alone(split):
    """Every job of a mix equals the oracle (small) or a standalone proof;
    split 13: the server's circuits use half-size chunks for product-weighted
    instances below 2^13 entries."""
    srv = Server(max_batch=4, max_inflight=3, pr_split_log=split)
    try:
        # inputs and transcript buffers first, then the submissions back to
        # back, so that jobs queue up behind the ones in flight
        prepared = []
        for k, (fam, logn) in enumerate(MIX * 2):
            w, kinds = circuits.by_name(fam, logn)
            x = I.job_inputs(fam, logn, 300 + k)
            tr = torch.empty(circuits.transcript_len(w), dtype=torch.int64, device="cuda")
            prepared.append((fam, logn, w, kinds, x, dev(x), 500 + k, tr))
        torch.cuda.synchronize()
        jobs = []
        for fam, logn, w, kinds, x, xd, seed, tr in prepared:
            jid = srv.submit(w, kinds, xd, seed, tr)
            jobs.append((jid, fam, logn, w, kinds, x, seed, tr))
        for jid, fam, logn, w, kinds, x, seed, tr in jobs:
            info = srv.wait(jid)
            assert info["done"] and info["status"] == 0
            assert info["submit_ns"] <= info["start_ns"] <= info["done_ns"]
            want = oracle_prove(w, kinds, x, seed) if logn <= 12 else standalone(w, kinds, x, seed)
            assert (to_np(tr) == want).all(), (fam, logn)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["pending"] == 0
        assert st["launch_sets"] < len(jobs)  # jobs were merged into launch sets
    finally:
        srv.close()


def test_server_host_buffers():
    srv = Server()
    try:
        jobs = []
        for k, (fam, logn) in enumerate(MIX[:6]):
            w, kinds = circuits.by_name(fam, logn)
            x = np.ascontiguousarray(I.job_inputs(fam, logn, 700 + k))
            tr = np.zeros(circuits.transcript_len(w), np.uint64)
            jobs.append((srv.submit(w, kinds, x, 900 + k, tr), w, kinds, x, 900 + k, tr))
        for jid, w, kinds, x, seed, tr in jobs:
            assert srv.wait(jid)["status"] == 0
            assert (tr == oracle_prove(w, kinds, x, seed)).all()
    finally:
        srv.close()


def test_server_memory_cap_admission_and_eviction():
    """A cap that holds only a few circuits: every job still completes, the
    resident bytes never exceed the cap, and idle circuits of other shapes
    are evicted to admit new shapes."""
    sizes = [9, 10, 11, 12]
    h = vc.vc_circuit_create(*circuits.f2(12))
    big = vc.vc_circuit_bytes(h)
    vc.vc_circuit_destroy(h)
    cap = int(big * 2.5)
    srv = Server(mem_cap_bytes=cap, max_batch=2, max_inflight=2)
    try:
        jobs = []
        for k in range(16):
            logn = sizes[k % 4]
            w, kinds = circuits.f2(logn)
            x = I.f2_inputs(logn, 1 << 16, 40 + k)
            tr = torch.empty(circuits.transcript_len(w), dtype=torch.int64, device="cuda")
            jobs.append((srv.submit(w, kinds, dev(x), k + 1, tr), w, kinds, x, k + 1, tr))
        for jid, w, kinds, x, seed, tr in jobs:
            assert srv.wait(jid)["status"] == 0
            assert (to_np(tr) == oracle_prove(w, kinds, x, seed)).all()
        st = srv.stats()
        assert st["peak_held_bytes"] <= cap
        assert st["circuits_evicted"] > 0
    finally:
        srv.close()


def test_server_rejects_oversized_and_explicit():
    w, kinds = circuits.f2(8)
    srv = Server(mem_cap_bytes=1 << 16)
    try:
        x = dev(I.f2_inputs(8, 1 << 16, 1))
        tr = torch.empty(circuits.transcript_len(w), dtype=torch.int64, device="cuda")
        with pytest.raises(vc.VcError) as e:
            srv.submit(w, kinds, x, 1, tr)
        assert e.value.status == vc.VC_EBUSY
        with pytest.raises(vc.VcError) as e:
            srv.submit([1, 2], [vc.EXPLICIT], x, 1, tr)
        assert e.value.status == vc.VC_EINVAL
    finally:
        srv.close()
    with pytest.raises(vc.VcError) as e:  # a split threshold beyond any layer width
        Server(pr_split_log=41)
    assert e.value.status == vc.VC_EINVAL


def test_server_noncanonical_job_reported_alone():
    w, kinds = circuits.f2(6)
    srv = Server(max_batch=8)
    try:
        xs = [I.f2_inputs(6, 1 << 16, s) for s in range(3)]
        xs[1][3] = P
        trs = [torch.empty(circuits.transcript_len(w), dtype=torch.int64, device="cuda") for _ in range(3)]
        ids = [srv.submit(w, kinds, dev(x), 10 + k, tr) for k, (x, tr) in enumerate(zip(xs, trs))]
        infos = [srv.wait(j) for j in ids]
        assert [i["status"] for i in infos] == [0, vc.VC_EINVAL, 0]
        for k in (0, 2):
            assert (to_np(trs[k]) == oracle_prove(w, kinds, xs[k], 10 + k)).all()
    finally:
        srv.close()


def test_server_overlaps_launch_sets():
    """A burst larger than one launch set keeps more than one set on the device."""
    w, kinds = circuits.f2(14)
    srv = Server(max_batch=4, max_inflight=3)
    try:
        x = dev(I.f2_inputs(14, 1 << 16, 5))
        trs = [torch.empty(circuits.transcript_len(w), dtype=torch.int64, device="cuda") for _ in range(24)]
        ids = [srv.submit(w, kinds, x, 100 + k, tr) for k, tr in enumerate(trs)]
        for j in ids:
            assert srv.wait(j)["status"] == 0
        st = srv.stats()
        assert st["max_jobs_in_flight"] > 4
        want = standalone(w, kinds, I.f2_inputs(14, 1 << 16, 5), 123)
        assert (to_np(trs[23]) == want).all()
    finally:
        srv.close()


def test_over_cap_job_proved_with_windowed_values():
    """A job whose circuit does not fit the memory cap with every layer on the
    device is proved with windowed values (the wide layers through device
    slots) instead of being refused; it equals the oracle, and jobs of other
    shapes around it are unaffected.  Below even the windowed footprint the
    submission is refused (VC_EBUSY)."""
    w, k = circuits.f0(8)
    hd = vc.vc_circuit_create(w, k)
    hs = vc.vc_circuit_create(w, k, windowed=True)
    resident, staged = vc.vc_circuit_bytes(hd), vc.vc_circuit_bytes(hs)
    vc.vc_circuit_destroy(hd)
    vc.vc_circuit_destroy(hs)
    assert staged < resident
    srv = Server(mem_cap_bytes=(staged + resident) // 2, max_batch=4, max_inflight=2)
    try:
        jobs = []
        for j, (fam, logn) in enumerate([("f2", 6), ("f0", 8), ("f2", 7), ("f0", 8), ("matmult", 2)]):
            wj, kj = circuits.by_name(fam, logn)
            x = I.job_inputs(fam, logn, 700 + j)
            host = j == 3  # one windowed job with a host transcript
            tr = np.zeros(circuits.transcript_len(wj), np.uint64) if host else \
                torch.empty(circuits.transcript_len(wj), dtype=torch.int64, device="cuda")
            jobs.append((srv.submit(wj, kj, dev(x), 40 + j, tr), wj, kj, x, 40 + j, tr))
        for jid, wj, kj, x, seed, tr in jobs:
            assert srv.wait(jid)["status"] == 0
            got = tr if isinstance(tr, np.ndarray) else to_np(tr)
            assert (got == oracle_prove(wj, kj, x, seed)).all()
    finally:
        srv.close()
    srv = Server(mem_cap_bytes=staged // 2)
    try:
        tr = torch.empty(circuits.transcript_len(w), dtype=torch.int64, device="cuda")
        with pytest.raises(vc.VcError) as e:
            srv.submit(w, k, dev(I.job_inputs("f0", 8, 1)), 1, tr)
        assert e.value.status == vc.VC_EBUSY
    finally:
        srv.close()
