"""Host-side failure handling, made to happen on purpose without faulting the
GPU: an allocation refused by the library's memory budget (vc_circuit_create
and a served job that needs a new circuit report VC_ENOMEM, nothing leaks,
and the other jobs' transcripts still equal the oracle's), and a queued
served job cancelled before it reaches the device."""
import time

import numpy as np
import pytest

from gpu_util import ensure_built, oracle_prove, to_np
from paper_1202_1350_gb300 import Server, circuits, vc
from paper_1202_1350_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()
    yield
    vc.vc_set_memory_limit(0, 0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.uint64)).view(np.int64).copy()).cuda()


def test_circuit_create_refused_by_budget():
    widths, kinds = circuits.f2(16)
    used0 = vc.vc_get_memory_usage()
    vc.vc_set_memory_limit(used0[0] + (1 << 20), 0)
    try:
        with pytest.raises(vc.VcError) as e:
            vc.vc_circuit_create(widths, kinds)
        assert e.value.status == vc.VC_ENOMEM
        assert vc.vc_get_memory_usage() == used0  # nothing kept by the failed call
    finally:
        vc.vc_set_memory_limit(0, 0)
    h = vc.vc_circuit_create(widths, kinds)
    try:
        assert vc.vc_get_memory_usage()[0] > used0[0]
        x = I.f2_inputs(16, 1 << 16, 3)
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        vc.vc_prove(h, dev(x), 9, tr)
        vc.vc_circuit_sync(h)
        assert (to_np(tr) == oracle_prove(widths, kinds, x, 9)).all()
    finally:
        vc.vc_circuit_destroy(h)
    assert vc.vc_get_memory_usage() == used0


def test_served_job_refused_others_unaffected():
    srv = Server(max_batch=1, max_inflight=1)
    try:
        wa, ka = circuits.f2(10)
        xa = I.f2_inputs(10, 1 << 16, 4)
        ta = torch.empty(circuits.transcript_len(wa), dtype=torch.int64, device="cuda")
        assert srv.wait(srv.submit(wa, ka, dev(xa), 11, ta))["status"] == vc.VC_OK
        # no room for any new circuit: a job of a new shape is refused ...
        vc.vc_set_memory_limit(vc.vc_get_memory_usage()[0], 0)
        wb, kb = circuits.f2(12)
        xb = I.f2_inputs(12, 1 << 16, 5)
        tb = torch.empty(circuits.transcript_len(wb), dtype=torch.int64, device="cuda")
        assert srv.wait(srv.submit(wb, kb, dev(xb), 12, tb))["status"] == vc.VC_ENOMEM
        # ... while one of a pooled shape still runs and matches the oracle
        xc = I.f2_inputs(10, 1 << 16, 6)
        tc = torch.empty(circuits.transcript_len(wa), dtype=torch.int64, device="cuda")
        assert srv.wait(srv.submit(wa, ka, dev(xc), 13, tc))["status"] == vc.VC_OK
        assert (to_np(ta) == oracle_prove(wa, ka, xa, 11)).all()
        assert (to_np(tc) == oracle_prove(wa, ka, xc, 13)).all()
    finally:
        vc.vc_set_memory_limit(0, 0)
        srv.close()


def test_cancel_queued_job():
    srv = Server(max_batch=1, max_inflight=1)
    try:
        w, k = circuits.f2(18)
        n = 120
        xs = [dev(I.f2_inputs(18, 1 << 16, 100 + j)) for j in range(n)]
        trs = [torch.full((circuits.transcript_len(w),), -1, dtype=torch.int64, device="cuda") for _ in range(n)]
        torch.cuda.synchronize()
        # one job at a time on the device: submitted back to back, the last
        # one waits behind n - 1 proofs when it is cancelled
        jobs = [(srv.submit(w, k, xs[j], 200 + j, trs[j]), xs[j], trs[j]) for j in range(n)]
        last, _, last_tr = jobs[-1]
        srv.cancel(last)
        with pytest.raises(vc.VcError) as e:
            srv.cancel(10 ** 12)
        assert e.value.status == vc.VC_EINVAL
        infos = [srv.wait(jid) for jid, _, _ in jobs]
        assert infos[-1]["status"] == vc.VC_ECANCELED and infos[-1]["done"]
        assert all(i["status"] == vc.VC_OK for i in infos[:-1])
        assert bool((last_tr == -1).all().item())  # never written
        for j in (0, n - 2):
            jid, x, tr = jobs[j]
            assert (to_np(tr) == oracle_prove(w, k, to_np(x), 200 + j)).all()
        assert srv.stats()["cancelled"] == 1
        # a finished (not yet collected) job can no longer be cancelled
        x = I.f2_inputs(18, 1 << 16, 999)
        tr = torch.empty(circuits.transcript_len(w), dtype=torch.int64, device="cuda")
        jid = srv.submit(w, k, dev(x), 7, tr)
        time.sleep(0.5)
        with pytest.raises(vc.VcError) as e:
            srv.cancel(jid)
        assert e.value.status == vc.VC_EBUSY
        assert srv.wait(jid)["status"] == vc.VC_OK
    finally:
        srv.close()
