"""The convenience classes over the C ABI (paper_1202_1350_gb300.api):
Circuit, Batch and Server give the oracle's transcripts and verdicts."""
import numpy as np
import pytest

import oracle
from gpu_util import ensure_built, oracle_prove, to_np
from paper_1202_1350_gb300 import api, circuits
from paper_1202_1350_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
P = (1 << 61) - 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def test_circuit_roundtrip():
    c = api.Circuit.f2(9)
    try:
        x = I.f2_inputs(9, 1 << 16, 31)
        assert c.n_inputs == 512 and c.n_outputs == 1
        assert c.gates == circuits.non_input_gates(c.log_width)
        out = c.evaluate(x)
        assert int(out[0]) == sum(int(v) ** 2 for v in x) % P
        tr = c.prove(x, 5)
        assert (to_np(tr) == oracle_prove(*circuits.f2(9), x, 5)).all()
        assert c.verify(x, 5, tr)
        c.verify_input(x, 5, stream=torch.cuda.Stream())
        torch.cuda.synchronize()
        assert c.verify_transcript(5, tr)
        bad = tr.clone()
        bad[1] = (int(bad[1]) + 1) % P
        assert not c.verify(x, 5, bad)
        tr2, ok = c.prove_verify(x, 6)
        assert ok and (to_np(tr2) == oracle_prove(*circuits.f2(9), x, 6)).all()
    finally:
        c.close()


def test_batch_and_server():
    cs = [api.Circuit.f2(8), api.Circuit.matmult(3), api.Circuit.f0(3)]
    xs = [I.job_inputs("f2", 8, 1), I.job_inputs("matmult", 3, 2), I.job_inputs("f0", 3, 3)]
    b = api.Batch(cs)
    try:
        assert b.info()["n_members"] == 3
        trs = b.prove(xs, [11, 12, 13])
        for c, x, s, tr in zip(cs, xs, [11, 12, 13], trs):
            assert (to_np(tr) == oracle_prove(c.log_width, c.wiring, x, s)).all()
    finally:
        b.close()
        for c in cs:
            c.close()
    srv = api.Server()
    try:
        w, k = circuits.f2(10)
        x = torch.from_numpy(I.f2_inputs(10, 1 << 16, 4).view(np.int64).copy()).cuda()
        tr = torch.empty(len(oracle_prove(w, k, to_np(x), 9)), dtype=torch.int64, device="cuda")
        jid = srv.submit(w, k, x, 9, tr)
        info = srv.wait(jid)
        assert info["done"]
        assert (to_np(tr) == oracle_prove(w, k, to_np(x), 9)).all()
        assert srv.stats()["completed"] >= 1
    finally:
        srv.close()
