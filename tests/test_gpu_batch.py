"""Batches (merged launches over several circuits) and CUDA-graph replay,
against the oracle on the same seeded inputs."""
import numpy as np
import pytest

from gpu_util import ensure_built, oracle_prove, to_np
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


def explicit_circuit(seed):
    """A small random explicit circuit: widths 2^3 <- 2^4 <- 2^5."""
    rng = np.random.default_rng(seed)
    widths = [3, 4, 5]
    layers = []
    for i in range(2):
        S, Sn = 1 << widths[i], 1 << widths[i + 1]
        layers.append((rng.integers(0, 2, S).astype(np.uint8), rng.integers(0, Sn, S).astype(np.uint32),
                       rng.integers(0, Sn, S).astype(np.uint32)))
    return widths, [vc.EXPLICIT, vc.EXPLICIT], layers


JOBS = [("f2", 10), ("f2", 3), ("matmult", 3), ("f0", 3), ("f2", 0), ("explicit", 0), ("f2", 13)]


def make_job(fam, logn, k):
    if fam == "explicit":
        w, kinds, ex = explicit_circuit(k)
        x = I.f2_inputs(w[-1], P, 40 + k)
        return w, kinds, ex, x
    w, kinds = circuits.by_name(fam, logn)
    return w, kinds, None, I.job_inputs(fam, logn, 40 + k)


def test_batch_mixed_families_repeated():
    """Every member of a mixed batch equals its oracle transcript, over
    several calls (the first captures the graph, the others replay it)."""
    specs = [make_job(f, n, k) for k, (f, n) in enumerate(JOBS)]
    hs = [vc.vc_circuit_create(w, k, ex) for w, k, ex, _ in specs]
    b = vc.vc_batch_create(hs)
    try:
        for call in range(3):
            xs, seeds, trs = [], [], []
            for j, (w, k, ex, x) in enumerate(specs):
                x = x if call == 0 else (x + call * (j + 1)) % P
                xs.append(x)
                seeds.append(1000 * call + j)
                trs.append(torch.empty(vc.vc_transcript_len(hs[j]), dtype=torch.int64, device="cuda"))
            vc.vc_batch_prove(b, [dev(x) for x in xs], seeds, trs)
            vc.vc_batch_sync(b)
            for j, (w, k, ex, _) in enumerate(specs):
                want = oracle_prove(w, k, xs[j], seeds[j], explicit=ex)
                assert (to_np(trs[j]) == want).all(), (call, JOBS[j])
    finally:
        vc.vc_batch_destroy(b)
        for h in hs:
            vc.vc_circuit_destroy(h)


def test_large_batch_final_reduction_paths():
    """A batch with more rounds than one final-reduction launch has warps
    (80 F2 circuits of 2^8..2^12 inputs plus MatMult members, about 12 K
    rounds): rounds with many chunk partials are summed a warp each, the rest
    a thread each.  Every member equals its standalone proof; a sample equals
    the oracle's transcript."""
    shapes = [("f2", 8 + (j % 5)) for j in range(80)] + [("matmult", 3), ("matmult", 4)]
    specs = [make_job(f, n, k) for k, (f, n) in enumerate(shapes)]
    hs = [vc.vc_circuit_create(w, k, ex) for w, k, ex, _ in specs]
    rounds = sum(vc.vc_circuit_get_info(h)["n_rounds"] for h in hs)
    assert rounds > 152 * 8 * 8
    b = vc.vc_batch_create(hs)
    try:
        trs = [torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda") for h in hs]
        vc.vc_batch_prove(b, [dev(x) for *_, x in specs], [300 + j for j in range(len(hs))], trs)
        vc.vc_batch_sync(b)
        for j, (w, k, ex, x) in enumerate(specs):
            one = torch.empty_like(trs[j])
            vc.vc_prove(hs[j], dev(x), 300 + j, one)
            vc.vc_circuit_sync(hs[j])
            assert (to_np(trs[j]) == to_np(one)).all(), shapes[j]
            if j % 20 == 0 or shapes[j][0] == "matmult":
                assert (to_np(trs[j]) == oracle_prove(w, k, x, 300 + j, explicit=ex)).all(), shapes[j]
    finally:
        vc.vc_batch_destroy(b)
        for h in hs:
            vc.vc_circuit_destroy(h)


def test_batch_host_pointers():
    """Host inputs and host transcripts: synchronous form."""
    specs = [make_job(f, n, k) for k, (f, n) in enumerate(JOBS[:4])]
    hs = [vc.vc_circuit_create(w, k, ex) for w, k, ex, _ in specs]
    b = vc.vc_batch_create(hs)
    try:
        xs = [np.ascontiguousarray(x) for *_, x in specs]
        trs = [np.zeros(vc.vc_transcript_len(h), np.uint64) for h in hs]
        vc.vc_batch_prove(b, xs, [7, 8, 9, 10], trs)
        for j, (w, k, ex, x) in enumerate(specs):
            assert (trs[j] == oracle_prove(w, k, x, 7 + j, explicit=ex)).all()
    finally:
        vc.vc_batch_destroy(b)
        for h in hs:
            vc.vc_circuit_destroy(h)


def test_batch_of_equal_shapes_shares_launches():
    """n circuits of one shape cost the launches of one proof."""
    w, k = circuits.f2(10)
    hs = [vc.vc_circuit_create(w, k) for _ in range(8)]
    b = vc.vc_batch_create(hs)
    try:
        single = vc.vc_circuit_get_info(hs[0])["prove_launches"]
        info = vc.vc_batch_get_info(b)
        assert info["n_members"] == 8
        assert info["prove_launches"] == single
        assert info["gates"] == 8 * circuits.non_input_gates(w)
        xs = [I.f2_inputs(10, 1 << 20, s) for s in range(8)]
        trs = [torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda") for h in hs]
        vc.vc_batch_prove(b, [dev(x) for x in xs], list(range(50, 58)), trs)
        vc.vc_batch_sync(b)
        for j in range(8):
            assert (to_np(trs[j]) == oracle_prove(w, k, xs[j], 50 + j)).all()
    finally:
        vc.vc_batch_destroy(b)
        for h in hs:
            vc.vc_circuit_destroy(h)


def test_batch_noncanonical_member_reported():
    w, k = circuits.f2(5)
    hs = [vc.vc_circuit_create(w, k) for _ in range(3)]
    b = vc.vc_batch_create(hs)
    try:
        xs = [I.f2_inputs(5, 1 << 16, s) for s in range(3)]
        xs[1][7] = P
        trs = [torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda") for h in hs]
        vc.vc_batch_prove(b, [dev(x) for x in xs], [1, 2, 3], trs)
        with pytest.raises(vc.VcError) as e:
            vc.vc_batch_sync(b)
        assert e.value.status == vc.VC_EINVAL
        vc.vc_batch_sync(b)  # cleared
        # the other members are unaffected
        for j in (0, 2):
            assert (to_np(trs[j]) == oracle_prove(w, k, xs[j], j + 1)).all()
    finally:
        vc.vc_batch_destroy(b)
        for h in hs:
            vc.vc_circuit_destroy(h)


def test_batch_create_rejects_duplicates():
    w, k = circuits.f2(4)
    h = vc.vc_circuit_create(w, k)
    try:
        with pytest.raises(vc.VcError) as e:
            vc.vc_batch_create([h, h])
        assert e.value.status == vc.VC_EINVAL
    finally:
        vc.vc_circuit_destroy(h)


def test_noncanonical_matmult_input_reported():
    """MATMULT input layers are checked by the plan's own input check."""
    w, k = circuits.matmult(3)
    x = I.matmult_inputs(3, 1 << 10, 4)
    x[5] = P
    h = vc.vc_circuit_create(w, k)
    try:
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        vc.vc_prove(h, dev(x), 1, tr)
        with pytest.raises(vc.VcError) as e:
            vc.vc_circuit_sync(h)
        assert e.value.status == vc.VC_EINVAL
    finally:
        vc.vc_circuit_destroy(h)


def test_stage_events_recapture():
    """Setting stage events re-captures the graph with event-record nodes;
    the transcript is unchanged and every stage has a non-negative time."""
    w, k = circuits.f2(12)
    x = I.f2_inputs(12, 1 << 20, 9)
    h = vc.vc_circuit_create(w, k)
    try:
        tr1 = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        vc.vc_prove(h, dev(x), 77, tr1)
        vc.vc_circuit_sync(h)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * vc.NUM_STAGES)]
        evs[2 * vc.STAGES.index("build")] = None  # a skipped mark
        vc.vc_circuit_set_stage_events(h, evs)
        tr2 = torch.empty_like(tr1)
        vc.vc_prove(h, dev(x), 77, tr2)
        vc.vc_circuit_sync(h)
        torch.cuda.synchronize()
        for name in ("proof", "tables", "eval", "waves", "final"):  # the stages F2 has work in
            s = vc.STAGES.index(name)
            assert evs[2 * s].elapsed_time(evs[2 * s + 1]) >= 0.0
        vc.vc_circuit_set_stage_events(h, None)
        tr3 = torch.empty_like(tr1)
        vc.vc_prove(h, dev(x), 77, tr3)
        vc.vc_circuit_sync(h)
        assert (to_np(tr1) == to_np(tr2)).all() and (to_np(tr1) == to_np(tr3)).all()
        assert (to_np(tr1) == oracle_prove(w, k, x, 77)).all()
    finally:
        vc.vc_circuit_destroy(h)
