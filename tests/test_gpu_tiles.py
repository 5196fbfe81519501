"""Tile shapes change the launch plan (chunk sizes, number of waves and of
persistent launches, tails) but never the transcript: every shape gives the
oracle's transcript.  The autotuner's choice is used by later circuits."""
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


def prove_with(widths, kinds, x, seed, tiles):
    h = vc.vc_circuit_create_tiles(widths, kinds, tiles)
    try:
        assert vc.vc_circuit_get_tiles(h) == tiles
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        vc.vc_prove(h, dev(x), seed, tr)
        vc.vc_circuit_sync(h)
        return to_np(tr)
    finally:
        vc.vc_circuit_destroy(h)


W = vc.VC_SPLIT_WIDEST
TILES = [(13, 12, 13, 10, W), (12, 11, 12, 9, 0), (9, 8, 10, 8, W), (5, 4, 3, 11, 12), (7, 7, 7, 8, 0),
         (1, 1, 1, 1, W), (13, 12, 6, 11, 13), (8, 12, 13, 9, 5), (2, 12, 13, 11, W)]


@pytest.mark.parametrize("family,logn", [("f2", 14), ("matmult", 4), ("f0", 3)])
def test_every_tile_shape_gives_the_oracle_transcript(family, logn):
    w, k = circuits.by_name(family, logn)
    x = I.job_inputs(family, logn, 21)
    want = oracle_prove(w, k, x, 33)
    for pr, gn, ln, ev, sp in TILES:
        tiles = {"pr_chunk_log": pr, "gn_chunk_log": gn, "line_chunk_log": ln, "eval_chunk_log": ev,
                 "pr_split_log": sp}
        got = prove_with(w, k, x, 33, tiles)
        assert (got == want).all(), tiles


def test_autotune_records_tiles_for_the_size_class():
    w, k = circuits.f2(12)
    best, ms = vc.vc_autotune(w, k, reps=2)
    assert ms > 0
    h = vc.vc_circuit_create(w, k)
    try:
        assert vc.vc_circuit_get_tiles(h) == best
        x = I.f2_inputs(12, 1 << 16, 4)
        tr = torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda")
        vc.vc_prove(h, dev(x), 8, tr)
        vc.vc_circuit_sync(h)
        assert (to_np(tr) == oracle_prove(w, k, x, 8)).all()
    finally:
        vc.vc_circuit_destroy(h)


def test_batch_autotune_tunes_the_merged_batch():
    """vc_autotune_batch times candidate configurations on the merged batch
    and records its choice for every member's size class; a batch of
    circuits built afterwards uses it and still gives the oracle's
    transcripts."""
    mix = [("f2", 9), ("f2", 11), ("matmult", 3), ("f0", 3), ("f2", 10), ("matmult", 4)]
    shapes = [circuits.by_name(f, n) for f, n in mix]
    best, ms = vc.vc_autotune_batch(shapes, reps=1)
    assert ms > 0
    hs = [vc.vc_circuit_create(w, k) for w, k in shapes]
    b = vc.vc_batch_create(hs)
    try:
        assert all(vc.vc_circuit_get_tiles(h) == best for h in hs)
        xs = [I.job_inputs(f, n, 60 + j) for j, (f, n) in enumerate(mix)]
        trs = [torch.empty(vc.vc_transcript_len(h), dtype=torch.int64, device="cuda") for h in hs]
        seeds = [90 + j for j in range(len(mix))]
        vc.vc_batch_prove(b, [dev(x) for x in xs], seeds, trs)
        vc.vc_batch_sync(b)
        for (w, k), x, s, tr in zip(shapes, xs, seeds, trs):
            assert (to_np(tr) == oracle_prove(w, k, x, s)).all()
    finally:
        vc.vc_batch_destroy(b)
        for h in hs:
            vc.vc_circuit_destroy(h)
    with pytest.raises(vc.VcError):
        vc.vc_autotune_batch([circuits.by_name("f2", 4)], reps=0)
