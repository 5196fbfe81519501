"""Helpers of the GPU tests: run the CUDA path through the C ABI and the oracle
on the same seeded inputs."""
import numpy as np

import oracle
from paper_1202_1350_gb300 import build, vc


def ensure_built():
    build.build()
    vc.lib()


def to_np(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


def gpu_prove(widths, kinds, x, seed, explicit=None):
    """Transcript from the CUDA path, device inputs and device transcript."""
    import torch
    h = vc.vc_circuit_create(widths, kinds, explicit, 0)
    try:
        n = vc.vc_transcript_len(h)
        xt = torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.uint64)).view(np.int64).copy()).cuda()
        tr = torch.empty(n, dtype=torch.int64, device="cuda")
        vc.vc_prove(h, xt, seed, tr)
        vc.vc_circuit_sync(h)
        return to_np(tr)
    finally:
        vc.vc_circuit_destroy(h)


def oracle_prove(widths, kinds, x, seed, explicit=None):
    c = oracle.Circuit(widths, kinds, explicit=explicit)
    return c.prove(np.asarray(x, np.uint64), seed)


def first_mismatch(a, b):
    bad = np.nonzero(a != b)[0]
    return None if len(bad) == 0 else int(bad[0])
