"""Convenience wrapper over the C ABI: a circuit handle with torch-tensor I/O.

Field elements travel as 64-bit torch tensors (int64 storage; every value is
below p < 2^63, so the bits are the same as uint64).
"""
from __future__ import annotations

import numpy as np

from . import circuits as _circuits
from . import vc as _vc


def _as_tensor(x, device):
    import torch
    if isinstance(x, torch.Tensor):
        return x
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint64)).view(np.int64)
    return torch.from_numpy(a.copy()).to(device)


class Circuit:
    def __init__(self, log_width, wiring, explicit=None, device: int = 0):
        self.log_width = [int(s) for s in log_width]
        self.wiring = [int(k) for k in wiring]
        self.device = device
        self.handle = _vc.vc_circuit_create(self.log_width, self.wiring, explicit, device)
        self.transcript_len = _vc.vc_transcript_len(self.handle)

    @classmethod
    def f2(cls, logn: int, device: int = 0):
        return cls(*_circuits.f2(logn), device=device)

    @classmethod
    def f0(cls, logn: int, device: int = 0):
        return cls(*_circuits.f0(logn), device=device)

    @classmethod
    def matmult(cls, logn: int, device: int = 0):
        return cls(*_circuits.matmult(logn), device=device)

    @property
    def n_inputs(self) -> int:
        return 1 << self.log_width[-1]

    @property
    def n_outputs(self) -> int:
        return 1 << self.log_width[0]

    @property
    def gates(self) -> int:
        return _circuits.non_input_gates(self.log_width)

    def new_transcript(self):
        import torch
        return torch.empty(self.transcript_len, dtype=torch.int64, device=f"cuda:{self.device}")

    def evaluate(self, inputs):
        import torch
        x = _as_tensor(inputs, f"cuda:{self.device}")
        out = torch.empty(self.n_outputs, dtype=torch.int64, device=x.device)
        _vc.vc_evaluate(self.handle, x, out, device=self.device)
        return out

    def prove(self, inputs, seed: int, transcript=None, sync: bool = True):
        x = _as_tensor(inputs, f"cuda:{self.device}")
        tr = self.new_transcript() if transcript is None else transcript
        _vc.vc_prove(self.handle, x, seed, tr, device=self.device)
        if sync:
            _vc.vc_circuit_sync(self.handle, device=self.device)
        return tr

    def verify(self, inputs, seed: int, transcript) -> bool:
        x = _as_tensor(inputs, f"cuda:{self.device}")
        return _vc.vc_verify(self.handle, x, seed, transcript, device=self.device)

    def prove_verify(self, inputs, seed: int, transcript=None):
        """Proof and verification in one graph launch; returns (transcript,
        accept bit)."""
        x = _as_tensor(inputs, f"cuda:{self.device}")
        tr = self.new_transcript() if transcript is None else transcript
        ok = _vc.vc_prove_verify(self.handle, x, seed, tr, device=self.device)
        return tr, ok

    def verify_input(self, inputs, seed: int, stream=None):
        """The verifier's input pass for `seed` (its coins and the inputs'
        multilinear extension at the final point), queued on `stream` (a torch
        stream; default: the current one) after the work already queued on the
        current stream; it may run beside a proof on this circuit.  The inputs
        (or their device copy) are held until verify_transcript, which waits
        for the pass."""
        import torch
        x = _as_tensor(inputs, f"cuda:{self.device}")
        cur = torch.cuda.current_stream(self.device)
        st = cur if stream is None else stream
        if st != cur:
            st.wait_stream(cur)
        _vc.vc_verify_input(self.handle, x, seed, stream=st, device=self.device)
        ev = torch.cuda.Event()
        ev.record(st)
        self._vin = (x, ev)

    def verify_transcript(self, seed: int, transcript, stream=None) -> bool:
        """The rest of the verification, after verify_input for the same seed,
        queued on `stream` (default: the current one) behind the input pass."""
        import torch
        st = torch.cuda.current_stream(self.device) if stream is None else stream
        vin = getattr(self, "_vin", None)
        if vin is not None:
            st.wait_event(vin[1])
        ok = _vc.vc_verify_transcript(self.handle, seed, transcript, stream=st, device=self.device)
        self._vin = None
        return ok

    def close(self):
        if getattr(self, "handle", None):
            _vc.vc_circuit_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A fixed set of distinct circuits proved by one set of merged launches."""

    def __init__(self, circuits):
        self.circuits = list(circuits)
        self.device = self.circuits[0].device
        self.handle = _vc.vc_batch_create([c.handle for c in self.circuits])

    def info(self) -> dict:
        return _vc.vc_batch_get_info(self.handle)

    def prove(self, inputs, seeds, transcripts=None, sync: bool = True):
        dev = f"cuda:{self.device}"
        xs = [_as_tensor(x, dev) for x in inputs]
        trs = [c.new_transcript() for c in self.circuits] if transcripts is None else transcripts
        _vc.vc_batch_prove(self.handle, xs, list(seeds), trs, device=self.device)
        if sync:
            _vc.vc_batch_sync(self.handle, device=self.device)
        return trs

    def close(self):
        if getattr(self, "handle", None):
            _vc.vc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Proof server: submit jobs (circuit shape, inputs, seed); results are
    written into the caller's transcript buffers (continuous batching under a
    device-memory cap)."""

    def __init__(self, device: int = 0, mem_cap_bytes: int = 0, max_batch: int = 0, max_inflight: int = 0,
                 pr_split_log: int = 0):
        self.device = device
        self.handle = _vc.vc_server_create(device, mem_cap_bytes, max_batch, max_inflight, pr_split_log)
        self._keep = {}  # job id -> buffers that must outlive the job

    def submit(self, log_width, wiring, inputs, seed: int, transcript) -> int:
        jid = _vc.vc_server_submit(self.handle, log_width, wiring, inputs, seed, transcript)
        self._keep[jid] = (inputs, transcript)
        return jid

    def wait(self, job_id: int) -> dict:
        info = _vc.vc_server_wait(self.handle, job_id)
        self._keep.pop(job_id, None)
        return info

    def poll(self, job_id: int) -> dict:
        info = _vc.vc_server_poll(self.handle, job_id)
        if info["done"]:
            self._keep.pop(job_id, None)
        return info

    def cancel(self, job_id: int) -> None:
        """Cancel a queued job; it then reports status VC_ECANCELED."""
        _vc.vc_server_cancel(self.handle, job_id)

    def stats(self) -> dict:
        return _vc.vc_server_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            _vc.vc_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
