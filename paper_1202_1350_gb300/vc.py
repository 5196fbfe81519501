"""Thin ctypes binding of the C ABI in include/vc.h (argument marshalling only).

Every function keeps the C name.  Array arguments may be torch tensors (int64
or uint64, CPU or CUDA, contiguous) or numpy uint64 arrays; the library itself
decides host vs device from the pointer.  `stream` defaults to PyTorch's
current stream on the circuit's device.  There is no CPU fallback: if the CUDA
library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

P = (1 << 61) - 1
SQUARE, TREE, MATMULT, F0_FIRST, F0_PAIR, F0_FINAL, EXPLICIT = range(7)

VC_OK, VC_EINVAL, VC_ENOMEM, VC_ECUDA, VC_ETIMEOUT, VC_EBUSY, VC_ECANCELED = range(7)
_STATUS = {0: "VC_OK", 1: "VC_EINVAL", 2: "VC_ENOMEM", 3: "VC_ECUDA", 4: "VC_ETIMEOUT", 5: "VC_EBUSY",
           6: "VC_ECANCELED"}


class VcError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}")
        self.status = status


_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class _Desc(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_uint32),
                ("log_width", _u32p),
                ("wiring", _u32p),
                ("gate_type", ctypes.POINTER(_u8p)),
                ("in1", ctypes.POINTER(_u32p)),
                ("in2", ctypes.POINTER(_u32p))]


NUM_STAGES = 8
STAGES = ("proof", "tables", "eval", "waves", "wavesn", "build", "tabwaves", "final")


class CircuitInfo(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_uint32), ("n_rounds", ctypes.c_uint32),
                ("transcript_len", ctypes.c_uint64), ("gates", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("prove_launches", ctypes.c_uint32),
                ("verify_launches", ctypes.c_uint32), ("wave_tasks", ctypes.c_uint32),
                ("verify2_launches", ctypes.c_uint32), ("link_bytes", ctypes.c_uint64),
                ("residency", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_members", ctypes.c_uint32), ("prove_launches", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64), ("gates", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("mem_cap_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("pr_split_log", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class JobInfo(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("submit_ns", ctypes.c_uint64),
                ("start_ns", ctypes.c_uint64), ("done_ns", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("launch_sets", ctypes.c_uint64),
                ("circuits_created", ctypes.c_uint64), ("circuits_evicted", ctypes.c_uint64),
                ("held_bytes", ctypes.c_uint64), ("peak_held_bytes", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("max_jobs_in_flight", ctypes.c_uint32), ("cancelled", ctypes.c_uint32)]


VC_SPLIT_WIDEST = 0xFFFFFFFF


class TileConfig(ctypes.Structure):
    _fields_ = [("pr_chunk_log", ctypes.c_uint32), ("gn_chunk_log", ctypes.c_uint32),
                ("line_chunk_log", ctypes.c_uint32), ("eval_chunk_log", ctypes.c_uint32),
                ("pr_split_log", ctypes.c_uint32)]


_lock = threading.Lock()
_lib = None
_shapes = {}  # handle -> (inputs, outputs, transcript length), for size checks


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libvc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with `python -m paper_1202_1350_gb300.build` "
                                   "(there is no CPU fallback)")
            L = ctypes.CDLL(path)
            vp = ctypes.c_void_p
            st = ctypes.c_int
            L.vc_circuit_create.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.POINTER(vp)]
            L.vc_circuit_create_ex.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(vp)]
            L.vc_circuit_destroy.argtypes = [vp]
            L.vc_transcript_len.argtypes = [vp, _u64p]
            L.vc_circuit_bytes.argtypes = [vp, _u64p]
            L.vc_evaluate.argtypes = [vp, vp, vp, vp]
            L.vc_prove.argtypes = [vp, vp, ctypes.c_uint64, vp, vp]
            L.vc_prove_pergate.argtypes = [vp, vp, ctypes.c_uint64, vp, vp]
            L.vc_f2sp_create.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(vp)]
            L.vc_f2sp_destroy.argtypes = [vp]
            L.vc_f2sp_prove.argtypes = [vp, vp, vp, vp]
            L.vc_f2sp_verify_begin.argtypes = [vp, ctypes.c_uint64, vp]
            L.vc_f2sp_verify_absorb.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint64, vp]
            L.vc_f2sp_verify_absorb_async.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint64, vp]
            L.vc_f2sp_verify_end.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int),
                                             vp]
            L.vc_circuit_sync.argtypes = [vp, vp]
            L.vc_verify.argtypes = [vp, vp, ctypes.c_uint64, vp, ctypes.POINTER(ctypes.c_int), vp]
            L.vc_verify_input.argtypes = [vp, vp, ctypes.c_uint64, vp]
            L.vc_verify_transcript.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(ctypes.c_int), vp]
            L.vc_prove_verify.argtypes = [vp, vp, ctypes.c_uint64, vp, ctypes.POINTER(ctypes.c_int), vp]
            L.vc_prove_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), _u64p, ctypes.POINTER(vp),
                                         ctypes.c_int, vp]
            L.vc_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
            L.vc_batch_destroy.argtypes = [vp]
            L.vc_batch_prove.argtypes = [vp, ctypes.POINTER(vp), _u64p, ctypes.POINTER(vp), vp]
            L.vc_batch_sync.argtypes = [vp, vp]
            L.vc_batch_get_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
            L.vc_server_create.argtypes = [ctypes.c_int, ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
            L.vc_server_destroy.argtypes = [vp]
            L.vc_server_submit.argtypes = [vp, ctypes.POINTER(_Desc), vp, ctypes.c_uint64, vp,
                                           ctypes.POINTER(ctypes.c_uint64)]
            L.vc_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(JobInfo)]
            L.vc_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(JobInfo)]
            L.vc_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
            L.vc_server_cancel.argtypes = [vp, ctypes.c_uint64]
            L.vc_set_memory_limit.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.vc_get_memory_usage.argtypes = [_u64p, _u64p]
            L.vc_autotune.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.c_int, ctypes.POINTER(TileConfig),
                                      ctypes.POINTER(ctypes.c_double)]
            L.vc_autotune_batch.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(TileConfig), ctypes.POINTER(ctypes.c_double)]
            L.vc_circuit_create_tiles.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.POINTER(TileConfig),
                                                  ctypes.POINTER(vp)]
            L.vc_circuit_get_tiles.argtypes = [vp, ctypes.POINTER(TileConfig)]
            L.vc_field_mul.argtypes = [vp, vp, vp, ctypes.c_uint64, vp]
            L.vc_field_mul_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                            ctypes.POINTER(ctypes.c_double)]
            L.vc_circuit_set_stage_events.argtypes = [vp, ctypes.POINTER(vp)]
            L.vc_circuit_get_info.argtypes = [vp, ctypes.POINTER(CircuitInfo)]
            L.vc_evaluate_noalloc.argtypes = [ctypes.POINTER(_Desc), vp, vp, vp]
            L.vc_evaluate_noalloc.restype = st
            L.vc_status_string.argtypes = [ctypes.c_int]
            L.vc_status_string.restype = ctypes.c_char_p
            for name in ("vc_circuit_create", "vc_circuit_destroy", "vc_transcript_len", "vc_circuit_bytes",
                         "vc_evaluate", "vc_prove", "vc_circuit_sync", "vc_verify", "vc_prove_batch",
                         "vc_field_mul", "vc_field_mul_rate", "vc_circuit_set_stage_events",
                         "vc_circuit_get_info", "vc_batch_create", "vc_batch_destroy", "vc_batch_prove",
                         "vc_batch_sync", "vc_batch_get_info", "vc_server_create", "vc_server_destroy",
                         "vc_server_submit", "vc_server_poll", "vc_server_wait", "vc_server_get_stats",
                         "vc_server_cancel", "vc_set_memory_limit", "vc_get_memory_usage", "vc_autotune",
                         "vc_autotune_batch", "vc_circuit_create_tiles", "vc_circuit_get_tiles", "vc_prove_pergate",
                         "vc_circuit_create_ex", "vc_f2sp_create", "vc_f2sp_destroy", "vc_f2sp_prove",
                         "vc_f2sp_verify_begin", "vc_f2sp_verify_absorb", "vc_f2sp_verify_absorb_async",
                         "vc_f2sp_verify_end", "vc_verify_input", "vc_verify_transcript", "vc_prove_verify"):
                getattr(L, name).restype = st
            _lib = L
    return _lib


def header_functions() -> list:
    """Function names declared in include/vc.h."""
    hdr = os.path.join(_build.INCLUDE, "vc.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:vc_status|const\s+char\s*\*)\s*(vc_\w+)\s*\(", text, re.M)))


def _check(status: int, where: str):
    if status != VC_OK:
        raise VcError(status, where)


def _ptr(x):
    """Raw address of a contiguous torch tensor or numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"] or x.dtype.itemsize != 8:
            raise ValueError("numpy arrays must be contiguous 64-bit")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous() or x.element_size() != 8:
            raise ValueError("tensors must be contiguous 64-bit")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _numel(x) -> int:
    return int(x.size if isinstance(x, np.ndarray) else x.numel())


_current_stream = None  # device -> raw handle of torch's current stream (resolved once)


def _stream(stream, device: int):
    """Raw cudaStream_t of `stream` (a torch stream or an int), else torch's
    current stream on `device` (None without CUDA: the legacy default stream)."""
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    global _current_stream
    if _current_stream is None:
        _current_stream = lambda d: None
        try:
            import torch
            if torch.cuda.is_available():
                raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
                _current_stream = raw if raw is not None else (lambda d: torch.cuda.current_stream(d).cuda_stream)
        except Exception:
            pass
    return _current_stream(device)


# --- C ABI ----------------------------------------------------------------------------

VC_VALUES_IN_HOST_MEMORY = 1
VC_VALUES_STAGED = 2
VC_VALUES_AUTO = 4
VC_VALUES_WINDOWED = 8
VC_INPUTS_UPLOAD = 16


def vc_circuit_create(log_width, wiring, explicit=None, device: int = 0, host_values: bool = False,
                      staged: bool = False, auto: bool = False, windowed: bool = False, upload: bool = False):
    """Returns an opaque handle (int).  explicit: per-layer (type, in1, in2) or
    None.  host_values: keep the layer values in mapped host memory; staged:
    keep the wide layers in host memory and pass them through device slots
    (copy-once-per-layer); windowed: the wide layers through device slots
    only, each iteration run while its layers are there; auto: the first of
    device memory, windowed and mapped host memory whose memory can be had
    (vc_circuit_get_info's "residency" says which); upload (device-resident
    values only): page-locked host inputs are copied to the device by one
    transfer per call instead of being read in place."""
    lw = [int(x) for x in log_width]
    kinds = [int(k) for k in wiring]
    d = len(kinds)
    if len(lw) != d + 1:
        raise ValueError("log_width must have len(wiring) + 1 entries")
    keep = []
    lw_a = (ctypes.c_uint32 * (d + 1))(*lw)
    k_a = (ctypes.c_uint32 * max(d, 1))(*kinds)
    desc = _Desc(d, ctypes.cast(lw_a, _u32p), ctypes.cast(k_a, _u32p), None, None, None)
    if explicit is not None:
        tys = (_u8p * d)()
        i1s = (_u32p * d)()
        i2s = (_u32p * d)()
        for i, layer in enumerate(explicit):
            if layer is None:
                continue
            ty = np.ascontiguousarray(layer[0], dtype=np.uint8)
            a = np.ascontiguousarray(layer[1], dtype=np.uint32)
            b = np.ascontiguousarray(layer[2], dtype=np.uint32)
            keep += [ty, a, b]
            tys[i] = ty.ctypes.data_as(_u8p)
            i1s[i] = a.ctypes.data_as(_u32p)
            i2s[i] = b.ctypes.data_as(_u32p)
        desc.gate_type = tys
        desc.in1 = i1s
        desc.in2 = i2s
    h = ctypes.c_void_p()
    if host_values or staged or auto or windowed or upload:
        flags = (VC_VALUES_AUTO if auto else VC_VALUES_WINDOWED if windowed else
                 VC_VALUES_STAGED if staged else VC_VALUES_IN_HOST_MEMORY if host_values else 0)
        flags |= VC_INPUTS_UPLOAD if upload else 0
        _check(lib().vc_circuit_create_ex(ctypes.byref(desc), device, flags, ctypes.byref(h)),
               "vc_circuit_create_ex")
    else:
        _check(lib().vc_circuit_create(ctypes.byref(desc), device, ctypes.byref(h)), "vc_circuit_create")
    del keep
    n = ctypes.c_uint64()
    _check(lib().vc_transcript_len(h, ctypes.byref(n)), "vc_transcript_len")
    _shapes[h.value] = (1 << lw[-1], 1 << lw[0], n.value)
    return h.value


def _need(x, n: int, what: str):
    if x is None or _numel(x) < n:
        raise ValueError(f"{what} needs at least {n} elements")


def vc_circuit_destroy(h):
    _check(lib().vc_circuit_destroy(h), "vc_circuit_destroy")
    _shapes.pop(h, None)


def vc_transcript_len(h) -> int:
    n = ctypes.c_uint64()
    _check(lib().vc_transcript_len(h, ctypes.byref(n)), "vc_transcript_len")
    return n.value


def vc_circuit_bytes(h) -> int:
    n = ctypes.c_uint64()
    _check(lib().vc_circuit_bytes(h, ctypes.byref(n)), "vc_circuit_bytes")
    return n.value


def vc_evaluate(h, inputs, outputs, stream=None, device: int = 0):
    nin, nout, _ = _shapes[h]
    _need(inputs, nin, "inputs")
    _need(outputs, nout, "outputs")
    _check(lib().vc_evaluate(h, _ptr(inputs), _ptr(outputs), _stream(stream, device)), "vc_evaluate")
    return outputs


def vc_prove(h, inputs, seed: int, transcript, stream=None, device: int = 0):
    nin, _, ntr = _shapes[h]
    _need(inputs, nin, "inputs")
    _need(transcript, ntr, "transcript")
    _check(lib().vc_prove(h, _ptr(inputs), seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript),
                          _stream(stream, device)), "vc_prove")
    return transcript


def vc_prove_pergate(h, inputs, seed: int, transcript, stream=None, device: int = 0):
    """The same proof by the paper's per-gate method (one thread per gate per
    round); the transcript equals vc_prove's."""
    nin, _, ntr = _shapes[h]
    _need(inputs, nin, "inputs")
    _need(transcript, ntr, "transcript")
    _check(lib().vc_prove_pergate(h, _ptr(inputs), seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript),
                                  _stream(stream, device)), "vc_prove_pergate")
    return transcript


# ---- special-purpose non-interactive F2 protocol ---------------------------------------

def vc_f2sp_create(v: int, h: int, device: int = 0):
    s = ctypes.c_void_p()
    _check(lib().vc_f2sp_create(v, h, device, ctypes.byref(s)), "vc_f2sp_create")
    _shapes[("f2sp", s.value)] = (v, h)
    return s.value


def vc_f2sp_destroy(s):
    _shapes.pop(("f2sp", s), None)
    _check(lib().vc_f2sp_destroy(s), "vc_f2sp_destroy")


F2SP_FACTORS = (9, 3, 25, 5, 7, 11, 13, 31, 41, 61)


def f2sp_valid_h(h: int) -> bool:
    """h of the special-purpose protocol: a product of distinct members of
    {3 or 9, 5 or 25, 7, 11, 13, 31, 41, 61}, at most VC_F2SP_MAX_H (7000)."""
    if h < 1 or h > 7000 or (P - 1) % (2 * h):
        return False
    for pr in (3, 5, 7, 11, 13, 31, 41, 61):
        pp = 1
        while h % pr == 0:
            h //= pr
            pp *= pr
        if pp > 61:
            return False
    return h == 1


def vc_f2sp_prove(s, a, proof, stream=None, device: int = 0):
    """proof: 2h entries (host or device), written synchronously."""
    v, h = _shapes[("f2sp", s)]
    _need(a, v * h, "a")
    _need(proof, 2 * h, "proof")
    _check(lib().vc_f2sp_prove(s, _ptr(a), _ptr(proof), _stream(stream, device)), "vc_f2sp_prove")
    return proof


def vc_f2sp_verify_begin(s, seed: int, stream=None, device: int = 0):
    _check(lib().vc_f2sp_verify_begin(s, seed & 0xFFFFFFFFFFFFFFFF, _stream(stream, device)), "vc_f2sp_verify_begin")


def vc_f2sp_verify_absorb(s, rows, first_row: int, nrows: int, stream=None, device: int = 0):
    v, h = _shapes[("f2sp", s)]
    _need(rows, nrows * h, "rows")
    _check(lib().vc_f2sp_verify_absorb(s, _ptr(rows), first_row, nrows, _stream(stream, device)),
           "vc_f2sp_verify_absorb")


def vc_f2sp_verify_absorb_async(s, rows, first_row: int, nrows: int, stream=None, device: int = 0):
    """Host rows: returns once the previous call's rows are copied (alternate
    at least two host buffers)."""
    v, h = _shapes[("f2sp", s)]
    _need(rows, nrows * h, "rows")
    _check(lib().vc_f2sp_verify_absorb_async(s, _ptr(rows), first_row, nrows, _stream(stream, device)),
           "vc_f2sp_verify_absorb_async")


def vc_f2sp_verify_end(s, proof, stream=None, device: int = 0):
    """Returns (accept, F2 answer)."""
    v, h = _shapes[("f2sp", s)]
    _need(proof, 2 * h, "proof")
    f2 = ctypes.c_uint64()
    acc = ctypes.c_int()
    _check(lib().vc_f2sp_verify_end(s, _ptr(proof), ctypes.byref(f2), ctypes.byref(acc), _stream(stream, device)),
           "vc_f2sp_verify_end")
    return bool(acc.value), f2.value


def vc_circuit_sync(h, stream=None, device: int = 0):
    _check(lib().vc_circuit_sync(h, _stream(stream, device)), "vc_circuit_sync")


def vc_verify_input(h, inputs, seed: int, stream=None, device: int = 0):
    """The verifier's input pass for `seed` (coins and the input's MLE at the
    final point): inputs on the device or in page-locked host memory, read in
    place; asynchronous.  May run on another stream beside a proof."""
    nin, _, _ = _shapes[h]
    _need(inputs, nin, "inputs")
    _check(lib().vc_verify_input(h, _ptr(inputs), seed & 0xFFFFFFFFFFFFFFFF, _stream(stream, device)),
           "vc_verify_input")


def vc_verify_transcript(h, seed: int, transcript, stream=None, device: int = 0, accept=None) -> bool:
    """The rest of the verification, after vc_verify_input for the same seed.
    Returns the accept bit; with `accept` (a CUDA int32 tensor) the call is
    asynchronous where vc_verify's would be and the bit is written there."""
    _, _, ntr = _shapes[h]
    _need(transcript, ntr, "transcript")
    if accept is not None:
        if accept.element_size() != 4 or accept.numel() < 1:
            raise ValueError("accept must be an int32 tensor")
        _check(lib().vc_verify_transcript(h, seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript),
                                          ctypes.cast(ctypes.c_void_p(accept.data_ptr()), ctypes.POINTER(ctypes.c_int)),
                                          _stream(stream, device)), "vc_verify_transcript")
        return None
    acc = ctypes.c_int(0)
    _check(lib().vc_verify_transcript(h, seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript), ctypes.byref(acc),
                                      _stream(stream, device)), "vc_verify_transcript")
    return bool(acc.value)


def vc_prove_verify(h, inputs, seed: int, transcript, stream=None, device: int = 0, accept=None):
    """Prove and verify in one graph launch: writes the transcript and returns
    the accept bit; with `accept` (a CUDA int32 tensor) the call is
    asynchronous where vc_prove's would be and the bit is written there."""
    nin, _, ntr = _shapes[h]
    _need(inputs, nin, "inputs")
    _need(transcript, ntr, "transcript")
    if accept is not None:
        if accept.element_size() != 4 or accept.numel() < 1:
            raise ValueError("accept must be an int32 tensor")
        _check(lib().vc_prove_verify(h, _ptr(inputs), seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript),
                                     ctypes.cast(ctypes.c_void_p(accept.data_ptr()), ctypes.POINTER(ctypes.c_int)),
                                     _stream(stream, device)), "vc_prove_verify")
        return None
    acc = ctypes.c_int(0)
    _check(lib().vc_prove_verify(h, _ptr(inputs), seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript), ctypes.byref(acc),
                                 _stream(stream, device)), "vc_prove_verify")
    return bool(acc.value)


def vc_verify(h, inputs, seed: int, transcript, stream=None, device: int = 0, accept=None) -> bool:
    """Returns the accept bit; with `accept` (a CUDA int32 tensor of >= 1
    element) the call is asynchronous and the bit is written there instead."""
    nin, _, ntr = _shapes[h]
    _need(inputs, nin, "inputs")
    _need(transcript, ntr, "transcript")
    if accept is not None:
        if accept.element_size() != 4 or accept.numel() < 1:
            raise ValueError("accept must be an int32 tensor")
        _check(lib().vc_verify(h, _ptr(inputs), seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript),
                               ctypes.cast(ctypes.c_void_p(accept.data_ptr()), ctypes.POINTER(ctypes.c_int)),
                               _stream(stream, device)), "vc_verify")
        return None
    acc = ctypes.c_int(0)
    _check(lib().vc_verify(h, _ptr(inputs), seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript), ctypes.byref(acc),
                           _stream(stream, device)), "vc_verify")
    return bool(acc.value)


def vc_circuit_set_stage_events(h, events):
    """events: 2 * NUM_STAGES entries, torch.cuda.Event (enable_timing=True)
    or None to skip that mark: start and end of every stage; or None."""
    if events is None:
        _check(lib().vc_circuit_set_stage_events(h, None), "vc_circuit_set_stage_events")
        return
    if len(events) != 2 * NUM_STAGES:
        raise ValueError(f"need {2 * NUM_STAGES} events")
    for e in events:  # make sure each event exists on the device
        if e is not None and getattr(e, "cuda_event", 0) == 0:
            e.record()
    arr = (ctypes.c_void_p * (2 * NUM_STAGES))(*[None if e is None else e.cuda_event for e in events])
    _check(lib().vc_circuit_set_stage_events(h, arr), "vc_circuit_set_stage_events")


def vc_circuit_get_info(h) -> dict:
    info = CircuitInfo()
    _check(lib().vc_circuit_get_info(h, ctypes.byref(info)), "vc_circuit_get_info")
    return {name: getattr(info, name) for name, _ in CircuitInfo._fields_ if name != "pad"}


def vc_prove_batch(handles, inputs, seeds, transcripts, stream=None, device: int = 0):
    n = len(handles)
    if not (len(inputs) == len(seeds) == len(transcripts) == n):
        raise ValueError("one input, seed and transcript per circuit")
    for h, x, t in zip(handles, inputs, transcripts):
        _need(x, _shapes[h][0], "inputs")
        _need(t, _shapes[h][2], "transcript")
    hs = (ctypes.c_void_p * n)(*handles)
    ins = (ctypes.c_void_p * n)(*[_ptr(x) for x in inputs])
    sd = (ctypes.c_uint64 * n)(*[s & 0xFFFFFFFFFFFFFFFF for s in seeds])
    trs = (ctypes.c_void_p * n)(*[_ptr(t) for t in transcripts])
    _check(lib().vc_prove_batch(hs, ins, sd, trs, n, _stream(stream, device)), "vc_prove_batch")
    return transcripts


_batches = {}  # batch handle -> member handles


def vc_batch_create(handles):
    """Returns an opaque batch handle (int) over distinct circuit handles."""
    n = len(handles)
    hs = (ctypes.c_void_p * max(n, 1))(*handles)
    b = ctypes.c_void_p()
    _check(lib().vc_batch_create(hs, n, ctypes.byref(b)), "vc_batch_create")
    _batches[b.value] = list(handles)
    return b.value


def vc_batch_destroy(b):
    _check(lib().vc_batch_destroy(b), "vc_batch_destroy")
    _batches.pop(b, None)


def vc_batch_prove(b, inputs, seeds, transcripts, stream=None, device: int = 0):
    handles = _batches[b]
    n = len(handles)
    if not (len(inputs) == len(seeds) == len(transcripts) == n):
        raise ValueError("one input, seed and transcript per member")
    for h, x, t in zip(handles, inputs, transcripts):
        _need(x, _shapes[h][0], "inputs")
        _need(t, _shapes[h][2], "transcript")
    ins = (ctypes.c_void_p * n)(*[_ptr(x) for x in inputs])
    sd = (ctypes.c_uint64 * n)(*[s & 0xFFFFFFFFFFFFFFFF for s in seeds])
    trs = (ctypes.c_void_p * n)(*[_ptr(t) for t in transcripts])
    _check(lib().vc_batch_prove(b, ins, sd, trs, _stream(stream, device)), "vc_batch_prove")
    return transcripts


def vc_batch_sync(b, stream=None, device: int = 0):
    _check(lib().vc_batch_sync(b, _stream(stream, device)), "vc_batch_sync")


def vc_batch_get_info(b) -> dict:
    info = BatchInfo()
    _check(lib().vc_batch_get_info(b, ctypes.byref(info)), "vc_batch_get_info")
    return {name: getattr(info, name) for name, _ in BatchInfo._fields_}


def _desc_struct(log_width, wiring):
    lw = [int(x) for x in log_width]
    kinds = [int(k) for k in wiring]
    d = len(kinds)
    if len(lw) != d + 1:
        raise ValueError("log_width must have len(wiring) + 1 entries")
    lw_a = (ctypes.c_uint32 * (d + 1))(*lw)
    k_a = (ctypes.c_uint32 * max(d, 1))(*kinds)
    return _Desc(d, ctypes.cast(lw_a, _u32p), ctypes.cast(k_a, _u32p), None, None, None), (lw_a, k_a)


def vc_server_create(device: int = 0, mem_cap_bytes: int = 0, max_batch: int = 0, max_inflight: int = 0,
                     pr_split_log: int = 0):
    """pr_split_log: the server's circuits split product-weighted instances
    below 2^pr_split_log entries into half-size chunks (0: each circuit's own
    tile shapes)."""
    cfg = ServerConfig(mem_cap_bytes, max_batch, max_inflight, pr_split_log, 0)
    h = ctypes.c_void_p()
    _check(lib().vc_server_create(device, ctypes.byref(cfg), ctypes.byref(h)), "vc_server_create")
    return h.value


def vc_server_destroy(s):
    _check(lib().vc_server_destroy(s), "vc_server_destroy")


def vc_server_submit(s, log_width, wiring, inputs, seed: int, transcript) -> int:
    """Queue a proof; `inputs` and `transcript` must stay alive until the job is done."""
    desc, keep = _desc_struct(log_width, wiring)
    _need(inputs, 1 << int(log_width[-1]), "inputs")
    jid = ctypes.c_uint64()
    _check(lib().vc_server_submit(s, ctypes.byref(desc), _ptr(inputs), seed & 0xFFFFFFFFFFFFFFFF, _ptr(transcript),
                                  ctypes.byref(jid)), "vc_server_submit")
    del keep
    return jid.value


def _job(info: JobInfo) -> dict:
    return {"done": bool(info.done), "status": info.status, "submit_ns": info.submit_ns,
            "start_ns": info.start_ns, "done_ns": info.done_ns}


def vc_server_poll(s, job_id: int) -> dict:
    info = JobInfo()
    _check(lib().vc_server_poll(s, job_id, ctypes.byref(info)), "vc_server_poll")
    return _job(info)


def vc_server_wait(s, job_id: int) -> dict:
    info = JobInfo()
    _check(lib().vc_server_wait(s, job_id, ctypes.byref(info)), "vc_server_wait")
    return _job(info)


def vc_server_get_stats(s) -> dict:
    st = ServerStats()
    _check(lib().vc_server_get_stats(s, ctypes.byref(st)), "vc_server_get_stats")
    return {name: getattr(st, name) for name, _ in ServerStats._fields_}


def vc_server_cancel(s, job_id: int) -> None:
    """Cancel a queued job (raises VcError VC_EBUSY once it is on the device or done)."""
    _check(lib().vc_server_cancel(s, job_id), "vc_server_cancel")


def vc_set_memory_limit(device_bytes: int = 0, pinned_bytes: int = 0) -> None:
    """Cap the device / page-locked host bytes the library holds (0: no cap)."""
    _check(lib().vc_set_memory_limit(int(device_bytes), int(pinned_bytes)), "vc_set_memory_limit")


def vc_get_memory_usage() -> tuple:
    """(device bytes, page-locked host bytes) the library holds now."""
    d, h = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().vc_get_memory_usage(ctypes.byref(d), ctypes.byref(h)), "vc_get_memory_usage")
    return d.value, h.value


def _tiles(t: TileConfig) -> dict:
    return {name: getattr(t, name) for name, _ in TileConfig._fields_}


def vc_autotune(log_width, wiring, device: int = 0, reps: int = 5):
    """Time candidate tile shapes for this circuit shape; the fastest is
    recorded for its size class and used by later vc_circuit_create calls.
    Returns (tiles dict, mean proof ms)."""
    desc, keep = _desc_struct(log_width, wiring)
    best = TileConfig()
    ms = ctypes.c_double(0)
    _check(lib().vc_autotune(ctypes.byref(desc), device, reps, ctypes.byref(best), ctypes.byref(ms)), "vc_autotune")
    del keep
    return _tiles(best), ms.value


def vc_autotune_batch(shapes, device: int = 0, reps: int = 3):
    """Tune one tile configuration for the merged batch of `shapes` (a list of
    (log_width, wiring)); it is recorded for every shape's size class.
    Returns (tiles dict, mean batch ms)."""
    descs = (_Desc * len(shapes))()
    keep = []
    for j, (lw, wr) in enumerate(shapes):
        d, k = _desc_struct(lw, wr)
        descs[j] = d
        keep.append(k)
    best = TileConfig()
    ms = ctypes.c_double(0)
    _check(lib().vc_autotune_batch(descs, len(shapes), device, reps, ctypes.byref(best), ctypes.byref(ms)),
           "vc_autotune_batch")
    del keep
    return _tiles(best), ms.value


def vc_circuit_create_tiles(log_width, wiring, tiles: dict, device: int = 0):
    desc, keep = _desc_struct(log_width, wiring)
    t = TileConfig(tiles["pr_chunk_log"], tiles["gn_chunk_log"], tiles["line_chunk_log"], tiles["eval_chunk_log"],
                   tiles.get("pr_split_log", VC_SPLIT_WIDEST))
    h = ctypes.c_void_p()
    _check(lib().vc_circuit_create_tiles(ctypes.byref(desc), device, ctypes.byref(t), ctypes.byref(h)),
           "vc_circuit_create_tiles")
    del keep
    n = ctypes.c_uint64()
    _check(lib().vc_transcript_len(h, ctypes.byref(n)), "vc_transcript_len")
    _shapes[h.value] = (1 << int(log_width[-1]), 1 << int(log_width[0]), n.value)
    return h.value


def vc_circuit_get_tiles(h) -> dict:
    t = TileConfig()
    _check(lib().vc_circuit_get_tiles(h, ctypes.byref(t)), "vc_circuit_get_tiles")
    return _tiles(t)


def vc_field_mul(a, b, out, stream=None, device: int = 0):
    _need(a, _numel(out), "a")
    _need(b, _numel(out), "b")
    _check(lib().vc_field_mul(_ptr(a), _ptr(b), _ptr(out), _numel(out), _stream(stream, device)), "vc_field_mul")
    return out


def vc_field_mul_rate(device: int = 0, variant: int = 0, iters: int = 1 << 14) -> float:
    r = ctypes.c_double(0)
    _check(lib().vc_field_mul_rate(device, variant, iters, ctypes.byref(r)), "vc_field_mul_rate")
    return r.value


NOALLOC_MAX_VALUES = 1 << 20


def vc_evaluate_noalloc(log_width, wiring, inputs, outputs, stream=None, device: int = 0):
    """Evaluate a structured-wiring circuit without any device allocation.

    For callers that cannot allocate device memory (their device memory is
    owned by another allocator, or allocation's implicit synchronisation is
    unacceptable).  inputs/outputs must be CUDA tensors on the current device;
    intermediate layers live in the library's fixed 2^20-element device array,
    shared by all calls (overlapping calls race)."""
    lw = [int(x) for x in log_width]
    kinds = [int(k) for k in wiring]
    d = len(kinds)
    if len(lw) != d + 1:
        raise ValueError("log_width must have len(wiring) + 1 entries")
    need = sum(1 << s for s in lw[1:d])
    if need > NOALLOC_MAX_VALUES:
        raise VcError(VC_EINVAL, f"vc_evaluate_noalloc: intermediate layers need {need} field elements, "
                                 f"the fixed array holds {NOALLOC_MAX_VALUES}")
    _need(inputs, 1 << lw[-1], "inputs")
    _need(outputs, 1 << lw[0], "outputs")
    lw_a = (ctypes.c_uint32 * (d + 1))(*lw)
    k_a = (ctypes.c_uint32 * max(d, 1))(*kinds)
    desc = _Desc(d, ctypes.cast(lw_a, _u32p), ctypes.cast(k_a, _u32p), None, None, None)
    _check(lib().vc_evaluate_noalloc(ctypes.byref(desc), _ptr(inputs), _ptr(outputs), _stream(stream, device)),
           "vc_evaluate_noalloc")
    return outputs


def vc_status_string(status: int) -> str:
    return lib().vc_status_string(status).decode()
