"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
function declared in include/vc.h, and rejects malformed circuits before it
touches a device."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1202_1350_gb300 import build, circuits, vc


@pytest.fixture(scope="module")
def libvc():
    build.build()
    return vc.lib()


def test_exports_every_declared_function(libvc):
    names = vc.header_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(libvc, name), name
        assert isinstance(getattr(libvc, name), ctypes._CFuncPtr)


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets: a C program compiled with gcc against include/vc.h prints them."""
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    mirrors = {"vc_circuit_desc": vc._Desc, "vc_circuit_info": vc.CircuitInfo, "vc_batch_info": vc.BatchInfo,
               "vc_server_config": vc.ServerConfig, "vc_job_info": vc.JobInfo, "vc_server_stats": vc.ServerStats,
               "vc_tile_config": vc.TileConfig}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "vc.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([gcc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, what, val = line.split()
            got[(cname, what)] = int(val)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_status_strings(libvc):
    assert vc.vc_status_string(0) == "ok"
    assert vc.vc_status_string(1) == "invalid argument"
    assert vc.vc_status_string(vc.VC_ECANCELED) == "cancelled"


def test_memory_budget_host_side(libvc):
    """The library-wide memory budget is host state: it can be set and read
    without a device, and a refused allocation (exercised on the GPU) leaves
    the accounting unchanged."""
    assert vc.vc_get_memory_usage() == (0, 0)
    vc.vc_set_memory_limit(1 << 20, 1 << 10)
    vc.vc_set_memory_limit(0, 0)
    assert libvc.vc_get_memory_usage(None, None) == vc.VC_EINVAL


@pytest.mark.parametrize("widths,kinds", [
    ([2, 2], [vc.TREE]), ([1, 3], [vc.SQUARE]), ([3, 4], [vc.MATMULT]), ([4, 3], [vc.MATMULT]), ([1, 3], [vc.F0_FIRST]),
    ([0, 0], [vc.F0_PAIR]), ([2, 2], [vc.F0_FINAL]), ([31, 31], [vc.SQUARE]), ([1, 1], [9])])
def test_bad_shapes_rejected_without_device(libvc, widths, kinds):
    with pytest.raises(vc.VcError) as e:
        vc.vc_circuit_create(widths, kinds)
    assert e.value.status == vc.VC_EINVAL


def test_bad_explicit_wiring_rejected(libvc):
    ex = [(np.array([0, 1]), np.array([0, 2]), np.array([1, 1]))]
    with pytest.raises(vc.VcError) as e:
        vc.vc_circuit_create([1, 1], [vc.EXPLICIT], explicit=ex)
    assert e.value.status == vc.VC_EINVAL
    ex = [(np.array([0, 2]), np.array([0, 1]), np.array([1, 1]))]
    with pytest.raises(vc.VcError):
        vc.vc_circuit_create([1, 1], [vc.EXPLICIT], explicit=ex)


@pytest.mark.parametrize("family,logn", [("f2", 10), ("f2", 20), ("f0", 16), ("matmult", 7), ("matmult", 1)])
def test_circuit_descriptions_agree_with_oracle(family, logn):
    """The product's layer descriptions and the oracle's are written separately;
    both must describe the same circuit."""
    assert circuits.by_name(family, logn) == getattr(oracle, f"{family}_layers")(logn)


def test_gate_counts():
    # F2 at n = 2^20: 2^20 squaring gates and 2^20 - 1 addition gates
    assert circuits.non_input_gates(circuits.f2(20)[0]) == 2 * (1 << 20) - 1
    assert circuits.non_input_gates(circuits.matmult(7)[0]) == (1 << 21) + (1 << 21) - (1 << 14)


def test_batch_arguments_rejected_without_device(libvc):
    with pytest.raises(vc.VcError) as e:
        vc.vc_batch_create([])
    assert e.value.status == vc.VC_EINVAL
    with pytest.raises(vc.VcError) as e:
        vc.vc_batch_create([None])
    assert e.value.status == vc.VC_EINVAL
    assert libvc.vc_batch_get_info(None, None) == vc.VC_EINVAL
    assert libvc.vc_batch_sync(None, None) == vc.VC_EINVAL
    assert libvc.vc_batch_prove(None, None, None, None, None) == vc.VC_EINVAL
    assert libvc.vc_batch_destroy(None) == vc.VC_OK
    assert libvc.vc_prove_batch(None, None, None, None, 0, None) == vc.VC_OK
    assert libvc.vc_prove_batch(None, None, None, None, -1, None) == vc.VC_EINVAL


@pytest.mark.parametrize("family,logn", [("f2", 0), ("f2", 10), ("f0", 3), ("matmult", 3)])
def test_transcript_len_matches_library(libvc, family, logn):
    w, k = circuits.by_name(family, logn)
    c = oracle.Circuit(w, k)
    assert circuits.transcript_len(w) == len(c.prove(np.zeros(1 << w[-1], np.uint64), 1))


def test_tile_arguments_rejected_without_device(libvc):
    w, k = circuits.f2(6)
    for bad in ({"pr_chunk_log": 14, "gn_chunk_log": 12, "line_chunk_log": 13, "eval_chunk_log": 10},
                {"pr_chunk_log": 13, "gn_chunk_log": 13, "line_chunk_log": 13, "eval_chunk_log": 10},
                {"pr_chunk_log": 13, "gn_chunk_log": 12, "line_chunk_log": 14, "eval_chunk_log": 10},
                {"pr_chunk_log": 13, "gn_chunk_log": 12, "line_chunk_log": 13, "eval_chunk_log": 12},
                {"pr_chunk_log": 0, "gn_chunk_log": 12, "line_chunk_log": 13, "eval_chunk_log": 10},
                {"pr_chunk_log": 13, "gn_chunk_log": 12, "line_chunk_log": 13, "eval_chunk_log": 10,
                 "pr_split_log": 41}):
        with pytest.raises(vc.VcError) as e:
            vc.vc_circuit_create_tiles(w, k, bad)
        assert e.value.status == vc.VC_EINVAL
    with pytest.raises(vc.VcError) as e:
        vc.vc_autotune([1, 1], [vc.EXPLICIT])
    assert e.value.status == vc.VC_EINVAL
