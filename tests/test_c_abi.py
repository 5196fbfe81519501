"""The C ABI used from C: tests/c/prove_f2.c includes include/vc.h, links
libvc.so and proves and verifies F2 with host buffers, separately and in one
call.  On CPU the program compiles and links; on the GPU its transcript
equals the oracle's, the honest proof is accepted (both ways) and a changed
one rejected."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1202_1350_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compile(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path / "prove_f2"
    subprocess.run([gcc, "-std=c11", "-O2", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "prove_f2.c"), "-L", libdir, "-lvc",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    return exe


def test_c_program_compiles_and_links(tmp_path):
    assert os.access(_compile(tmp_path), os.X_OK)


@pytest.mark.gpu
@pytest.mark.parametrize("n,seed", [(4, 3), (12, 77)])
def test_c_program_proof_equals_oracle(tmp_path, n, seed):
    exe = _compile(tmp_path)
    out = subprocess.run([str(exe), str(n), str(seed)], check=True, capture_output=True, text=True).stdout.split()
    assert out[:2] == ["prove", "ok"]
    assert out[2:5] == ["verify", "ok", "1"]
    assert out[5:7] == ["tampered", "0"]
    assert out[7:11] == ["prove_verify", "ok", "1", "1"]  # accepted, same transcript
    got = np.array([int(v) for v in out[11:]], dtype=np.uint64)
    x = np.array([(i * 2654435761) % 65537 for i in range(1 << n)], dtype=np.uint64)
    want = oracle.Circuit(*oracle.f2_layers(n)).prove(x, seed)
    assert len(got) == len(want)
    assert (got == want).all()
