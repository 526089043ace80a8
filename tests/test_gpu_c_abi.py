"""The C ABI from plain C: build tests/c_abi/nf_c_example.c against libnf.so
with gcc, run it on the GPU, and compare its output with the oracle."""
import os
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "nf_c_example.c")


def _build(tmp_path):
    from paper_2110_11392_gb300 import _build as b
    lib = b.build_library()
    cuda = os.path.dirname(os.path.dirname(b.nvcc()))
    libdir = os.path.join(cuda, "lib64")
    if not os.path.isdir(libdir):
        libdir = os.path.join(cuda, "lib")
    exe = str(tmp_path / "nf_c_example")
    cmd = ["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           SRC, "-o", exe, "-L", os.path.dirname(lib), "-lnf", "-L", libdir, "-lcudart", "-lm",
           f"-Wl,-rpath,{os.path.dirname(lib)}", f"-Wl,-rpath,{libdir}"]
    subprocess.check_call(cmd)
    return exe


def test_c_example_compiles(tmp_path):
    """Compiling and linking needs no GPU."""
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_example_runs_and_matches_oracle(tmp_path):
    exe = _build(tmp_path)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    line = out.stdout.strip().split()
    assert line[0] == "ok"
    kv = dict(t.split("=") for t in line[1:8])
    acc0 = np.array([float(kv["acc0"]), float(line[8]), float(line[9])])
    # regenerate the C program's positions (its LCG) and check particle 0
    N = 20000
    state = 88172645463325252
    vals = np.empty(3 * N, np.float32)
    for i in range(3 * N):
        state = (state * 6364136223846793005 + 1442695040888963407) % (1 << 64)
        u = np.float32((state >> 40) * (1.0 / 16777216.0))
        vals[i] = u if u < 1.0 else 0.0
    pos = vals.reshape(N, 3)
    eps = 1.0 / (40.0 * np.cbrt(N))
    ref = oracle.forces(pos, 1.0, 7, 2, eps, sinks=np.array([0]))[0]
    assert np.linalg.norm(acc0 - ref) / np.linalg.norm(ref) < 1e-5
    assert line[10].startswith("far0=")
    far0 = np.array([float(line[10][5:]), float(line[11]), float(line[12])])
    fref = oracle.far_field(pos, 1.0, 7, 2, 4)
    assert np.abs(far0 - fref[0]).max() < 1e-10 * np.abs(fref).max()
    assert int(kv["N"]) == N and int(kv["pairs"]) > 0 and int(kv["items"]) > 0
    assert float(kv["net"]) < 1e-3 * float(kv["mean_abs_acc"])
