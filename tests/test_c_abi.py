"""The C ABI used from plain C (tests/c/abi_example.c): the program builds
against include/ldupcg.h and links libldupcg.so and the CUDA runtime here;
on a GPU it runs FP64 Jacobi-PCG, the mixed pipelined solve and AMG-PCG on
an 8^3 box and checks every true residual on the host."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_example.c")


def build_example(tmp_path):
    from paper_1505_07630_gb300 import build
    lib = build.build()
    cuda = os.path.dirname(os.path.dirname(shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"))
    exe = str(tmp_path / "abi_example")
    libdir = os.path.dirname(lib)
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.isdir(d)), os.path.join(cuda, "lib64"))
    cmd = ["gcc", "-std=c11", "-O2", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(cuda, "include"), SRC, "-o", exe, "-L" + libdir, "-lldupcg",
           "-L" + cudalib, "-lcudart", "-lm", "-Wl,-rpath," + libdir, "-Wl,-rpath," + cudalib]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


def test_c_example_builds_and_links(tmp_path):
    assert os.path.exists(build_example(tmp_path))


@pytest.mark.gpu
def test_c_example_solves(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = build_example(tmp_path)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "c abi ok" in res.stdout
