"""The C ABI used from C: tests/c/abi_smoke.c includes include/nmf.h alone,
compiles as C99 (checked here without a GPU), links against libnmf.so and
runs a small problem on the GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "abi_smoke.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    return cc


def test_header_and_program_compile_as_c99():
    r = subprocess.run([_cc(), "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                        SRC], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
def test_c_program_runs(tmp_path):
    from paper_1003_3272_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "abi_smoke")
    libdir = os.path.dirname(lib)
    r = subprocess.run([_cc(), "-std=c99", "-O1", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(CUDA, "include"), SRC, "-o", exe,
                        "-L", libdir, "-lnmf", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                        "-lm", "-Wl,-rpath," + libdir + ":" + os.path.join(CUDA, "lib64")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ok" in r.stdout
