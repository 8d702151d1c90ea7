"""The C ABI from plain C: paper_2508_16121_gb300/examples/c_client.c is
compiled and linked against libsvdlut.so and the CUDA runtime (CPU test), and
run on the GPU (gpu test), where every output pixel must equal its channel's
bias."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build_client(tmp_path):
    from paper_2508_16121_gb300 import build
    lib = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime_api.h")):
        pytest.skip("no C compiler or CUDA headers")
    exe = str(tmp_path / "c_client")
    libdir = os.path.dirname(lib)
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-o", exe,
           os.path.join(ROOT, "paper_2508_16121_gb300", "examples", "c_client.c"),
           "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(CUDA, "include"),
           lib, "-L" + os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + libdir,
           "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert os.path.exists(_build_client(tmp_path))


@pytest.mark.gpu
def test_c_client_runs(tmp_path):
    exe = _build_client(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c_client: ok" in r.stdout
