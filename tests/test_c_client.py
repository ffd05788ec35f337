"""The C ABI from a plain C99 program (tests/c_client/etc_client.c).

include/etc.h must compile as strict C99 (gcc -std=c99 -pedantic -Werror) and
a C program must link against libetc.so and use it without Python: host-side
validation on the CPU, and on the GPU the closed-form homogeneous solve
(tensor diag(kx, ky, kz) in one PCG iteration, linear temperature field).
"""
import os
import shutil
import subprocess

import pytest

from paper_2404_02433_b300 import build as BUILD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "etc_client.c")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = BUILD.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("c_client") / "etc_client")
    cmd = ["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-O1",
           "-I", os.path.join(ROOT, "include"), SRC, "-o", exe,
           "-L", libdir, "-letc", f"-Wl,-rpath,{libdir}", "-lm"]
    out = subprocess.run(cmd, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    return exe


def test_c_client_host_checks(client):
    out = subprocess.run([client], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "etc_client: ok" in out.stdout


@pytest.mark.gpu
def test_c_client_solves_homogeneous_medium(client):
    out = subprocess.run([client, "--gpu"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "etc_client: ok" in out.stdout
