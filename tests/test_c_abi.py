"""The C ABI used from a plain C99 program (tests/abi_example.c).

CPU: the program is compiled with gcc -std=c99 -Wall -Wextra -Werror against
include/mdp.h and include/mdp_ingest.h, linked to the library, and runs its
host-only part (ingest, PETSc files, host entry points).  GPU: the same
program, built with the CUDA runtime for its own buffers, also creates,
solves and checks a handle.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "abi_example.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _cuda_libdir():
    for sub in ("lib64", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        d = os.path.join(CUDA, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    pytest.skip("no libcudart.so under " + CUDA)


def _compile(tmp_path, cuda):
    from paper_2502_14474_gb300 import capi
    lib = capi.load() and capi.library_path()
    exe = os.path.join(tmp_path, "abi_example")
    cmd = ["gcc", "-std=c99", "-O1", "-Wall", "-Wextra", "-Werror", "-I",
           os.path.join(ROOT, "include"), SRC, "-o", exe, lib,
           "-Wl,-rpath," + os.path.dirname(lib), "-lm"]
    if cuda:
        cmd[1:1] = ["-DMDP_EXAMPLE_CUDA", "-I", os.path.join(CUDA, "include")]
        libdir = _cuda_libdir()
        cmd += ["-L", libdir, "-lcudart", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_program_host_part(tmp_path):
    exe = _compile(str(tmp_path), cuda=False)
    r = subprocess.run([exe, "host", str(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


@pytest.mark.gpu
def test_c_program_solves_on_the_gpu(tmp_path):
    exe = _compile(str(tmp_path), cuda=True)
    r = subprocess.run([exe, "gpu", str(tmp_path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
