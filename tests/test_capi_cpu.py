"""Host-side checks of the C ABI library (no GPU needed).

The library is built for sm_103a with nvcc (cross-compiles here) and loaded
with ctypes; every function include/*.h declares must be exported.  Only
calls that do no device work are made.
"""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdp.h")


def _declared():
    names = set()
    for header in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = re.sub(r"/\*.*?\*/", "", open(header).read(), flags=re.S)
        names.update(re.findall(r"\b(mdp_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2502_14474_gb300 import capi
    return capi.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mdp_create", "mdp_bellman", "mdp_policy_eval", "mdp_solve", "mdp_destroy",
              "mdp_last_error", "mdp_bytes_required"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2502_14474_gb300 import capi
    declared = _declared()
    assert sorted(capi.EXPORTED) == declared
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", capi.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (mdp_\w+)", out))
    assert set(declared) <= exported


def test_library_is_built_for_sm_103a(lib):
    from paper_2502_14474_gb300 import capi
    out = subprocess.run(["cuobjdump", "--list-elf", capi.library_path()], capture_output=True,
                         text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_host_only_entry_points(lib):
    from paper_2502_14474_gb300 import capi
    assert capi.mdp_version().startswith("mdp-gb300")
    o = capi.mdp_default_opts()
    assert o.tol == 1e-9 and o.inner_rtol == 0.1 and o.restart == 30
    # size model: CSR + basis dominate; grows with nnz and restart
    a = capi.mdp_bytes_required(1 << 22, 8, 1 << 29, capi.MDP_F32, capi.MDP_F32, 30)
    b = capi.mdp_bytes_required(1 << 22, 8, 1 << 29, capi.MDP_F32, capi.MDP_BF16, 30)
    c = capi.mdp_bytes_required(1 << 22, 8, 1 << 29, capi.MDP_F32, capi.MDP_F32, 60)
    assert 4.3e9 < a < 6e9 and b > a and c > a
    assert capi.mdp_bytes_required(0, 1, 1) == 0
    assert capi.mdp_last_error() == ""


def test_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2502_14474_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt
                assert "oracle.c" not in txt


def test_bytes_required_terms(lib):
    """The admission estimate covers the 16-bit copy at 4 bytes per entry (column
    offset + value, with up to a quarter of padding for short rows) and the
    action-major copy of short rows (one more 8-byte entry per nonzero, padded)."""
    from paper_2502_14474_gb300 import capi
    n, m, nnz = 1 << 20, 8, 1 << 27          # 16 entries per row: no short-row copy
    f32 = capi.mdp_bytes_required(n, m, nnz, capi.MDP_F32, capi.MDP_F32, 30)
    b16 = capi.mdp_bytes_required(n, m, nnz, capi.MDP_F32, capi.MDP_BF16, 30)
    assert b16 - f32 >= nnz * 4 * 1.25 + n * m * 4
    short = 5 * n * m                          # 5 entries per row: short rows
    s32 = capi.mdp_bytes_required(n, m, short, capi.MDP_F32, capi.MDP_F32, 30)
    plain = (n * m + 1) * 4 + short * 8 + n * m * 8
    assert s32 - plain >= short * 8 * 1.25    # the padded action-major copy
    f64 = capi.mdp_bytes_required(n, m, nnz, capi.MDP_F64, capi.MDP_F32, 30)
    assert f64 - f32 >= nnz * 4                # FP64 remainders of the probabilities
