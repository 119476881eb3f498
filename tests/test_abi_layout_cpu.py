"""The ctypes mirrors of the C ABI's structs and enums match the headers.

A C program compiled with gcc against include/mdp.h and include/mdp_ingest.h
prints sizeof and offsetof of every field of every struct the binding
mirrors, and the values of the enums it copies; the test compares them with
the ctypes layouts and constants.  A field added on one side only (a silent
memory corruption across the boundary) fails here, on the CPU.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

ENUMS = ["MDP_F32", "MDP_F64", "MDP_BF16", "MDP_F16", "MDP_OK", "MDP_FLAG_HOST_INPUT",
         "MDP_FLAG_NO_VALIDATE", "MDP_FLAG_AUTOTUNE", "MDP_FLAG_MAXIMIZE", "MDP_INNER_GMRES",
         "MDP_INNER_RICHARDSON", "MDP_INNER_BICGSTAB", "MDP_HISTORY", "MDP_UNSEEN_ERROR",
         "MDP_UNSEEN_SELF_LOOP", "MDP_MAX_RESTART"]
STATUSES = ["MDP_OK", "MDP_ERR_ARG", "MDP_ERR_NOT_STOCHASTIC", "MDP_ERR_OOM", "MDP_ERR_CUDA",
            "MDP_ERR_NOT_CONVERGED", "MDP_ERR_TIMEOUT", "MDP_ERR_CANCELLED", "MDP_ERR_BAD_CSR",
            "MDP_ERR_NONFINITE"]


def _structs():
    from paper_2502_14474_gb300 import capi
    return {"mdp_solve_opts": capi.mdp_solve_opts, "mdp_solve_stats": capi.mdp_solve_stats,
            "mdp_eval_stats": capi.mdp_eval_stats, "mdp_info_t": capi.mdp_info_t,
            "mdp_profile_t": capi.mdp_profile_t, "mdp_host_csr": capi.mdp_host_csr,
            "mdp_gmres_cycle_t": capi.mdp_gmres_cycle_t}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mdp.h"',
             '#include "mdp_ingest.h"', 'int main(void) {']
    for name, cls in _structs().items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu %zu\\n", offsetof({name}, {field}), '
                         f'sizeof((({name}*)0)->{field}));')
    for e in ENUMS + STATUSES:
        lines.append(f'  printf("enum {e} %lld\\n", (long long)({e}));')
    lines += ['  printf("enum MDP_PROF_KINDS %d\\n", (int)MDP_PROF_KINDS);',
              '  printf("enum MDP_PROF_BICGSTAB_SPMV %d\\n", (int)MDP_PROF_BICGSTAB_SPMV);',
              '  printf("enum MDP_PROF_ARNOLDI_DOTS %d\\n", (int)MDP_PROF_ARNOLDI_DOTS);',
              '  return 0;', '}']
    d = tmp_path_factory.mktemp("abi")
    src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    src, "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout, enums = {}, {}
    for line in out.splitlines():
        parts = line.split()
        if parts[0] == "enum":
            enums[parts[1]] = int(parts[2])
        elif parts[1] == "sizeof":
            layout[(parts[0], None)] = (0, int(parts[2]))
        else:
            layout[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return layout, enums


@pytest.mark.parametrize("name", ["mdp_solve_opts", "mdp_solve_stats", "mdp_eval_stats",
                                  "mdp_info_t", "mdp_profile_t", "mdp_host_csr",
                                  "mdp_gmres_cycle_t"])
def test_struct_layout_matches_the_header(c_layout, name):
    import ctypes
    layout, _ = c_layout
    cls = _structs()[name]
    assert ctypes.sizeof(cls) == layout[(name, None)][1], name
    for field, _ in cls._fields_:
        desc = getattr(cls, field)
        assert (desc.offset, desc.size) == layout[(name, field)], (name, field)


def test_constants_match_the_header(c_layout):
    from paper_2502_14474_gb300 import capi
    _, enums = c_layout
    for e in ENUMS:
        assert getattr(capi, e) == enums[e], e
    assert len(capi.PROF_KINDS) == enums["MDP_PROF_KINDS"]
    assert capi.PROF_KINDS[enums["MDP_PROF_BICGSTAB_SPMV"]] == "bicgstab_spmv"
    assert capi.PROF_KINDS[enums["MDP_PROF_ARNOLDI_DOTS"]] == "arnoldi_dots"


def test_status_names_match_the_header(c_layout):
    from paper_2502_14474_gb300 import capi
    _, enums = c_layout
    assert {enums[name]: name for name in STATUSES} == capi.STATUS_NAMES
