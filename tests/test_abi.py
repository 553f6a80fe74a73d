"""The C-ABI library loads on a machine without a GPU and exports every declared symbol."""
import os
import re

import pytest

from paper_1606_03135_gb300 import rbffd as R

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "rbffd.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbffd_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    L = R.load()
    names = declared_functions()
    assert "rbffd_plan" in names and "rbffd_assemble" in names and "rbffd_apply" in names
    for name in names:
        assert hasattr(L, name), name
    assert set(names) <= set(R._SIGS), set(names) - set(R._SIGS)


def test_strerror_and_argument_checks_need_no_gpu():
    assert R.rbffd_strerror(R.ETIMEOUT).startswith("a bounded")
    assert R.rbffd_strerror(12345) == "unknown error"
    import ctypes as C
    dummy = C.c_void_p(16)
    # every one of these is rejected before any CUDA call is made
    assert R.rbffd_plan(None, 10, 2, 5, 1, 3, 0.5)[0] == R.EINVAL
    assert R.rbffd_plan(dummy, 10, 4, 5, 1, 3, 0.5)[0] == R.EINVAL      # d
    assert R.rbffd_plan(dummy, 10, 2, 5, 1, 4, 0.5)[0] == R.EINVAL      # m even
    assert R.rbffd_plan(dummy, 10, 2, 5, 1, 3, 0.0)[0] == R.EINVAL      # delta = 0
    assert R.rbffd_plan(dummy, 10, 2, 5, 1, 3, 1.5)[0] == R.EINVAL      # delta > 1
    assert R.rbffd_plan(dummy, 4, 2, 5, 1, 3, 0.5)[0] == R.EINVAL       # N < n
    assert R.rbffd_plan(dummy, 100, 2, 5, 2, 3, 0.5)[0] == R.EINVAL     # n < M
    assert R.rbffd_plan(dummy, 1000, 2, 129, 2, 3, 0.5)[0] == R.EINVAL  # n too large
    assert R.rbffd_assemble(None)[0] == R.EINVAL
    assert R.rbffd_plan_delta(None, 0.5)[0] == R.EINVAL                 # no base plan
    assert R.rbffd_apply(None, None, None) == R.EINVAL
    # team sizes: 32, 64, 96, 128, 256, 512 or 0; 32, 64, 96 and 256 only for LDL^T
    bad_team = R.rbffd_opts(R.STAB_SEQ, 0, 5000, 1, 0, R.FACTOR_LDLT, 0, 48)
    assert R.rbffd_plan(dummy, 1000, 2, 12, 2, 3, 0.5, bad_team)[0] == R.EINVAL
    lu_warp = R.rbffd_opts(R.STAB_SEQ, 0, 5000, 1, 0, R.FACTOR_LU, 0, 32)
    assert R.rbffd_plan(dummy, 1000, 2, 12, 2, 3, 0.5, lu_warp)[0] == R.EINVAL
    lu_256 = R.rbffd_opts(R.STAB_SEQ, 0, 5000, 1, 0, R.FACTOR_LU, 0, 256)
    assert R.rbffd_plan(dummy, 1000, 2, 12, 2, 3, 0.5, lu_256)[0] == R.EINVAL
    assert R.load().rbffd_set_boundary(None, None, None) == R.EINVAL
    assert R.load().rbffd_timestep_matrix(None, 0.5, None, None) == R.EINVAL
    assert R.rbffd_export_async(None, None, None, None, None, None) == R.EINVAL
    neg_cap = R.rbffd_opts(R.STAB_SEQ, 0, 5000, 1, 0, R.FACTOR_LDLT, -1, 0)
    assert R.rbffd_plan(dummy, 1000, 2, 12, 2, 3, 0.5, neg_cap)[0] == R.EINVAL
    neg_chunk = R.rbffd_opts(R.STAB_SEQ, 0, 5000, 1, 0, R.FACTOR_LDLT, 0, 0, -1)
    assert R.rbffd_plan(dummy, 1000, 2, 12, 2, 3, 0.5, neg_chunk)[0] == R.EINVAL
    lu_chunk = R.rbffd_opts(R.STAB_SEQ, 0, 5000, 1, 0, R.FACTOR_LU, 0, 0, 4)
    assert R.rbffd_plan(dummy, 1000, 2, 12, 2, 3, 0.5, lu_chunk)[0] == R.EINVAL
    bad_ref = R.rbffd_opts(R.STAB_SEQ, 0, 5000, 1, 0, R.FACTOR_LDLT, 0, 0, 0, 2)
    assert R.rbffd_plan(dummy, 1000, 2, 12, 2, 3, 0.5, bad_ref)[0] == R.EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors of the C structs have the sizes and offsets gcc gives the header."""
    import ctypes as C
    import subprocess
    structs = {"rbffd_opts": R.rbffd_opts, "rbffd_csr": R.rbffd_csr,
               "rbffd_stats_t": R.rbffd_stats_t}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rbffd.h"', "int main(){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_fp64_probe_library_loads_exports_and_checks_arguments_without_a_gpu():
    from paper_1606_03135_gb300 import probe as P
    L = P.load()
    src = open(os.path.join(os.path.dirname(HEADER), "fp64_probe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for name in set(re.findall(r"\b(fp64_probe_[a-z_]+)\s*\(", src)):
        assert hasattr(L, name), name
    assert P.fp64_probe_run(7, 10)[0] == -1   # unknown kind: refused before any CUDA call
    assert P.fp64_probe_run(0, 0)[0] == -1    # no iterations
