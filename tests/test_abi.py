"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/rq.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rq.h")).read()
    return sorted(set(re.findall(r"^(?:rq_status|const char \*)\s*(rq_\w+)\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq.load()


def test_header_declares_the_binding_exports():
    from paper_2506_23775_gb300 import rq
    assert _declared() == sorted(rq.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_sm103a_only(lib):
    # one gencode target, compiled here for sm_103a
    from paper_2506_23775_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_null_arguments_are_rejected_without_a_device(lib):
    from paper_2506_23775_gb300 import rq
    assert lib.rq_create(None, 0, None) == rq.RQ_EINVAL
    assert lib.rq_destroy(None) == rq.RQ_OK
    assert lib.rq_cost(None, None, None) == rq.RQ_EINVAL
    assert lib.rq_get_info(None, None) == rq.RQ_EINVAL
    assert isinstance(lib.rq_last_error(None), bytes)


def test_struct_layouts_match_header(tmp_path):
    """Size and field offsets of every ctypes struct against the C compiler's
    layout of the header's struct."""
    import shutil
    import subprocess
    from paper_2506_23775_gb300 import rq
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rq_target": rq.RQTarget, "rq_circuit": rq.RQCircuit, "rq_tr_state": rq.RQTRState,
               "rq_info_t": rq.RQInfo, "rq_kernel_stat": rq.RQKernelStat}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rq.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[f"{cname} size"]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname} {fname}"]) == getattr(py, fname).offset, (cname, fname)
    # rq_tr_state: 5 doubles, int, 5 doubles, 3 ints (padded)
    assert ctypes.sizeof(rq.RQTarget) == 4 * 3 + 4 + 8 * 3 + 8
    assert ctypes.sizeof(rq.RQCircuit) == 16 + 16
    assert ctypes.sizeof(rq.RQInfo) == 4 * 4 + 8 * 2 + 4 * 3 + 4 + 8 * 3 + 4 + 4  # ctas_per_sweep, padding
