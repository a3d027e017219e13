"""The C ABI library builds, loads on a machine without a GPU, and exports every
entry point include/l1fct.h declares (no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "l1fct.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1207_4684_gb300 import build

    build.build()
    import paper_1207_4684_gb300 as L

    return L.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^L1S_API\s+[\w\s\*]+?\b(\w+)\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fct_embed", "l1_condition", "l1_sample", "l1_regress"):
        assert required in names
    assert len(names) >= 17


def test_every_declared_symbol_is_exported(lib):
    from paper_1207_4684_gb300 import l1fct

    out = subprocess.run(["nm", "-D", "--defined-only", l1fct.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    declared = set(declared_functions())
    assert declared <= exported, f"missing: {sorted(declared - exported)}"
    assert declared == set(l1fct.EXPORTS), "binding signatures out of sync with the header"
    for name in declared:
        assert hasattr(lib, name)


@pytest.mark.parametrize("cname,pyname", [("l1s_params", "Params"), ("l1s_schedule", "Schedule"),
                                          ("l1s_problem", "Problem")])
def test_struct_layout(tmp_path, cname, pyname):
    """Each ctypes structure mirrors its C struct byte for byte (checked with the C compiler)."""
    import ctypes

    from paper_1207_4684_gb300 import l1fct

    cls = getattr(l1fct, pyname)
    fields = [f for f, _ in cls._fields_]
    fmt = " ".join(["%zu"] * (len(fields) + 1))
    offs = ", ".join(f"offsetof({cname},{f})" for f in fields)
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "l1fct.h"\nint main(void){'
                   f'printf("{fmt}\\n", sizeof({cname}), {offs}); return 0;}}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(cls)] + [getattr(cls, f).offset for f in fields]
    assert got == want


def test_schedule_table_argument_checks(lib):
    import paper_1207_4684_gb300 as L

    with pytest.raises(L.L1SError) as e:
        L.l1s_schedule_set(16, L.F32, 48, {"fct_variant": 1})
    assert e.value.code == 1
    with pytest.raises(L.L1SError) as e:
        L.l1s_schedule_set(16, L.F32, 256, {"fct_variant": 8})
    assert e.value.code == 1 and "out of range" in str(e.value)


def test_version_and_argument_errors_without_gpu(lib):
    import paper_1207_4684_gb300 as L

    assert "sm_103a" in L.version()
    with pytest.raises(L.L1SError) as e:
        L.l1s_workspace_size(L.make_params(s=48, r1=40, r2=16, coreset=100.0), 1000, 4)
    assert e.value.code == 1 and "power of two" in str(e.value)
    with pytest.raises(L.L1SError) as e:
        L.l1s_workspace_size(L.make_params(s=64, r1=3, r2=16, coreset=100.0), 1000, 4)
    assert e.value.code == 1 and "r1" in str(e.value)
    with pytest.raises(L.L1SError) as e:
        L.l1s_workspace_size(L.make_params(s=64, r1=40, r2=16, coreset=100.0, global_row_offset=10), 1000, 4)
    assert e.value.code == 1 and "global_row_offset" in str(e.value)
    # empty input and the width limits are argument errors, decided before any device work
    prm = L.make_params(s=64, r1=300, r2=16, coreset=100.0)
    with pytest.raises(L.L1SError) as e:
        L.l1s_workspace_size(prm, 0, 4)
    assert e.value.code == 1 and "n must be" in str(e.value)
    for d in (0, 129):
        with pytest.raises(L.L1SError) as e:
            L.l1s_workspace_size(prm, 1000, d)
        assert e.value.code == 1 and "d must be" in str(e.value)
    with pytest.raises(L.L1SError) as e:
        L.l1s_workspace_size(L.make_params(s=64, r1=300, r2=0, coreset=100.0), 1000, 4)
    assert e.value.code == 1 and "r2" in str(e.value)


def test_product_code_never_touches_the_oracle():
    """Neither the package nor the CUDA sources import, read or call the oracle."""
    pkg = os.path.join(ROOT, "paper_1207_4684_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower().replace("oracle-", ""), f"{f} mentions the oracle"
    for dirpath, _, files in os.walk(os.path.join(ROOT, "oracle")):
        for f in files:
            if f.endswith(".py"):
                assert "paper_1207_4684_gb300" not in open(os.path.join(dirpath, f)).read()
