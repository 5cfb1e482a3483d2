"""The C ABI library loads without a GPU and exports every declared symbol;
host-side argument checks answer without touching the device."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_27086_gb300 import build
    build.build()
    import paper_2606_27086_gb300 as pk
    return pk.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "suppy.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(suppy_[a-z_]+)\s*\(", src)))


def test_every_declared_function_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for nm in names:
        assert hasattr(lib, nm), nm


def test_binding_covers_the_header():
    import paper_2606_27086_gb300 as pk
    assert sorted(pk.EXPORTED) == _declared()


def test_version_string(lib):
    assert b"sm_103a" in lib.suppy_version()


def test_params_default_are_the_papers(lib):
    """suppy_params_default fills the stopping defaults printed in the paper."""
    import paper_2606_27086_gb300 as pk
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_defaults.json")))["stopping"]
    p = pk.suppy_params_default()
    assert p.prox_abs == gold["prox_abs"] and p.prox_rel == gold["prox_rel"]
    assert p.patience == gold["patience"] and p.max_sweeps == gold["max_sweeps"]
    assert p.obj_rel == gold["obj_rel"]
    assert p.lambda_ == 1.0


def test_create_rejects_null_arguments_without_a_device(lib):
    import paper_2606_27086_gb300 as pk
    out = ctypes.c_void_p()
    st = lib.suppy_create(None, None, None, None, None, None, None, ctypes.byref(out))
    assert st == pk.SUPPY_EINVAL
    assert out.value is None
    assert b"NULL" in lib.suppy_last_error(None)


def test_null_context_calls_fail_cleanly(lib):
    import paper_2606_27086_gb300 as pk
    assert lib.suppy_proximity(None, None) == pk.SUPPY_EINVAL
    assert lib.suppy_set_dvc(None, None, None, 0, None, 0, 1.0) == pk.SUPPY_EINVAL
    assert lib.suppy_dvc_dose(None, None, 0) == pk.SUPPY_EINVAL
    assert lib.suppy_dvc_proximity(None, None) == pk.SUPPY_EINVAL
    assert lib.suppy_launch_count(None) == 0
    lib.suppy_destroy(None)


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets the C
    compiler gives the header's structs (compiled here with gcc)."""
    import subprocess
    import paper_2606_27086_gb300 as pk
    structs = {"suppy_csr": pk.suppy_csr, "suppy_opts": pk.suppy_opts,
               "suppy_params": pk.suppy_params, "suppy_stats": pk.suppy_stats,
               "suppy_info": pk.suppy_info, "suppy_server_opts": pk.suppy_server_opts,
               "suppy_request_info": pk.suppy_request_info, "suppy_dvc": pk.suppy_dvc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "suppy.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            cname = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {cname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)
