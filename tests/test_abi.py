"""The C-ABI library builds, loads and exports every entry point that
include/are.h declares; the binding's structs match the header's layout.
No compute call is made (these run without a GPU)."""
import ctypes as C
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "are.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"ARE_API\s+[^;]*?\b(are_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libare():
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_1308_2066_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("are_create", "are_destroy", "are_last_error", "are_load_yet",
                     "are_load_elt", "are_define_layer", "are_prepare", "are_simulate",
                     "are_risk_measures"):
        assert required in names


def test_library_exports_every_declared_symbol(libare):
    for name in declared_functions():
        assert hasattr(libare, name), f"{name} is declared in are.h but not exported"


def test_binding_covers_every_declared_symbol():
    import paper_1308_2066_gb300 as are
    for name in declared_functions():
        assert name in are._SIGS, f"binding has no signature for {name}"
        assert callable(getattr(are, name)), name


def test_struct_layouts():
    import paper_1308_2066_gb300 as are
    assert C.sizeof(are.FinTerms) == 32 and C.sizeof(are.LayerTerms) == 32
    assert [f for f, _ in are.FinTerms._fields_] == ["fx", "deductible", "limit", "share"]
    assert [f for f, _ in are.LayerTerms._fields_] == ["occ_ret", "occ_lim", "agg_ret", "agg_lim"]


def test_status_codes_match_header():
    import paper_1308_2066_gb300 as are
    src = open(HEADER).read()
    for name, value in re.findall(r"#define (ARE_E\w+|ARE_OK) (\d+)", src):
        assert getattr(are, name) == int(value)
    assert int(re.search(r"ARE_MAX_ELTS_PER_LAYER (\d+)", src).group(1)) == are.ARE_MAX_ELTS_PER_LAYER


def test_no_gpu_means_an_error_status_not_a_crash(libare):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1308_2066_gb300 as are
    with pytest.raises(are.AreError) as e:
        are.are_create(0)
    assert e.value.status == are.ARE_ECUDA
    assert are.lib().are_destroy(None) == 0
    assert are.lib().are_simulate(None, 1, 1, 0, 1, 0, None, None) == are.ARE_EINVAL


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1308_2066_gb300 as are
    monkeypatch.setattr(are, "_lib", None)
    monkeypatch.setattr(are, "LIB_PATH", str(tmp_path / "libare.so"))
    with pytest.raises(RuntimeError, match="missing"):
        are.lib()


def test_struct_layouts_match_the_header(tmp_path):
    """Compile a C program that prints sizeof/offsetof of every public struct
    and compare with the binding's ctypes definitions."""
    import paper_1308_2066_gb300 as are
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"are_fin_terms": are.FinTerms, "are_layer_terms": are.LayerTerms,
               "are_tune_result": are.TuneResult, "are_server_cfg": are.ServerCfg,
               "are_request": are.Request, "are_result": are.Result}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "are.h"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
