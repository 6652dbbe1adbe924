"""The C-ABI library builds, loads and exports every symbol of include/sgmf.h.

CPU only: nothing here launches a kernel.
"""
import ctypes
import os
import re

import pytest

from paper_2504_05148_gb300 import build, sgmf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(sgmf_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("sgmf_create", "sgmf_set_params", "sgmf_compute", "sgmf_destroy", "sgmf_compute_host",
                 "sgmf_sync", "sgmf_last_error", "sgmf_debug_stage", "sgmf_default_params"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the same set
    assert sorted(sgmf.EXPORTS) == _declared_functions()


def test_default_params_are_table_ii(libpath):
    p = sgmf.sgmf_default_params()
    assert (p.p1, p.p2, p.q1, p.q2) == (10, 120, 5, 160)
    assert (p.alpha_num, p.alpha_den) == (7, 10)
    assert (p.ts, p.rs, p.tc, p.rc) == (2, 6, 2, 20)
    assert p.num_paths == 8 and p.semidense == 1 and p.lr_max_diff == 1
    assert p.subpixel == 0


def _int32_fields(struct_name):
    import re
    src = open(os.path.join(ROOT, "include", "sgmf.h")).read()
    body = re.search(r"typedef struct \{([^{}]*?)\} " + struct_name + ";", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        assert decl.startswith("int32_t "), decl
        names += [n.strip() for n in decl[len("int32_t "):].split(",")]
    return names


def test_params_struct_matches_header_field_order():
    """The ctypes mirror lists the header's sgmf_params fields in order (all int32)."""
    assert [f[0] for f in sgmf.sgmf_params._fields_] == _int32_fields("sgmf_params")


def test_tuning_and_shape_structs_match_header():
    assert [f[0] for f in sgmf.sgmf_tuning._fields_] == _int32_fields("sgmf_tuning")
    assert [f[0] for f in sgmf.sgmf_shape._fields_] == _int32_fields("sgmf_shape")


def test_rates_struct_matches_header():
    """sgmf_rates: one int (sms), then doubles in the header's order."""
    h = open(os.path.join(ROOT, "include", "sgmf.h")).read()
    body = h[h.index("typedef struct {\n  int sms;"):]
    body = body[:body.index("} sgmf_rates;")]
    names = [ln.split(";")[0].split()[-1] for ln in body.splitlines()[1:] if ";" in ln]
    assert [f[0] for f in sgmf.sgmf_rates._fields_] == names
    assert sgmf.sgmf_rates._fields_[0][1] is ctypes.c_int


def test_status_strings(libpath):
    assert sgmf.lib().sgmf_status_string(sgmf.SGMF_ERR_PARAM) == b"SGMF_ERR_PARAM"
    assert sgmf.lib().sgmf_status_string(sgmf.SGMF_OK) == b"SGMF_OK"


def test_create_rejects_bad_shapes_without_touching_the_gpu(libpath):
    for w, h, d in ((0, 10, 16), (10, 0, 16), (10, 10, 0), (10, 10, 257), (9000, 10, 16)):
        with pytest.raises(sgmf.SgmfError) as e:
            sgmf.sgmf_create(w, h, d)
        assert e.value.status == sgmf.SGMF_ERR_SHAPE
    assert sgmf.lib().sgmf_create(8, 8, 8, None) == sgmf.SGMF_ERR_ARG


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(sgmf, "_lib", None)
    with pytest.raises(FileNotFoundError):
        sgmf.lib(str(tmp_path / "missing.so"))
