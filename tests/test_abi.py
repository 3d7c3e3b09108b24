"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports every
function include/stencil.h declares, and the Python binding names exactly those functions."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(stencil_\w+)\s*\(", src, re.M))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._engine_build_module().build()


def test_header_functions_exported(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names |= _declared(h)
    assert "stencil_run" in names and "stencil_plan_create" in names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_header(lib_path):
    import paper_1802_00438_gb300 as st
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names |= _declared(h)
    assert names == set(st.SIGNATURES), names ^ set(st.SIGNATURES)


_CTYPES = {"int": ctypes.c_int, "long long": ctypes.c_longlong, "double": ctypes.c_double,
           "float": ctypes.c_float, "void *": ctypes.c_void_p, "size_t": ctypes.c_size_t}


def _structs(header):
    """{typedef name: [(field, C type, array length)]} of the header's plain structs."""
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(long long|unsigned int|int|double|float|size_t|void \*|const \w+ \*)\s*(.*)", decl)
            assert m, decl
            ctype = m.group(1)
            for item in m.group(2).split(","):
                item = item.strip()
                star = item.startswith("*")
                item = item.lstrip("*").strip()
                am = re.match(r"(\w+)(?:\[(\d+)\])?$", item)
                assert am, item
                fields.append((am.group(1), "void *" if star else ctype,
                               int(am.group(2)) if am.group(2) else 0))
        out[name] = fields
    return out


def test_binding_structs_match_header(lib_path):
    # every struct of the header has a ctypes twin with the same fields, in order, of the same
    # types: a field added on one side only would shift everything after it
    import paper_1802_00438_gb300 as st
    structs = _structs("stencil.h")
    assert {"stencil_desc", "stencil_plan_info", "stencil_tune_result"} <= set(structs)
    for name, fields in structs.items():
        twin = getattr(st, name)
        got = [(f, t) for f, t in twin._fields_]
        assert [f for f, _ in got] == [f for f, _, _ in fields], name
        for (f, t), (_, ctype, n) in zip(got, fields):
            want = _CTYPES.get(ctype, ctypes.c_void_p)
            if n:
                assert t._type_ is want and t._length_ == n, (name, f)
            else:
                assert ctypes.sizeof(t) == ctypes.sizeof(want), (name, f)


def test_host_only_calls(lib_path):
    import paper_1802_00438_gb300 as st
    assert st.lib.stencil_abi_version() == 4
    assert st.strerror(0) == "ok"
    assert "dimensions" in st.strerror(st.ST_ERR_DIMS_MISMATCH)
    assert st.strerror(12345) == "unknown status"
    # argument validation happens before any device work
    assert st.lib.stencil_plan_create(None, None) == st.ST_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    bad = st.stencil_desc(7, 2, 8, 8, 1, 0, 0, 0, 0, 0, 0, 0, None)
    assert st.lib.stencil_plan_create(ctypes.byref(h), ctypes.byref(bad)) == st.ST_ERR_INVALID_ARG
    bad = st.stencil_desc(0, 4, 8, 8, 1, 0, 0, 0, 0, 0, 0, 0, None)
    assert st.lib.stencil_plan_create(ctypes.byref(h), ctypes.byref(bad)) == st.ST_ERR_INVALID_ARG
    bad = st.stencil_desc(0, 2, 0, 8, 1, 0, 0, 0, 0, 0, 0, 0, None)
    assert st.lib.stencil_plan_create(ctypes.byref(h), ctypes.byref(bad)) == st.ST_ERR_INVALID_ARG
    assert st.lib.stencil_run(None, None, None, None, None, 1, 1, 1, 1) == st.ST_ERR_INVALID_ARG
    assert st.lib.stencil_plan_destroy(None) == st.ST_OK
    # allocation-failure hook: argument checks and the live count need no device
    assert st.lib.stencil_debug_fail_alloc(-1) == st.ST_ERR_INVALID_ARG
    assert st.lib.stencil_debug_fail_alloc(0) == st.ST_OK
    assert st.lib.stencil_debug_live_allocs() >= 0


def test_no_oracle_in_product():
    """The engine package never imports, links or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_1802_00438_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in txt.lower().replace("oracle's", ""), os.path.join(dp, f)


class _FakeGrid:
    """Stands in for a CUDA tensor in the binding's size and device checks: those checks run
    before the binding takes an address or calls the library, so nothing is launched."""

    def __init__(self, n, device):
        self.n, self.device_index = n, device

    def numel(self):
        return self.n

    def get_device(self):
        return self.device_index


def test_binding_refuses_short_or_foreign_tensors(lib_path, monkeypatch):
    import torch

    import paper_1802_00438_gb300 as st
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    ok = _FakeGrid(64 * 32, 0)
    short = _FakeGrid(64 * 32 - 1, 0)
    other = _FakeGrid(64 * 32, 1)
    for args in ((short, ok, None), (ok, short, None), (other, ok, None), (ok, other, None)):
        with pytest.raises(ValueError):
            st.stencil_run_noalloc(0, *args, [0.2] * 5, 64, 32, 3)
    with pytest.raises(ValueError):                       # short power map
        st.stencil_run_noalloc(1, ok, _FakeGrid(64 * 32, 0), short, [0.5, 0.1, 0.1, 1e-4, 80.0],
                               64, 32, 3)
    with pytest.raises(ValueError):                       # power map on another device
        st.stencil_run_noalloc(1, ok, _FakeGrid(64 * 32, 0), other, [0.5, 0.1, 0.1, 1e-4, 80.0],
                               64, 32, 3)
    # the plan wrapper applies the same checks (a plan object needs no device to be checked)
    plan = st.Plan.__new__(st.Plan)
    plan.kind, plan.ndim, plan.nx, plan.ny, plan.nz, plan.h = 2, 2, 64, 32, 1, None
    with pytest.raises(ValueError):                       # five coefficient planes expected
        plan.run(ok, _FakeGrid(64 * 32, 0), None, 1, power=_FakeGrid(4 * 64 * 32, 0))
