"""The C ABI: the library builds for sm_103a, loads, exports every symbol the
headers declare, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import dataclasses
import glob
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from paper_1010_2438_gb300 import capi
from paper_1010_2438_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cwc_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not capi.lib_exists():
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        from paper_1010_2438_gb300 import build
        build.build()
    return capi.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("cwc_model_create", "cwc_model_destroy", "cwc_simulate", "cwc_sensitivity", "cwc_last_error"):
        assert n in names
    assert set(capi.EXPORTED) <= names


def test_library_exports_every_declared_symbol(lib):
    for n in sorted(declared_functions()):
        assert hasattr(lib, n), n


def test_version(lib):
    assert "sm_103a" in capi.cwc_version()


def _desc(model):
    m = model.contiguous()
    keep = (m.kind, m.ctx_label, m.child_label, m.lhs, m.rhs, m.rate_law, m.rate_par)
    d = capi.cwc_model_desc(m.n_species, m.n_labels, m.n_rules, m.max_compartments,
                            *(a.ctypes.data for a in keep[:5]))
    d.rate_law = None if m.rate_law is None else m.rate_law.ctypes.data
    d.rate_par = None if m.rate_par is None else m.rate_par.ctypes.data
    return d, keep


def test_model_validation_on_host(lib):
    out = ctypes.c_void_p()
    assert lib.cwc_model_create(None, ctypes.byref(out)) == capi.CWC_ERR_INVALID_ARG
    assert "NULL" in capi.cwc_last_error()
    base = W.flat8x12(R=1).model
    cases = []
    m = base.contiguous()
    bad = W.Model(m.n_species, m.n_labels, m.max_compartments, m.kind.copy(), m.ctx_label, m.child_label,
                  m.lhs, m.rhs)
    bad.kind[0] = 9
    cases.append((bad, capi.CWC_ERR_INVALID_ARG, "kind"))
    bad = W.Model(m.n_species, m.n_labels, m.max_compartments, m.kind, m.ctx_label, m.child_label,
                  m.lhs.copy(), m.rhs)
    bad.lhs[0, 0, 0] = 3
    cases.append((bad, capi.CWC_ERR_INVALID_ARG, "lhs"))
    bad = W.Model(m.n_species, m.n_labels, m.max_compartments, m.kind, m.ctx_label, m.child_label,
                  m.lhs.copy(), m.rhs)
    bad.lhs[0, 0, :5] = 1
    cases.append((bad, capi.CWC_ERR_UNSUPPORTED, "4 reactant"))
    bad = W.Model(m.n_species, m.n_labels, m.max_compartments, m.kind, m.ctx_label, m.child_label,
                  m.lhs, m.rhs.copy())
    bad.rhs[0, 1, 0] = 1
    cases.append((bad, capi.CWC_ERR_INVALID_ARG, "LOCAL"))
    bad = W.Model(m.n_species, 1, 1, np.full(m.n_rules, 1, np.int32), m.ctx_label, m.child_label, m.lhs, m.rhs)
    cases.append((bad, capi.CWC_ERR_INVALID_ARG, "child_label"))
    bad = W.Model(0, 1, 1, m.kind, m.ctx_label, m.child_label, m.lhs, m.rhs)
    cases.append((bad, capi.CWC_ERR_INVALID_ARG, "sizes"))
    for model, code, text in cases:
        d, keep = _desc(model)
        rc = lib.cwc_model_create(ctypes.byref(d), ctypes.byref(out))
        assert rc == code, (rc, capi.cwc_last_error())
        assert text in capi.cwc_last_error()
        assert out.value is None


def test_simulate_argument_checks_on_host(lib):
    args = capi.cwc_sim_args()
    assert lib.cwc_simulate(None, ctypes.byref(args), None) == capi.CWC_ERR_INVALID_ARG
    assert lib.cwc_sensitivity(None, ctypes.byref(args), None, None) == capi.CWC_ERR_INVALID_ARG
    n = ctypes.c_size_t()
    assert lib.cwc_simulate_workspace_size(None, ctypes.byref(args), ctypes.byref(n)) == capi.CWC_ERR_INVALID_ARG
    assert lib.cwc_model_num_observables(None) == -1
    lib.cwc_model_destroy(None)  # NULL is ignored


def _header_struct_fields(name):
    """(field, is_pointer, base type) of a typedef'd struct in the header."""
    text = open(os.path.join(ROOT, "include", "cwcgpu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, rest = re.match(r"(?:const\s+)?([A-Za-z_0-9]+)\s*(.*)", decl).groups()
        for nm in rest.split(","):
            nm = nm.strip()
            fields.append((nm.lstrip("*").strip(), nm.startswith("*"), typ))
    return fields


@pytest.mark.parametrize("name", ["cwc_sim_args", "cwc_sens_args", "cwc_model_desc"])
def test_ctypes_structs_follow_the_header(name):
    """Field names, order and widths of the Python mirror equal the C
    declarations, so the binding passes what the library reads."""
    sizes = {"int32_t": 4, "uint32_t": 4, "int64_t": 8, "uint64_t": 8, "size_t": 8, "double": 8}
    hdr = _header_struct_fields(name)
    py = getattr(capi, name)._fields_
    assert [f[0] for f in hdr] == [f[0] for f in py]
    for (nm, is_ptr, typ), (_, ctype) in zip(hdr, py):
        want = 8 if is_ptr else sizes[typ]
        assert ctypes.sizeof(ctype) == want, nm


@pytest.mark.parametrize("name", ["cwc_sim_args", "cwc_sens_args", "cwc_model_desc"])
def test_ctypes_struct_offsets_equal_the_compiled_header(name, tmp_path):
    """Every field's offset and the struct's size, as a C compiler lays out
    the header's declaration, equal the ctypes mirror's (padding included)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    fields = [f[0] for f in _header_struct_fields(name)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cwcgpu.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(' + name + '));']
    lines += ['  printf("%zu\\n", offsetof(' + name + ', ' + f + '));' for f in fields]
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I" + os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True,
                   capture_output=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    py = getattr(capi, name)
    assert got[0] == ctypes.sizeof(py)
    assert got[1:] == [getattr(py, f).offset for f in fields]


def test_michaelis_menten_validation_on_host(lib):
    """Michaelis-Menten rules are LOCAL rules of flat models with one or two
    reactant species of multiplicity 1, the substrate among them, and a
    finite K > 0; anything else is refused before any device work."""
    out = ctypes.c_void_p()
    conv = ({0: 1, 2: 1}, {1: 1, 2: 1})
    ok = W.flat_model(3, [conv], michaelis_menten={0: (0, 10.0)})
    cases = [
        (W.flat_model(3, [conv], michaelis_menten={0: (0, 0.0)}), "K"),
        (W.flat_model(3, [conv], michaelis_menten={0: (0, float("inf"))}), "K"),
        (W.flat_model(3, [conv], michaelis_menten={0: (1, 10.0)}), "substrate"),       # product, not a reactant
        (W.flat_model(3, [({0: 2}, {1: 1})], michaelis_menten={0: (0, 10.0)}), "multiplicity"),
        (W.flat_model(3, [({}, {1: 1})], michaelis_menten={0: (0, 10.0)}), "substrate"),
    ]
    bad = dataclasses.replace(ok.contiguous(), rate_law=np.array([4], np.int32))
    cases.append((bad, "rate_law"))
    # a compartment model (two labels) may not use the law
    comp = dataclasses.replace(ok.contiguous(), n_labels=2, max_compartments=4)
    cases.append((comp, "flat"))
    for model, text in cases:
        d, keep = _desc(model)
        rc = lib.cwc_model_create(ctypes.byref(d), ctypes.byref(out))
        assert rc == capi.CWC_ERR_INVALID_ARG, (text, rc, capi.cwc_last_error())
        assert "Michaelis-Menten" in capi.cwc_last_error() or "rate_law" in capi.cwc_last_error(), text
        assert out.value is None
