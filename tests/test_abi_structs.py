"""The binding's ctypes structures mirror the C structs of include/gpubp.h field by field (name,
order and type), so a field added to one side alone fails here, without a GPU."""
import ctypes as C
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CTYPE = {"int32_t": C.c_int32, "uint32_t": C.c_uint32, "int64_t": C.c_int64, "uint64_t": C.c_uint64,
         "double": C.c_double, "float": C.c_float}

PAIRS = {"bp_params": "BpParams", "bp_result": "BpResult", "probe_cache": "ProbeCache",
         "probe_apply_result": "ProbeApplyResult", "bp_tuning": "BpTuning", "bp_tune_report": "BpTuneReport",
         "fp_params": "FpParams", "fp_cache": "FpCache", "fp_result": "FpResult", "pdhg_params": "PdhgParams",
         "pdhg_result": "PdhgResult", "ls_params": "LsParams", "ls_result": "LsResult",
         "ls_obj_params": "LsObjParams", "ls_obj_result": "LsObjResult", "efp_params": "EfpParams",
         "efp_result": "EfpResult"}


def header_structs():
    text = open(os.path.join(ROOT, "include", "gpubp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(const\s+)?([\w]+)\s*(\*?)\s*(\w+)$", decl)
            assert m, (name, decl)
            fields.append((m.group(4), m.group(2), bool(m.group(3))))
        out[name] = fields
    return out


def test_every_header_struct_has_a_mirror():
    assert set(header_structs()) == set(PAIRS)


def test_mirrors_match_field_by_field():
    import paper_2510_20499_gb300 as pkg
    hs = header_structs()
    for cname, pyname in PAIRS.items():
        py = getattr(pkg, pyname)._fields_
        assert [f for f, _ in py] == [f for f, _, _ in hs[cname]], cname
        for (fname, ctype), (_, htype, ptr) in zip(py, hs[cname]):
            if ptr:
                assert C.sizeof(ctype) == C.sizeof(C.c_void_p), (cname, fname)
            elif htype in PAIRS:   # a nested struct: its own mirror
                assert ctype is getattr(pkg, PAIRS[htype]), (cname, fname, ctype, htype)
            else:
                assert ctype._type_ == CTYPE[htype]._type_, (cname, fname, ctype, htype)
        assert C.sizeof(getattr(pkg, pyname)) > 0


def test_c_layout_equals_the_mirrors():
    """A C program compiled against the header prints every field's offset and every struct's
    size; the ctypes mirrors have the same layout (padding and widths included)."""
    import paper_2510_20499_gb300 as pkg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    hs = header_structs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gpubp.h"', "int main(void) {"]
    for cname in PAIRS:
        lines.append(f'printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _, _ in hs[cname]:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        cname, fname, val = line.split()
        cls = getattr(pkg, PAIRS[cname])
        want = C.sizeof(cls) if fname == "." else getattr(cls, fname).offset
        assert int(val) == want, (cname, fname, int(val), want)
