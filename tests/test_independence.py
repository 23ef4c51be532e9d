"""The oracle and the GPU path share no code: no module of the package imports the oracle, no
CUDA or C source of the package includes an oracle header, and the oracle neither imports the
package nor includes its headers (the seeded input generators, `synth`, serve the tests only)."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2510_20499_gb300")
ORC = os.path.join(ROOT, "oracle")


def _py_imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def _files(top, exts):
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_build", "__pycache__"))]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_package_does_not_import_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in _py_imports(f), f


def test_package_sources_include_no_oracle_header():
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    for f in _files(PKG, (".cu", ".cuh", ".h", ".c", ".cpp")):
        for h in inc.findall(open(f).read()):
            assert "oracle" not in h, (f, h)


def test_oracle_does_not_import_the_package():
    for f in _files(ORC, (".py",)):
        assert "paper_2510_20499_gb300" not in _py_imports(f), f


def test_oracle_sources_include_no_package_header():
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    package_headers = {os.path.basename(x) for x in _files(PKG, (".h", ".cuh"))} | {"gpubp.h"}
    for f in _files(ORC, (".c", ".h")):
        for h in inc.findall(open(f).read()):
            assert "/" not in h and h not in package_headers, (f, h)
