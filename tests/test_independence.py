"""The CPU oracle and the CUDA path share no code (no GPU).

The oracle (oracle/: orc.c, hyperbolic.py and their binding) is test
infrastructure.  These checks read the sources: the package never imports,
includes, links or names the oracle's files; the oracle never imports the
package or includes its headers; bench.py and the entry module call the
oracle only from their CPU-baseline, reference-arm, build and smoke
functions; the one shared module (workloads.py, seeded inputs) imports
neither side; and the binding raises when its CUDA library is missing instead
of falling back to anything else.
"""
import ast
import os
import re

import pytest


def _read_text(path):
    with open(path) as fh:
        return fh.read()


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_0901_0638_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if x not in ("__pycache__", "_lib")]
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _code(path):
    """The file's text without comments and docstrings (Python) or comments (C)."""
    text = _read_text(path)
    if path.endswith(".py"):
        tree = ast.parse(text)
        for node in ast.walk(tree):
            body = getattr(node, "body", None)
            if isinstance(body, list) and body and isinstance(body[0], ast.Expr) \
                    and isinstance(getattr(body[0], "value", None), ast.Constant) \
                    and isinstance(body[0].value.value, str):
                body[0].value.value = ""
        return ast.unparse(tree)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def test_package_never_reaches_the_oracle():
    pat = re.compile(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|orc\.h|liborc|['\"/]oracle['\"/]|__import__\(\s*['\"]oracle")
    found = [p for p in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".c", ".cpp")) if pat.search(_code(p))]
    assert not found, found


def test_oracle_never_reaches_the_package():
    pat = re.compile(r"paper_0901_0638_gb300|\bqm\.h\b|\bqm_\w+\.(h|cuh|cu)\b|libqm|\bworkloads\b")
    found = [p for p in _sources(ORACLE, (".py", ".c", ".h")) if pat.search(_code(p))]
    assert not found, found


def test_shared_input_module_imports_neither_side():
    tree = ast.parse(_read_text(os.path.join(PKG, "workloads.py")))
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add("." if node.level else (node.module or "").split(".")[0])
    assert not mods & {"oracle", ".", "paper_0901_0638_gb300", "ctypes"}, mods


@pytest.mark.parametrize("path, allowed", [
    ("bench.py", {"cpu_oracle_leg", "reference_sample", "run_reference"}),
    ("__graft_entry__.py", {"build", "smoke"}),
])
def test_oracle_called_only_from_baseline_build_and_smoke(path, allowed):
    tree = ast.parse(_read_text(os.path.join(ROOT, path)))
    users = set()

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                users.add(fn)
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                users.add(fn)
            visit(child, name)

    visit(tree, None)
    assert None not in users, f"{path}: the oracle is imported at module level"
    assert users <= allowed, users - allowed


def test_binding_raises_when_the_cuda_library_is_missing(tmp_path, monkeypatch):
    import paper_0901_0638_gb300 as qm
    monkeypatch.setattr(qm, "_lib", None)
    monkeypatch.setattr(qm, "LIB_PATH", str(tmp_path / "libqm.so"))
    with pytest.raises(RuntimeError, match="missing"):
        qm.load(build_if_missing=False)
