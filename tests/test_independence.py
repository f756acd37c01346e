"""The oracle and the CUDA path stay apart (CPU only, by reading the sources).

  * No module of the package imports the oracle: the product path cannot
    route through it.
  * The CUDA sources include nothing of the oracle, and the oracle's C source
    includes nothing of the library (its header, its kernels).
  * bench.py reaches the oracle only in its CPU-baseline and reference legs,
    and __graft_entry__ only in smoke() and in build() (which compiles it).
  * inputs.py, shared by both sides, imports neither.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2402_15641_gb300")


def _imports(path):
    """[(module, enclosing function or None)] for every import in a file."""
    tree = ast.parse(open(path).read())
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = fn
            if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)):
                name = child.name
            if isinstance(child, ast.Import):
                out.extend((a.name, fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = child.module or ""
                out.extend((f"{mod}.{a.name}" if mod else a.name, fn) for a in child.names)
            visit(child, name)

    visit(tree, None)
    return out


def _is_oracle(mod):
    return mod == "oracle" or mod.startswith("oracle.")


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                path = os.path.join(dirpath, f)
                bad = [m for m, _ in _imports(path) if _is_oracle(m)]
                assert not bad, (path, bad)


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), re.M)


def test_c_sources_share_no_headers():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            inc = _includes(os.path.join(csrc, f))
            assert not [i for i in inc if "oracle" in i or i.startswith("orc")], (f, inc)
    odir = os.path.join(ROOT, "oracle")
    ours = {"srt.h", "common.cuh", "devutil.cuh"}
    for f in os.listdir(odir):
        if f.endswith((".c", ".h")):
            inc = _includes(os.path.join(odir, f))
            assert not [i for i in inc if os.path.basename(i) in ours or "csrc" in i], (f, inc)


def test_oracle_reached_only_by_the_allowed_legs():
    allowed = {"bench.py": {"cpu_oracle_rate", "run_reference"},
               "__graft_entry__.py": {"smoke", "build"}}
    for f, fns in allowed.items():
        for mod, fn in _imports(os.path.join(ROOT, f)):
            if _is_oracle(mod):
                assert fn in fns, (f, mod, fn)


def test_shared_input_module_imports_neither_side():
    mods = [m for m, _ in _imports(os.path.join(PKG, "inputs.py"))]
    assert not [m for m in mods if _is_oracle(m) or "srt" in m or "_lib" in m], mods
