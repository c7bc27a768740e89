"""The product path has no CPU fallback: without the CUDA library the binding raises, and nothing in the package
imports the oracle (only the tests, the smoke check and the benchmark's CPU-baseline leg may)."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2407_19151_gb300")


def test_missing_library_raises():
    code = ("import paper_2407_19151_gb300._binding as B\n"
            "try:\n    B.lib()\nexcept RuntimeError as e:\n    print('raised:', e)\nelse:\n    print('loaded')\n")
    env = dict(os.environ, MCC_LIBRARY=os.path.join(ROOT, "_build_missing", "libmcc.so"))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised:") and "not built" in out.stdout


def _imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            names.add(node.module.split(".")[0])
    return names


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                assert "oracle" not in _imports(os.path.join(dirpath, f)), f


def test_bench_imports_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    allowed = {"cpu_baseline"}
    for node in tree.body:
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            mods = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
            assert not any(m.split(".")[0] == "oracle" for m in mods)
        if isinstance(node, ast.FunctionDef) and node.name not in allowed:
            for sub in ast.walk(node):
                if isinstance(sub, ast.Import):
                    assert not any(a.name.split(".")[0] == "oracle" for a in sub.names), node.name
                if isinstance(sub, ast.ImportFrom) and sub.module:
                    assert sub.module.split(".")[0] != "oracle", node.name
