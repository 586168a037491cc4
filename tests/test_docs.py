"""The README's usage instructions against the code (CPU only): its Python example
compiles and imports names that exist, every C entry point it names is exported by
the binding, and the build script flags it mentions are the ones the script reads."""
import ast
import importlib
import importlib.util
import os
import re

ROOT = os.path.join(os.path.dirname(__file__), "..")


def readme():
    with open(os.path.join(ROOT, "README.md")) as f:
        return f.read()


def test_python_example_compiles_and_its_imports_exist():
    blocks = re.findall(r"```python\n(.*?)```", readme(), re.S)
    assert blocks
    for code in blocks:
        tree = ast.parse(code)
        for node in ast.walk(tree):
            if isinstance(node, ast.ImportFrom):
                mod = importlib.import_module(node.module)
                for a in node.names:
                    assert hasattr(mod, a.name) or importlib.util.find_spec(f"{node.module}.{a.name}"), \
                        f"{node.module}.{a.name}"


def test_named_entry_points_are_exported():
    from paper_2602_22625_gb300 import dbmp
    names = set(re.findall(r"\b(dbmp_[a-z0-9_]+)\b", readme()))
    assert {"dbmp_batch_render", "dbmp_batch_render_mse", "dbmp_adam_step", "dbmp_status_poll"} <= names
    for n in names:
        assert hasattr(dbmp, n), n


def test_build_flags_exist():
    with open(os.path.join(ROOT, "paper_2602_22625_gb300", "_build.py")) as f:
        src = f.read()
    for flag in re.findall(r"_build\.py ((?:--?\w+ ?)+)", readme())[0].split():
        assert f'"{flag}" in sys.argv' in src, flag
