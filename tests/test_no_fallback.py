"""The product path has no CPU fallback: without a CUDA device the binding refuses to load
(and never reaches for the oracle), and neither the package nor its binding imports the
oracle.  Runs where no GPU is visible."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1709_05418_gb300")


def test_binding_refuses_without_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_1709_05418_gb300 import api
    with pytest.raises(RuntimeError, match="no CUDA device"):
        api.load()
    with pytest.raises(RuntimeError):
        api.Context()


def test_package_never_imports_the_oracle():
    for name in sorted(os.listdir(PKG)):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(PKG, name)).read())
        for node in ast.walk(tree):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (name, mods)
    for root, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            src = open(os.path.join(root, f), errors="replace").read()
            assert "rpnn_oracle" not in src and "orc_" not in src, f
