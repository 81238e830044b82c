"""Layout rules checked on the committed sources: the product package never
imports the oracle (its results cannot route through the CPU checker), and
the oracle imports nothing of the product or of the CUDA path, so the two
share no code."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_0904_4887_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            if node.level == 0 and node.module:
                names.add(node.module.split(".")[0])
    return names


def _py_files(top):
    for d, _, files in os.walk(top):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(d, f)


def test_product_package_does_not_import_the_oracle():
    files = list(_py_files(PKG))
    assert files
    for f in files:
        assert "oracle" not in _imports(f), f
        text = open(f).read()
        assert "gp_oracle" not in text, f


def test_oracle_does_not_import_the_product():
    for f in _py_files(os.path.join(ROOT, "oracle")):
        imp = _imports(f)
        assert not imp & {"paper_0904_4887_gb300", "torch", "bench", "workloads"}, (f, imp)


def test_cuda_sources_do_not_reference_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f
