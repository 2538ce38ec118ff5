"""The README's Python examples stay valid Python against the current API
names (they are executed on a GPU as a whole; here only parsed, and every
`lv.` / `LS.` / `V.` attribute they use must exist)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _blocks():
    src = open(os.path.join(ROOT, "README.md")).read()
    return re.findall(r"```python\n(.*?)```", src, re.S)


def test_readme_has_examples():
    assert len(_blocks()) >= 5


@pytest.mark.parametrize("i", range(5))
def test_readme_example_parses_and_names_exist(i):
    pytest.importorskip("torch")
    from paper_1707_01170_gb300 import learned as LS
    from paper_1707_01170_gb300 import lrvol as lv
    from paper_1707_01170_gb300.synth import volumes as V
    mods = {"lv": lv, "LS": LS, "V": V}
    tree = ast.parse(_blocks()[i])
    for node in ast.walk(tree):
        if isinstance(node, ast.Attribute) and isinstance(node.value, ast.Name) and node.value.id in mods:
            assert hasattr(mods[node.value.id], node.attr), f"{node.value.id}.{node.attr}"
