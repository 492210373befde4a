"""The README's Python example runs as written (its API names and call
shapes stay in step with the binding)."""
import os
import re

import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_runs():
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert len(blocks) == 1
    ns = {}
    exec(compile(blocks[0], "README.md", "exec"), ns)
    assert ns["w"].shape == (2048, 2048) and ns["records"].shape == (1000, 2)
    assert ns["eta"].shape == (2000, 16)
    assert ns["img"].shape == (2048, 2048, 4)
    assert ns["dL_dw0"].shape == (512, 512) and ns["dL_dz"].shape == (512, 512)
