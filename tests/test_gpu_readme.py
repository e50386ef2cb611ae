"""The Python example of README.md runs as written: it steps the 64 x 64,
p = 5 standing mode and sets up the mixed-precision mapped problem; the
energy it prints stays within the upwind flux's slight decay of the
standing mode's exact energy (pi^2 / 4 for u = sin(pi x) sin(pi y), v = 0)."""
import contextlib
import io
import os
import re

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert len(blocks) == 1, "README holds one Python example"
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        exec(compile(blocks[0], "README.md", "exec"), {})
    E = float(out.getvalue().split()[0])
    E0 = 3.141592653589793 ** 2 / 4
    assert 0.999 * E0 < E <= E0 * (1 + 1e-9), (E, E0)
