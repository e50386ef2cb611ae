"""The index-checking build (GDG_CHECKS, gdg_checks.cuh): built by the test
on the machine that runs it, then every form runs on small cases in a child process that loads it; no
element index a kernel derives (face neighbours, neighbour blocks, batched
work items) leaves its range, and the recording path itself works (a
self-test pair that fails records site 99 with its index and bound)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_form_stays_in_range_under_the_checking_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_01722_gb300 import build
    build.build(verbose=False, checks=True)
    env = dict(os.environ, GDG_CHECKS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "gpu_checks_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["selftest"] == {"count": 1, "site": 99, "index": 5, "bound": 3}
    assert out["forms"]["count"] == 0, out["forms"]
