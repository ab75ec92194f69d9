"""The batched kernels' index checks on the GPU: the whole batched test
module runs again in a process of its own against the debug build of the
library (libpsdf_b300_debug.so: every index the batched kernels take from
their data is checked and the first violation recorded), and its last test
asserts that none was recorded -- a bounds-checking stand-in that needs no
sanitizer."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

from paper_2607_04310_b300 import psdf

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batched_module_under_the_index_checking_build():
    assert os.path.exists(psdf.LIB_DEBUG_PATH), "debug library not built"
    env = dict(os.environ, PSDF_LIBRARY=psdf.LIB_DEBUG_PATH)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-rs", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_gpu_batched.py"), "-m", "gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-3000:]
    # every test ran, the last one reading the debug word (under the release
    # build it is skipped)
    summary = [line for line in out.splitlines() if " passed" in line][-1]
    assert "skipped" not in summary and "deselected" not in summary, out[-3000:]
