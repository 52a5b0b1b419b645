"""The debug build (CGH_DEBUG: device-side bounds checks that latch a status bit and skip the access instead
of faulting) on the small parity cases: the 256x256 and ragged holograms in every form and a persistent batch,
in a process of its own that loads libcgh_debug.so; every status must stay clear."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_small_cases_clear():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_2734_gb300.build import build
    lib = build(debug=True)
    assert lib.endswith("libcgh_debug.so")
    env = dict(os.environ, CGH_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_build_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "all cases clear" in r.stdout
