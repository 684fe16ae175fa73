"""The index-checking debug build (build.py check=True, -DAIM_CHECK): the
product kernels test every projection entry, near column and stencil before
they use it and report a failure as AIM_EINVAL.  On valid inputs the check
build must give the parity results of the regular one and report nothing;
tests/check_build_run.py exercises it in a process of its own, since a process
loads one build of the library."""

import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_check_build_passes_parity_without_index_failures():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1010_1456_gb300 import build

    build.build(check=True)
    env = dict(os.environ, AIM_LIBRARY="libaim_check.so")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "check_build_run.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.strip().endswith("ok")
