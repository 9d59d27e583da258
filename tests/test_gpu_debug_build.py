"""The MZ_DEBUG build (libmz_debug.so) on the GPU: bounds-checked kernels and poisoned
workspaces over every plan kind, against the oracle. It runs in a child process, since
one process loads one build of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_cases():
    env = dict(os.environ, MZ_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all debug cases ok" in r.stdout
