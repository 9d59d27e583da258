"""The MZ_DEBUG variant of the library builds for sm_103a and exports the same C ABI
(checked in a child process, which loads it through MZ_LIBRARY=debug; no GPU needed)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CODE = """
import paper_2211_13706_gb300 as mz
assert mz.LIBRARY_PATH.endswith("libmz_debug.so"), mz.LIBRARY_PATH
for name in mz.EXPORTED:
    getattr(mz.lib, name)
assert mz.lib.mz_status_string(mz.MZ_ERR_BOUNDS).decode() == "MZ_ERR_BOUNDS"
print("debug library ok")
"""


def test_debug_library_loads_and_exports_the_abi():
    env = dict(os.environ, MZ_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", CODE], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "debug library ok" in r.stdout
