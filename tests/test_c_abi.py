"""include/mz.h as a C99 header: tests/c_abi_example.c compiles against it with gcc
(-std=c99 -Wall -Werror), links against libmz.so and runs its host-only checks (a plan of
the paper's example, exports, a plan file, the documented errors). No GPU involved."""
import os
import shutil
import subprocess

import pytest

import paper_2211_13706_gb300 as mz

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_program_against_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.dirname(mz.LIBRARY_PATH)
    exe = tmp_path / "c_abi_example"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(HERE, "c_abi_example.c"), "-o", str(exe), "-L", lib_dir, "-lmz",
                        f"-Wl,-rpath,{lib_dir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe), str(tmp_path / "example.mzplan")], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c abi ok" in r.stdout
