"""The ABI from plain C: tests/c/abi_host.c is compiled with gcc as C11
against include/ok.h, linked to the library, and run (host-only calls; no GPU)."""
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_1603_04570_gb300 as ok

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_uses_the_abi():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    ok.load()                                        # builds the library if needed
    lib = ok.library_path()
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "abi_host")
        cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
               os.path.join(ROOT, "tests", "c", "abi_host.c"), lib, "-lm",
               f"-Wl,-rpath,{os.path.dirname(lib)}", "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
