"""The C-ABI from C: include/trids.h compiles as C99 and a C program linked against
libtrids.so gets the documented error codes from the entry points that need no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not installed")
def test_c99_program_links_and_calls_the_library(tmp_path):
    from paper_2510_24186_b300 import build
    lib = build.build()
    exe = tmp_path / "capi_consumer"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "capi_consumer.c"), "-L" + os.path.dirname(lib), "-ltrids",
                           "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("OK")
