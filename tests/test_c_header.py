"""The public headers compile for a plain C11 caller: a small C program
includes bsfp.h and bsfp_bench.h with no CUDA include path, builds with
-std=c11 -Wall -Wextra -Werror -pedantic, links against libbsfp.so and runs
the host-side calls (sizes, status strings, an op's argument validation), so
no GPU is needed."""
import os
import shutil
import subprocess
import tempfile

import pytest

import paper_1602_04716_gb300 as bs

HERE = os.path.dirname(os.path.abspath(__file__))
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c11_consumer_compiles_links_and_runs():
    lib = bs.lib_path()
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "c_consumer")
        cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", INCLUDE,
               os.path.join(HERE, "c_consumer.c"), "-o", exe, lib,
               "-Wl,-rpath," + os.path.dirname(lib)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stdout + r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("header", ["bsfp.h", "bsfp_bench.h"])
def test_each_header_stands_alone_in_c11(header):
    """Each header parses first in a translation unit, with nothing before it."""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "one.c")
        with open(src, "w") as fh:
            fh.write('#include "%s"\nint main(void) { return 0; }\n' % header)
        r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                            "-I", INCLUDE, src], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
