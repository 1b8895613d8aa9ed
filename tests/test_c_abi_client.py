"""The C ABI from plain C: a client that includes only include/kpp.h is compiled with gcc, linked against
libkpp.so and run (host-only entry points, no GPU), and its answers match the Python binding's."""
import os
import shutil
import subprocess

import pytest

from paper_2501_11673_gb300 import build as kbuild
from paper_2501_11673_gb300 import kpp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client_links_and_runs(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    lib = kbuild.build()
    libdir = os.path.dirname(lib)
    exe = tmp_path / "host_client"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi", "host_client.c"), "-o", str(exe),
                           "-L", libdir, "-l:libkpp.so", f"-Wl,-rpath,{libdir}"])
    out = dict(ln.split(" ", 1) for ln in subprocess.check_output([str(exe)], text=True).splitlines())
    assert out["partition_rc"] == "0" and out["partition_blocks"] == "11"
    assert out["bad_partition_rc"] == str(kpp.ERR_ARG) and out["last_error_mentions_call"] == "1"
    assert out["default_tol"] == "1.0e-08" and out["default_max_outer"] == "20"
    assert out["status_string"] == "KPP_ERR_NOT_SPD"
    blocks, subsets, nb = kpp.memo_sequence(11, 0, True, 256, 256, 16, 0, 64)
    assert out["memo_rc"] == "0" and int(out["memo_first_block"]) == int(blocks[0]) and int(out["memo_blocks"]) == nb
