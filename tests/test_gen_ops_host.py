"""The list-free split generator (device code, compiled for the host here)
regenerates exactly the stored operations of the builder's lists: same x
index, block index and sign for every split of every output, in order."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


def test_generator_matches_stored_lists(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "gen_ops_check")
    src = os.path.join(ROOT, "tests", "host", "gen_ops_check.cpp")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-I", os.path.join(ROOT, "include"), src,
                           "-o", exe])
    res = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0 and res.stdout.strip().endswith("OK"), res.stdout + res.stderr
