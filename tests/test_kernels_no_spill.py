"""Every kernel of libpg compiles for sm_103a without register spills (ptxas
reports 0 spill bytes for each entry function).  A spill in a hot kernel is a
silent slowdown that no parity test sees."""
import os
import re
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2010_01775_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_01775_gb300", "csrc")


def _ptxas_report(src, out):
    cmd = [B.NVCC, *B.ARCH, "-O3", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xptxas", "-v",
           "-c", src, "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stderr


def test_no_kernel_spills(tmp_path):
    if not (os.path.exists(B.NVCC) or shutil.which(B.NVCC)):
        pytest.skip("nvcc not available")
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        reports = list(ex.map(lambda f: _ptxas_report(os.path.join(CSRC, f), str(tmp_path / (f + ".o"))), srcs))
    entries = 0
    for f, rep in zip(srcs, reports):
        for stores, loads in re.findall(r"(\d+) bytes spill stores, (\d+) bytes spill loads", rep):
            entries += 1
            assert int(stores) == 0 and int(loads) == 0, (f, rep[-3000:])
    assert entries >= 20  # every file's entry functions were reported
