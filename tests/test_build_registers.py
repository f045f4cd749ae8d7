"""The pair kernel's default instances compile for sm_103a without register
spills.  ptxas reports registers and spill bytes per kernel (-Xptxas -v); a
spill in the hot loop costs more than any other single change measured on this
kernel, so this guards edits of the source.  Needs nvcc, not a GPU."""
import os
import re
import shutil
import subprocess

import pytest

from conftest import ROOT

CSRC = os.path.join(ROOT, "paper_0810_2273_gb300", "csrc")

# (precision, MODE (1 = E + v), threads, skewed): the shapes the library launches
# by default, FP32 E + v 448 (384 on skewed cells) and energy 512
DEFAULTS = [("f", 1, 448, 0), ("f", 1, 384, 1), ("f", 0, 512, 0), ("f", 0, 512, 1)]


@pytest.fixture(scope="module")
def ptxas_report(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("ptxas") / "pair.o"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xptxas", "-v", "-c",
           os.path.join(CSRC, "pair.cu"), "-o", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True, check=True)
    report = {}
    name = None
    for line in (r.stdout + r.stderr).splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            name = m.group(1)
            report[name] = {}
            continue
        if name is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            report[name]["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            report[name]["regs"] = int(m.group(1))
    return report


@pytest.mark.parametrize("prec,mode,threads,skew", DEFAULTS)
def test_default_instances_do_not_spill(ptxas_report, prec, mode, threads, skew):
    key = "k_pairI%sLi%dELi%dELb%dE" % (prec, mode, threads, skew)
    hits = [v for k, v in ptxas_report.items() if key in k]
    assert len(hits) == 1, (key, sorted(ptxas_report))
    rep = hits[0]
    assert rep.get("spill", 0) == 0, (key, rep)
    assert rep["regs"] * threads <= 65536, (key, rep)
