"""Register budgets of the kernels whose residency the throughput depends on,
read from ptxas's resource report of a cross-compile (no GPU needed):

* k_analyze2<float, 2, texture>: 192 threads, four CTAs per SM need at most
  80 registers (4 x 192 x 80 <= 65,536), and no spills;
* k_newton<float, plain>: 256 threads, two CTAs per SM need at most 128;
* k_soft_tile<4, 8, 36>: 324 threads (11 warps), two CTAs per SM need at
  most 93 registers (2 x 352 x 93 <= 65,536).
A change that crosses a budget drops a CTA per SM from every wave."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2603_15285_gb300", "csrc")


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def _resources(src, tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "--expt-relaxed-constexpr", "-Xptxas", "-v", "-c", os.path.join(CSRC, src),
           "-o", str(tmp_path / (src + ".o"))]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, cur = {}, None
    for line in (r.stdout + r.stderr).splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            cur = m.group(1)
            out[cur] = {"spill": 0}
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            out[cur]["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            out[cur]["regs"] = int(m.group(1))
    return out


def _one(res, pattern):
    hits = [v for k, v in res.items() if re.search(pattern, k)]
    assert len(hits) == 1, (pattern, sorted(res))
    return hits[0]


@pytest.mark.parametrize("src,pattern,budget", [
    ("analyze.cu", r"k_analyze2IfLi2ELb1E", 80),
    ("newton.cu", r"k_newtonIfLb0E", 128),
    ("soft.cu", r"k_soft_tileILi4ELi8ELi36E", 93),
], ids=["analysis", "refinement", "soft_tile"])
def test_register_budget(src, pattern, budget, tmp_path):
    k = _one(_resources(src, tmp_path), pattern)
    assert k["regs"] <= budget, k
    assert k["spill"] == 0, k
