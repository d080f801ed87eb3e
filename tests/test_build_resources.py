"""Resource assumptions of the launchers, checked from the compiler's own report
(nvcc -Xptxas -v) on the CPU: the tensor-core kernel (192 threads, one CTA per
SM by its shared memory) needs no more than 255 registers per thread and must not
spill; no hot kernel may spill."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_04406_gb300", "csrc")


def ptxas_report(src):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = subprocess.run(
        [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
         f"-I{os.path.join(ROOT, 'include')}", "-Xptxas", "-v", "-c", os.path.join(CSRC, src),
         "-o", os.devnull], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    report = {}
    current = None
    for line in out.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            current = m.group(1)
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and current:
            report.setdefault(current, {})["regs"] = int(m.group(1))
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and current:
            report.setdefault(current, {})["spill"] = int(m.group(1)) + int(m.group(2))
    return report


def test_tensor_core_kernel_does_not_spill():
    rep = ptxas_report("kernels_tcx.cu")
    tc = [v for k, v in rep.items() if "tcx3_kernel" in k]
    assert tc, rep
    assert tc[0]["regs"] <= 255 and tc[0].get("spill", 0) == 0


@pytest.mark.parametrize("src", ["kernels_gemm32.cu", "kernels_sddmm.cu", "kernels_df64.cu", "kernels_tcx.cu"])
def test_hot_kernels_do_not_spill(src):
    rep = ptxas_report(src)
    assert rep
    spills = {k: v.get("spill", 0) for k, v in rep.items() if v.get("spill", 0) > 0}
    assert not spills, spills
