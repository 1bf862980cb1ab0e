"""Register budgets of the kernels whose speed depends on occupancy, read
from ptxas for sm_103a (no GPU needed).  The batched dot kernel streams HBM
with 256-thread CTAs; above 96 registers per thread fewer of them fit on an
SM and it loses bandwidth (an earlier change that raised it to 244 registers
cost a third of its throughput).  The tensor-core block kernel runs one
480-thread CTA per SM at 128 registers per thread, where a change in how the
compiler overlaps its epilogue once left it spilling about 440 bytes per
thread."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_cs_0404008_gb300", "csrc")


def ptxas_info(src: str) -> tuple:
    """(registers, spill-store bytes) per kernel entry of one source file."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xptxas", "-v", "-c",
                        os.path.join(CSRC, src), "-o", os.devnull],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    regs, spills, current = {}, {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            current = m.group(1)
        m = re.search(r"Used (\d+) registers", line)
        if m and current:
            regs[current] = int(m.group(1))
        m = re.search(r"(\d+) bytes spill stores", line)
        if m and current:
            spills[current] = int(m.group(1))
    return regs, spills


def ptxas_registers(src: str) -> dict:
    return ptxas_info(src)[0]


def test_dot_kernels_register_budget():
    regs = ptxas_registers("gfp_dot.cu")
    batched = [v for k, v in regs.items() if "k_dot_batched" in k]
    assert batched and max(batched) <= 96, regs
    single_blocked = [v for k, v in regs.items() if "k_dot_single" in k and "AccBlock" in k]
    assert single_blocked and max(single_blocked) <= 96, regs


def test_block_kernel_fits_one_cta_per_sm():
    regs, spills = ptxas_info("gfp_block.cu")
    tc = [v for k, v in regs.items() if "k_block_tc" in k]
    assert tc and max(tc) * 480 <= 65536, regs
    tc_spills = [v for k, v in spills.items() if "k_block_tc" in k]
    assert tc_spills and max(tc_spills) <= 64, spills
