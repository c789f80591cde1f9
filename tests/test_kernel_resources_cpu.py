"""Resource budgets of the fused-step kernels, checked at compile time on the
CPU (nvcc cross-compiles for sm_103a; nothing runs on a GPU).

The step's speed rests on how many thread blocks an SM holds and on the
kernels not spilling registers:
- the FP32 strip (288 threads) is launched for 2 blocks per SM, so its shared
  memory must leave room for two;
- the FP32 32x8 tile (256 threads) for 3 blocks per SM;
- the FP64 strip and tile for 1.
A GB300 SM has 228 KB of shared memory, up to 227 KB per block, and reserves
1 KB per resident block.  The FP32 strip must also compile without spilling,
and the FP32 diagnostics kernel within 64 registers.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1802_02868_gb300", "csrc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
SM_SMEM = 228 * 1024
BLOCK_RESERVED = 1024


def _nvcc():
    p = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if p is None:
        pytest.skip("nvcc not available")
    return p


def _fits(nbytes, blocks):
    return blocks * (nbytes + BLOCK_RESERVED) <= SM_SMEM and nbytes <= 227 * 1024


def test_shared_memory_of_each_shape_fits_its_blocks_per_sm(tmp_path):
    src = tmp_path / "sizes.cu"
    src.write_text(
        '#include "%s"\n'
        "#include <cstdio>\n"
        "int main() {\n"
        '  printf("%%zu %%zu %%zu %%zu\\n", dugks::StripLayout<float, 32, 8>::bytes,\n'
        "         dugks::StripLayout<double, 32, 8>::bytes, dugks::FusedLayout<float, 32, 8, false>::bytes,\n"
        "         dugks::FusedLayout<double, 32, 8, false>::bytes);\n"
        "}\n" % os.path.join(CSRC, "dugks_strip.cuh"))
    exe = tmp_path / "sizes"
    r = subprocess.run([_nvcc(), str(src), "-o", str(exe)] + ARCH + FLAGS, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    strip32, strip64, tile32, tile64 = (int(v) for v in subprocess.run([str(exe)], capture_output=True,
                                                                          text=True).stdout.split())
    assert _fits(strip32, 2), strip32
    assert _fits(tile32, 3), tile32
    assert _fits(strip64, 1) and _fits(tile64, 1), (strip64, tile64)


def test_fp32_strips_and_diagnostics_compile_within_budget(tmp_path):
    """The FP32 strips spill nothing; the FP32 diagnostics kernel fits 64
    registers without spills, which holds four of its 256-thread blocks per
    SM (its speed rests on that occupancy)."""
    out = tmp_path / "api.o"
    r = subprocess.run([_nvcc(), "-c", os.path.join(CSRC, "dugks_api.cu"), "-o", str(out), "-O3", "-Xptxas", "-v",
                        "-Xcompiler", "-fPIC"] + ARCH + FLAGS, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lines = r.stderr.splitlines()
    found = {"k_strip": 0}
    for i, line in enumerate(lines):
        m = re.search(r"Compiling entry function '(\S+)'", line)
        # mangled k_strip<float, 32, 8, 288, ...>
        for name in found:
            if m and (name + "IfLi32ELi8ELi288E") in m.group(1):
                found[name] += 1
                props = " ".join(lines[i + 1:i + 4])
                spill = re.search(r"(\d+) bytes spill stores", props)
                assert spill is not None and int(spill.group(1)) == 0, (m.group(1), props)
    assert found == {"k_strip": 2}, "expected the general and the uniform FP32 strip: %s" % found
    diag = [i for i, line in enumerate(lines) if re.search(r"Compiling entry function '\S*k_diag_fIfE", line)]
    assert len(diag) == 1, diag
    props = " ".join(lines[diag[0] + 1:diag[0] + 4])
    spill = re.search(r"(\d+) bytes spill stores", props)
    regs = re.search(r"Used (\d+) registers", props)
    assert spill is not None and int(spill.group(1)) == 0, props
    assert regs is not None and int(regs.group(1)) <= 64, props
