"""Host check of the division magic the kernels use for site indices
(kernels.h: DivMagic / div_magic, Granlund and Montgomery 1994): a small C++
harness built against the library's own header computes the magic for many
divisors and checks n / d = (t + ((n - t) >> sh1)) >> sh2, t = mulhi(m, n),
for every n the kernels can pass (n < 2^31): small and large divisors,
powers of two and their neighbours, and the edges 0, d - 1, d, d + 1 and
2^31 - 1.  No GPU needed (the header's device helpers are not compiled)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1808_02281_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include "kernels.h"

static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint32_t next_u32() {            // xorshift64*: test inputs only
    state ^= state >> 12; state ^= state << 25; state ^= state >> 27;
    return (uint32_t)((state * 0x2545f4914f6cdd1dull) >> 32);
}

int main() {
    std::vector<uint32_t> ds;
    for (uint32_t d = 1; d <= 5000; ++d) ds.push_back(d);
    for (int k = 1; k < 31; ++k) {
        ds.push_back(1u << k);
        ds.push_back((1u << k) - 1);
        ds.push_back((1u << k) + 1);
    }
    for (int i = 0; i < 3000; ++i) ds.push_back(1 + next_u32() % 0x7fffffffu);
    long bad = 0, checked = 0;
    for (uint32_t d : ds) {
        const lqcd::DivMagic g = lqcd::div_magic(d);
        std::vector<uint32_t> ns = {0u, d - 1, d, d + 1, 0x7fffffffu, 0x7ffffffeu};
        for (int i = 0; i < 200; ++i) ns.push_back(next_u32() & 0x7fffffffu);
        for (uint32_t n : ns) {
            if (n > 0x7fffffffu) continue;
            const uint32_t t = (uint32_t)(((uint64_t)g.m * n) >> 32);
            const uint32_t q = (t + ((n - t) >> g.sh1)) >> g.sh2;
            ++checked;
            if (q != n / d) {
                if (bad < 5) std::printf("d=%u n=%u got %u want %u\n", d, n, q, n / d);
                ++bad;
            }
        }
    }
    std::printf("checked %ld bad %ld\n", checked, bad);
    return bad != 0;
}
"""


def _cuda_include():
    for root in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if root and os.path.isfile(os.path.join(root, "include", "cuda_runtime.h")):
            return os.path.join(root, "include")
    return None


def test_division_magic_is_exact_below_2_31(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    src = tmp_path / "div_magic_check.cpp"
    exe = tmp_path / "div_magic_check"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "bad 0" in out.stdout
