"""The charges' spatial order (csrc/psum_internal.cuh, hilbert_key24): the key is a
bijection of the 256^3 cells onto 0 .. 2^24 - 1, consecutive keys are face neighbours (the
Hilbert curve), and the curve starts at cell (0, 0, 0) and ends at (255, 0, 0) -- the corners
the full-size parity samples take whole tiles from (tests/parity_check.full_size_sample).

Host only: the key function is compiled for the host by the C++ compiler against the CUDA
headers; the test is skipped where either is missing."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1310_4374_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "psum_internal.cuh"
int main() {
    const uint32_t n = 1u << 24;
    std::vector<uint32_t> cell(n, 0xffffffffu);      // key -> cell (x + 256 y + 65536 z)
    for (uint32_t z = 0; z < 256; ++z)
        for (uint32_t y = 0; y < 256; ++y)
            for (uint32_t x = 0; x < 256; ++x) {
                const uint32_t k = psum::hilbert_key24(x, y, z);
                if (k >= n || cell[k] != 0xffffffffu) { printf("not a bijection at %u %u %u\n", x, y, z); return 1; }
                cell[k] = x + 256 * y + 65536 * z;
            }
    for (uint32_t k = 1; k < n; ++k) {
        const int a = (int)cell[k - 1], b = (int)cell[k];
        const int d = std::abs(a % 256 - b % 256) + std::abs(a / 256 % 256 - b / 256 % 256) + std::abs(a / 65536 - b / 65536);
        if (d != 1) { printf("keys %u and %u are not face neighbours\n", k - 1, k); return 1; }
    }
    printf("%u %u\n", cell[0], cell[n - 1]);
    return 0;
}
"""


def _cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return os.path.join(cand, "include")
    return None


def test_hilbert_key_is_a_face_connected_bijection(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("no host C++ compiler or CUDA headers")
    src = tmp_path / "curve.cpp"
    exe = tmp_path / "curve"
    src.write_text(PROGRAM)
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", inc, "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout
    first, last = (int(v) for v in r.stdout.split())
    assert first == 0                      # cell (0, 0, 0)
    assert last == 255                     # cell (255, 0, 0)
