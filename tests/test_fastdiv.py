"""The invariant-divisor division used for site coordinates (fastdiv.h), checked on the host
against plain integer division: every divisor up to 5000 and the lattice edges up to 2^16,
numerators at the edges of every quotient step and across the 32-bit range."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <cstdio>
#include <cstdint>
#include "fastdiv.h"
using namespace lbmd;
static uint64_t st = 88172645463325252ull;
static uint32_t rnd() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return (uint32_t)st; }
int main() {
  long bad = 0, n_checked = 0;
  auto check = [&](uint32_t n, uint32_t d, const FastDiv &f) {
    ++n_checked;
    if (fast_div(n, f) != n / d) { if (bad < 5) std::printf("bad %u / %u\n", n, d); ++bad; }
  };
  for (uint32_t d = 1; d <= 70000; d = d < 5000 ? d + 1 : d + 97) {
    const FastDiv f = make_fastdiv(d);
    const uint32_t edges[] = {0u, 1u, d - 1, d, d + 1, 2 * d - 1, 2 * d, 0xffffffffu, 0xfffffffeu, 0x80000000u,
                              0x7fffffffu, (0xffffffffu / d) * d, (0xffffffffu / d) * d - 1};
    for (uint32_t n : edges) check(n, d, f);
    for (int k = 0; k < 2000; ++k) check(rnd(), d, f);
    for (uint32_t q = 0; q < 300; ++q) { check(q * d, d, f); if (q) check(q * d - 1, d, f); }
  }
  std::printf("%ld %ld\n", n_checked, bad);
  return bad != 0;
}
"""


def test_fast_division_is_exact(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "fd.cpp"
    src.write_text(SRC)
    exe = tmp_path / "fd"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1306_0788_gb300", "csrc"), str(src),
                    "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
    checked, bad = map(int, r.stdout.split()[-2:])
    assert bad == 0 and checked > 10_000_000
