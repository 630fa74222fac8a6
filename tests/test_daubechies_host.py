"""The CUDA path's host-side Daubechies factorisation (compiled here with the host C++ compiler)
against the SARA oracle's filters: the same definition reached by two implementations."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import sara as osa

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER_DIR = os.path.join(os.path.dirname(HERE), "paper_2207_11336_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include "daubechies.h"
int main() {
  for (int N = 1; N <= 8; ++N) {
    const std::vector<double> h = pnp::daub::daubechies(N);
    std::printf("%d", (int)h.size());
    for (double v : h) std::printf(" %.17g", v);
    std::printf("\n");
  }
  return 0;
}
"""


def test_host_daubechies_filters_match_the_oracle(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "daub.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "daub"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.strip().splitlines()
    assert len(out) == 8
    for N, line in enumerate(out, start=1):
        vals = line.split()
        h = np.array([float(v) for v in vals[1:]])
        assert int(vals[0]) == 2 * N == h.size
        assert np.allclose(h, osa.daubechies(N), rtol=0, atol=1e-12), N
