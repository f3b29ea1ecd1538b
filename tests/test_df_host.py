"""The double-float arithmetic of the refinement passes (csrc/df.cuh),
compiled for the host: conversions, sums and products of 2e6 random pairs
over twelve decades against long-double results. The bounds are those of
the method (Knuth two-sum, FMA two-product): about 2^-44 relative to the
operands for a sum and to the result for a product."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), os.pardir, "paper_1905_07622_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cmath>
#include <random>
#include "df.cuh"
using heat::DF;
int main() {
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double wc = 0, wa = 0, wm = 0, wz = 0;
  for (int t = 0; t < 2000000; ++t) {
    const double a = U(g) * std::pow(10.0, (int)(U(g) * 6)), b = U(g) * std::pow(10.0, (int)(U(g) * 6));
    const DF A(a), B(b);
    wc = std::fmax(wc, std::fabs(A.to_double() - a) / std::fabs(a));
    const long double ea = A.to_double(), eb = B.to_double();
    wa = std::fmax(wa, (double)(std::fabs((long double)(A + B).to_double() - (ea + eb)) / (std::fabs(ea) + std::fabs(eb))));
    wm = std::fmax(wm, (double)(std::fabs((long double)(A * B).to_double() - ea * eb) / std::fabs(ea * eb)));
    wz = std::fmax(wz, std::fabs((A - A).to_double()));
  }
  std::printf("%.6e %.6e %.6e %.6e\n", wc, wa, wm, wz);
  return 0;
}
"""


def test_double_float_error_bounds(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "df_host.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "df_host"
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.abspath(CSRC), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    conv, add, mul, zero = (float(v) for v in out)
    ulp44 = 2.0 ** -44
    assert conv <= 2.0 ** -47  # hi + lo carries 48 bits of a double
    assert add <= ulp44 and mul <= 2 * ulp44
    assert zero == 0.0  # a - a is exactly zero
