"""The double-float arithmetic of the refinement passes (csrc/df.cuh),
compiled for the host: conversions, sums and products of 2e6 random pairs
over twelve decades against long-double results, and the integer-field
conversions between double and float pairs against the hardware ones. The bounds are those of
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
  // the integer-field conversions against the hardware ones, over the whole
  // exponent range the solver meets and the rounding ties
  long long diff = 0, cnt = 0;
  std::uniform_int_distribution<int> X(-80, 120);
  for (int t = 0; t < 2000000; ++t) {
    double d = U(g) * std::ldexp(1.0, X(g));
    if (t % 7 == 0) d = (double)(float)d + std::ldexp((float)d, -24) * (t % 2 ? 1 : -1) * std::fabs(U(g)) ;
    if (t % 11 == 0) {  // exact ties: hi's last bit and a remainder of half an ulp
      const float h = (float)d;
      d = (double)h + std::ldexp(1.0, std::ilogb(h) - 24);
    }
    const double a = std::fabs(d);
    float hi, lo;
    heat::df_split(d, hi, lo);
    const float h2 = (float)d, l2 = (float)(d - (double)h2);
    if (a >= std::ldexp(1.0, -74)) {
      diff += (hi != h2) || (lo != l2);
    } else {
      diff += std::fabs((double)hi + (double)lo - d) > std::ldexp(1.0, -98);
    }
    const float f = (float)d;
    diff += heat::df_f2d(f) != (double)f;
    ++cnt;
  }
  const float zs[4] = {0.f, -0.f, 1.f, -3.5e-20f};
  for (float z : zs) diff += std::signbit(heat::df_f2d(z)) != std::signbit(z) || heat::df_f2d(z) != (double)z;
  std::printf("%.6e %.6e %.6e %.6e %lld %lld\n", wc, wa, wm, wz, diff, cnt);
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
    conv, add, mul, zero = (float(v) for v in out[:4])
    mismatches, count = int(out[4]), int(out[5])
    assert count == 2000000 and mismatches == 0  # field conversions equal the hardware ones
    ulp44 = 2.0 ** -44
    assert conv <= 2.0 ** -47  # hi + lo carries 48 bits of a double
    assert add <= ulp44 and mul <= 2 * ulp44
    assert zero == 0.0  # a - a is exactly zero
