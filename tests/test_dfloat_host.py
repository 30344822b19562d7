"""Host check of the FP64 -> double-FP32 split used by the double-FP32
operator kernel (dfloat.cuh compiles for the host too).

The split must represent every FP64 value in the FP32 normal range to
2^-47 of its magnitude, with the low word below 2^-23 of the high word, and
map magnitudes below 2^-126 to zero.  Checked on 4 million values drawn over
the exponent range with g++ (no GPU).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2201_12931_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cstdio>
#include <cmath>
#include <cstring>
#include <random>
#include "dfloat.cuh"
using namespace topo;
int main() {
    std::mt19937_64 g(1);
    double worst = 0; long bad = 0;
    for (int i = 0; i < 4000000; ++i) {
        uint64_t b = g();
        double x;
        switch (i % 4) {
            case 0: x = std::ldexp((double)(b >> 11), -53) * std::ldexp(1.0, (int)(g() % 260) - 130); break;
            case 1: std::memcpy(&x, &b, 8); break;
            case 2: x = -std::ldexp((double)(b >> 11), -53) * std::ldexp(1.0, (int)(g() % 60) - 30); break;
            default: x = (double)(int64_t)(b >> 20) * 1e-7;
        }
        if (!std::isfinite(x)) continue;
        const dfl d = df_from_double(x);
        const long double err = fabsl((long double)d.h + (long double)d.l - (long double)x);
        const double ax = std::fabs(x);
        if (ax >= std::ldexp(1.0, -103) && ax < std::ldexp(1.0, 127)) {
            const double rel = (double)(err / ax);
            if (rel > worst) worst = rel;
            if (rel > std::ldexp(1.0, -47)) ++bad;
            if (std::fabs(d.l) > std::fabs(d.h) * std::ldexp(1.0, -23)) ++bad;
        } else if (ax < std::ldexp(1.0, -126)) {
            if (d.h != 0.f || d.l != 0.f) ++bad;
        }
    }
    std::printf("%.6e %ld\n", worst, bad);
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC), reason="needs g++ and CUDA headers")
def test_split_error_bound(tmp_path):
    src = tmp_path / "h.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "h"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CUDA_INC, "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    worst, bad = float(out[0]), int(out[1])
    assert bad == 0
    assert worst <= 2.0 ** -47
