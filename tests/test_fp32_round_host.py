"""Host-side pins of the FP32 rounding of unitary gate matrices
(csrc/fp32_round.h): on random unitaries the chosen FP32 matrix is never
farther from unitary than the entry-by-entry rounding, and every entry stays
within about one and a half units in the last place of the exact value."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cstdio>
#include <random>
#include <complex>
#include "fp32_round.h"
using namespace nqs;
int main() {
    std::mt19937_64 g(7);
    std::normal_distribution<double> nd;
    double worse = 0, maxdist = 0, sum_naive = 0, sum_chosen = 0, unit_mod = 0;
    int better = 0, total = 0;
    for (int dim : {2, 4})
        for (int t = 0; t < 200; ++t) {
            std::complex<double> a[16], q[16];
            for (int e = 0; e < dim * dim; ++e) a[e] = {nd(g), nd(g)};
            for (int c = 0; c < dim; ++c) {   // Gram-Schmidt on the columns
                for (int r = 0; r < dim; ++r) q[r * dim + c] = a[r * dim + c];
                for (int p = 0; p < c; ++p) {
                    std::complex<double> d = 0;
                    for (int r = 0; r < dim; ++r) d += std::conj(q[r * dim + p]) * q[r * dim + c];
                    for (int r = 0; r < dim; ++r) q[r * dim + c] -= d * q[r * dim + p];
                }
                double nn = 0;
                for (int r = 0; r < dim; ++r) nn += std::norm(q[r * dim + c]);
                for (int r = 0; r < dim; ++r) q[r * dim + c] /= std::sqrt(nn);
            }
            float2 out[16];
            float naive[32], chosen[32];
            round_matrix_c64(q, dim, out);
            for (int e = 0; e < dim * dim; ++e) {
                naive[2 * e] = (float)q[e].real();
                naive[2 * e + 1] = (float)q[e].imag();
                chosen[2 * e] = out[e].x;
                chosen[2 * e + 1] = out[e].y;
                maxdist = std::max(maxdist, std::abs(std::complex<double>(out[e].x, out[e].y) - q[e]));
            }
            const double dn = fp32r::unitarity_defect(naive, dim), dc = fp32r::unitarity_defect(chosen, dim);
            sum_naive += dn;
            sum_chosen += dc;
            ++total;
            better += dc <= dn;
            worse = std::max(worse, dc - dn);
        }
    for (int t = 0; t < 1000; ++t) {   // phases e^{i theta}: modulus as close to 1 as FP32 allows
        const double th = 6.283185307179586 * (t + 0.5) / 1000.0;
        const float2 f = round_c64(std::polar(1.0, th));
        unit_mod = std::max(unit_mod, std::abs((double)f.x * f.x + (double)f.y * f.y - 1.0));
    }
    printf("%d %d %.17g %.17g %.17g %.17g %.17g\n", total, better, worse, maxdist, sum_naive, sum_chosen, unit_mod);
}
'''


def test_unitary_rounding(tmp_path):
    cxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(inc):
        pytest.skip("no host C++ compiler or CUDA headers")
    src = tmp_path / "fr.cpp"
    src.write_text(SRC)
    exe = tmp_path / "fr"
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2211_17028_gb300", "csrc"), "-I", inc,
                    str(src), "-o", str(exe)], check=True)
    total, better, worse, maxdist, sum_naive, sum_chosen, unit_mod = subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(better) == int(total) == 400 and float(worse) <= 0.0
    assert float(maxdist) <= 1.2e-7                      # about one and a half ulps of entries below 1
    assert float(sum_chosen) < 0.5 * float(sum_naive)    # the coherent part of the rounding is gone
    assert float(unit_mod) <= 1.2e-7                     # |e^{i theta}|^2 - 1 within one ulp of 1
