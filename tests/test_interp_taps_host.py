"""Host-side check of the CUDA path's 6- and 8-point interpolation taps
(mid_taps in csrc/mg_kernels.cu, a __host__ __device__ function): a small
host program built with nvcc from that source prints the one-axis
interpolation of fixed coarse lines, which must equal the oracle's rule
(weights from the Lagrange product formula, odd extension about both ends),
on coarse lines of 1, 3, 7 and 15 points, where the 8-point stencil wraps
around the boundaries.  No GPU is used: no kernel is launched."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include "paper_1307_7867_gb300/csrc/mg_kernels.cu"
namespace h3d { void count_launch() {} }
#include <cstdio>
#include <cmath>
template <int NT> void run(int Nc) {
  double e[64];
  for (int a = 0; a < Nc; ++a) e[a] = std::sin(1.3 * (a + 1) + 0.7) + 0.1 * a;
  for (int f = 0; f < 2 * Nc + 1; ++f) {
    int ix[NT];
    double w[NT];
    h3d::mid_taps<NT>(f, Nc, ix, w);
    double s = 0.0;
    for (int q = 0; q < NT; ++q) {
      if (ix[q] < 0 || ix[q] >= Nc) { std::printf("BAD %d %d %d\n", NT, Nc, f); return; }
      s += w[q] * e[ix[q]];
    }
    std::printf("%d %d %d %.17g\n", NT, Nc, f, s);
  }
}
int main() {
  for (int Nc : {1, 3, 7, 15}) { run<6>(Nc); run<8>(Nc); }
  return 0;
}
'''


def nvcc():
    return shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)


def test_cuda_midpoint_taps_equal_the_oracle_rule(oracle, tmp_path):
    cc = nvcc()
    if cc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "taps.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "taps"
    subprocess.run([cc, "-std=c++17", f"-I{ROOT}", f"-I{os.path.join(ROOT, 'include')}",
                    "-gencode", "arch=compute_103a,code=sm_103a", "-o", str(exe), str(src)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [line.split() for line in out if line.strip()]
    assert not any(r[0] == "BAD" for r in rows)
    for npts in (6, 8):
        for nc in (1, 3, 7, 15):
            nf = 2 * nc + 1
            got = np.array([float(r[3]) for r in rows if int(r[0]) == npts and int(r[1]) == nc])
            assert got.size == nf
            a = np.arange(nc)
            line = np.sin(1.3 * (a + 1) + 0.7) + 0.1 * a
            # a separable coarse field whose y and z factors are one unit point:
            # the fine row through that point is the one-axis interpolation
            unit = np.zeros(nc)
            unit[nc // 2] = 1.0
            e3 = line[None, None, :] * unit[None, :, None] * unit[:, None, None]
            ref3 = oracle.prolong_add_lagrange(e3, np.zeros((nf, nf, nf)), npts)
            j = 2 * (nc // 2) + 1
            assert np.abs(got - ref3[j, j, :]).max() <= 1e-15, (npts, nc)
