"""Host-side check of the CUDA path's full-weighting restriction (fw3 in
csrc/common.cuh, a __host__ __device__ function that the restriction kernel,
the persistent solve kernel and the fused coarse levels all use): a small
host program built with nvcc from that header restricts fixed fine fields
separably (x per fine row, y per fine plane, z, then 1/64), which must equal
the oracle's full weighting (the 27 weights (1, 2, 1)^3 / 64 summed
directly, Sec. 1.2) up to rounding, on grids of 3, 7, 15 and 31 points per
axis.  It also checks the plane-sum sharing of the z-marching kernel: the
restriction computed with each fine plane's sum formed once and reused by
both coarse planes that share it is bitwise the per-point one.  No GPU is
used: no kernel is launched."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include "paper_1307_7867_gb300/csrc/common.cuh"
#include <cstdio>
#include <cstring>
#include <vector>
using h3d::fw3;
// fine field (dense N^3, x fastest) from stdin; per-point restriction and the
// z-marching one (shared plane sums) to stdout, with a flag for bitwise equality
int main() {
  int N = 0;
  if (std::fread(&N, sizeof(int), 1, stdin) != 1) return 1;
  const int Nc = (N - 1) / 2;
  std::vector<double> t((size_t)N * N * N);
  if (std::fread(t.data(), sizeof(double), t.size(), stdin) != t.size()) return 2;
  auto at = [&](int i, int j, int k) { return t[((size_t)k * N + j) * N + i]; };
  auto plane_sum = [&](int I, int J, int p) {
    double x[3];
    for (int cy = 0; cy < 3; ++cy)
      x[cy] = fw3(at(2 * I, 2 * J + cy, p), at(2 * I + 1, 2 * J + cy, p), at(2 * I + 2, 2 * J + cy, p));
    return fw3(x[0], x[1], x[2]);
  };
  const double sc = 1.0 * 0.015625;
  std::vector<double> a((size_t)Nc * Nc * Nc), b(a.size());
  for (int K = 0; K < Nc; ++K)
    for (int J = 0; J < Nc; ++J)
      for (int I = 0; I < Nc; ++I) {
        double y[3];
        for (int cz = 0; cz < 3; ++cz) y[cz] = plane_sum(I, J, 2 * K + cz);
        a[((size_t)K * Nc + J) * Nc + I] = fw3(y[0], y[1], y[2]) * sc;
      }
  for (int J = 0; J < Nc; ++J)
    for (int I = 0; I < Nc; ++I) {
      double ylo = plane_sum(I, J, 0);
      for (int K = 0; K < Nc; ++K) {
        const double y1 = plane_sum(I, J, 2 * K + 1), y2 = plane_sum(I, J, 2 * K + 2);
        b[((size_t)K * Nc + J) * Nc + I] = fw3(ylo, y1, y2) * sc;
        ylo = y2;
      }
    }
  const int same = std::memcmp(a.data(), b.data(), a.size() * sizeof(double)) == 0;
  std::fwrite(&same, sizeof(int), 1, stdout);
  std::fwrite(a.data(), sizeof(double), a.size(), stdout);
  return 0;
}
'''


def nvcc():
    return shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)


def test_separable_full_weighting_equals_the_oracle(oracle, tmp_path):
    cc = nvcc()
    if cc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "fw.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "fw"
    subprocess.run([cc, "-std=c++17", f"-I{ROOT}", f"-I{os.path.join(ROOT, 'include')}",
                    "-o", str(exe), str(src)], check=True, capture_output=True)
    rng = np.random.default_rng(1307)
    for N in (3, 7, 15, 31):
        t = rng.standard_normal((N, N, N))
        inp = np.int32(N).tobytes() + np.ascontiguousarray(t).tobytes()
        out = subprocess.run([str(exe)], input=inp, check=True, capture_output=True).stdout
        same = int(np.frombuffer(out[:4], dtype=np.int32)[0])
        nc = (N - 1) // 2
        got = np.frombuffer(out[4:], dtype=np.float64).reshape(nc, nc, nc)
        ref = oracle.restrict_fw(t)
        assert same == 1, N
        assert np.abs(got - ref).max() <= 4e-16 * np.abs(t).max(), N
