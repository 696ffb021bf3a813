"""Host-side check of the CUDA path's damped-Jacobi and residual formulas on
the scaled right-hand side (jacobi_point and resid_point in
csrc/stencil_impl.cuh, with the level coefficients of mg_level_coef in
csrc/common.cuh; both __host__ __device__): every multigrid level stores
b' = wd b, a sweep is v = (1 - omega) u + wd e S + b' and the restricted
residual is t' = b' - omega u + wd e S.  A small host program built with
nvcc from those headers applies them to fixed fields with the stencils'
boundary rule; v must equal the oracle's damped-Jacobi sweep u + omega r / d
and t' / wd the oracle's residual b - A u (Sec. 1.2), up to rounding, for
the 7-point and the wide stencil on 7^3 and 15^3 grids.  No GPU is used: no
kernel is launched."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include "paper_1307_7867_gb300/csrc/stencil_impl.cuh"
#include <cstdio>
#include <vector>
namespace h3d { void count_launch() {} }
using namespace h3d;
// stdin: N, order, c, u (N^3), b (N^3); stdout: v (N^3), t'/wd (N^3)
int main() {
  int N = 0, order = 0;
  double c = 0;
  if (std::fread(&N, sizeof(int), 1, stdin) != 1 || std::fread(&order, sizeof(int), 1, stdin) != 1 ||
      std::fread(&c, sizeof(double), 1, stdin) != 1)
    return 1;
  const size_t n = (size_t)N * N * N;
  std::vector<double> u(n), b(n), v(n), r(n);
  if (std::fread(u.data(), sizeof(double), n, stdin) != n) return 2;
  if (std::fread(b.data(), sizeof(double), n, stdin) != n) return 3;
  const Coef<double> q = mg_level_coef(order, c, 1.0 / (N + 1), 0.0);
  // boundary rule of the stencil kernels: indices -1 and N read 0, the wide
  // stencil's -2 and N+1 read minus the value at 0 and N-1
  auto at = [&](int i, int j, int k) {
    double s = 1.0;
    int* ix[3] = {&i, &j, &k};
    for (int a = 0; a < 3; ++a) {
      int& p = *ix[a];
      if (p == -1 || p == N) return 0.0;
      if (p == -2) { p = 0; s = -s; }
      if (p == N + 1) { p = N - 1; s = -s; }
    }
    return s * u[((size_t)k * N + j) * N + i];
  };
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        const size_t p = ((size_t)k * N + j) * N + i;
        const double s1 = ((at(i - 1, j, k) + at(i + 1, j, k)) + (at(i, j - 1, k) + at(i, j + 1, k))) +
                          (at(i, j, k - 1) + at(i, j, k + 1));
        const double s2 = order == 4 ? ((at(i - 2, j, k) + at(i + 2, j, k)) +
                                        (at(i, j - 2, k) + at(i, j + 2, k))) +
                                           (at(i, j, k - 2) + at(i, j, k + 2))
                                     : 0.0;
        const double bp = q.wd * b[p];
        if (order == 4) {
          v[p] = jacobi_point<double, 4>(q.al, q.be, q.be2, u[p], s1, s2, bp);
          r[p] = resid_point<double, 4>(q.om, q.be, q.be2, u[p], s1, s2, bp) / q.wd;
        } else {
          v[p] = jacobi_point<double, 2>(q.al, q.be, q.be2, u[p], s1, s2, bp);
          r[p] = resid_point<double, 2>(q.om, q.be, q.be2, u[p], s1, s2, bp) / q.wd;
        }
      }
  std::fwrite(v.data(), sizeof(double), n, stdout);
  std::fwrite(r.data(), sizeof(double), n, stdout);
  return 0;
}
'''


def nvcc():
    return shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc"
                                    if os.path.exists("/usr/local/cuda/bin/nvcc") else None)


def test_scaled_jacobi_and_residual_equal_the_oracle(oracle, tmp_path):
    cc = nvcc()
    if cc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "sj.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "sj"
    subprocess.run([cc, "-std=c++17", f"-I{ROOT}", f"-I{os.path.join(ROOT, 'include')}",
                    "-gencode", "arch=compute_103a,code=sm_103a", "-o", str(exe), str(src)],
                   check=True, capture_output=True)
    rng = np.random.default_rng(7867)
    for N in (7, 15):
        for order in (2, 4):
            for c in (0.0005, 0.02):
                u = rng.standard_normal((N, N, N))
                b = rng.standard_normal((N, N, N))
                inp = (np.int32(N).tobytes() + np.int32(order).tobytes() + np.float64(c).tobytes()
                       + u.tobytes() + b.tobytes())
                out = subprocess.run([str(exe)], input=inp, check=True,
                                     capture_output=True).stdout
                got = np.frombuffer(out, dtype=np.float64).reshape(2, N, N, N)
                v_ref = oracle.jacobi(u, b, order, c)
                r_ref = oracle.residual(u, b, order, c)
                scale_v = np.abs(v_ref).max() + np.abs(u).max()
                scale_r = np.abs(r_ref).max() + np.abs(oracle.apply_A(u, order, c)).max()
                assert np.abs(got[0] - v_ref).max() <= 1e-14 * scale_v, (N, order, c)
                assert np.abs(got[1] - r_ref).max() <= 1e-14 * scale_r, (N, order, c)
                # a wrong coefficient or sign moves the sweep far more than rounding
                assert np.abs(got[0] - u).max() > 1e-3 * np.abs(u).max()
