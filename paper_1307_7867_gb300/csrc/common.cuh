// common.cuh -- shared types of the heat3d CUDA library (sm_103a).
//
// Field layout in device memory: for a grid with N interior points per axis a
// field is px * N * N elements, x fastest, with the x pitch px = N rounded up
// to 4 (the 2^k - 1 grids of the hierarchy get px = 2^k, so every row starts
// 128-byte aligned once px * sizeof(T) >= 128).  The pad columns stay zero
// and are never read as data.  Items of a batch (PFASST slices, serving
// requests, nodes) follow each other at the field stride fs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace h3d {

constexpr int kMaxNodes = 5;
constexpr int kMaxLevels = 12;  // multigrid levels: N up to 2^12 - 1

struct Grid {
  int N;            // interior points per axis
  int px;           // x pitch in elements
  long long plane;  // px * N
  long long fs;     // field stride (elements) between consecutive items
};

inline Grid make_grid(int N) {
  Grid g;
  g.N = N;
  g.px = (N + 3) / 4 * 4;
  g.plane = (long long)g.px * N;
  long long f = g.plane * N;
  g.fs = (f + 63) / 64 * 64;  // keeps every field 256-byte aligned for 4- and 8-byte types
  return g;
}

// Coefficients of A = W - c Delta_h on one multigrid level for one item:
//   A u = d u - e S, with S = sum of the 6 nearest neighbours (7 points) or
//   16 * (6 nearest) - (6 second neighbours) (wide stencil), W = I;
//   compact stencil: A u = d u - e S1 - e2 S2 with S1 the 6 face and S2 the
//   12 edge neighbours (W - c L of the Mehrstellen scheme);
//   wd = omega / d for damped Jacobi; a11 = A on the one-unknown grid.
// The V-cycle keeps every level's right-hand side scaled, b' = wd b (it is
// also the first Jacobi iterate from zero), so that a sweep is
//   v = al u + be S + b'          (al = 1 - omega, be = wd e; compact: + be2 S2)
// and the residual it restricts is t' = wd (b - A u) = b' - om u + be S
// (om = omega); the restriction into level k multiplies by rs = wd_k / wd_{k-1},
// and the one-unknown grid solves e = b' / a11w (a11w = wd a11).
template <typename T>
struct Coef {
  T d, e, wd, a11, e2;
  T al, om, be, be2, rs, a11w;
};

// Order code of the compact 19-point (Mehrstellen) stencil.
constexpr int kCompact = 19;

// Coefficients of A = W - c Delta_h on a multigrid level of spacing h for
// stencil `order` (Sec. 1.2; see Coef), with the damped-Jacobi weights of
// the scaled V-cycle; wd_finer: wd of the next finer level (0 on the finest,
// rs = 1 there).
inline Coef<double> mg_level_coef(int order, double c, double h, double wd_finer) {
  Coef<double> q;
  double omega;
  q.e2 = 0.0;
  if (order == kCompact) {
    // W - c L: centre 1/2 + 4c/h^2, faces 1/12 - c/(3h^2), edges -c/(6h^2);
    // omega = 12/11 from local Fourier analysis of the Mehrstellen operator
    q.e = c / (3.0 * h * h) - 1.0 / 12.0;
    q.e2 = c / (6.0 * h * h);
    q.d = 0.5 + 4.0 * c / (h * h);
    omega = 12.0 / 11.0;
    q.a11 = q.d;
  } else if (order == 2) {
    q.e = c / (h * h);
    q.d = 1.0 + 6.0 * q.e;
    omega = 6.0 / 7.0;
    q.a11 = 1.0 + 6.0 * q.e;
  } else {
    q.e = c / (12.0 * h * h);
    q.d = 1.0 + 90.0 * q.e;
    omega = 9.0 / 11.0;
    q.a11 = 1.0 + 84.0 * q.e;
  }
  q.wd = omega / q.d;
  q.al = 1.0 - omega;
  q.om = omega;
  q.be = q.wd * q.e;
  q.be2 = q.wd * q.e2;
  q.a11w = q.wd * q.a11;
  q.rs = wd_finer > 0.0 ? q.wd / wd_finer : 1.0;
  return q;
}

// Full weighting (Sec. 1.2) of a fine field onto coarse point (I, J, K), the
// fine points 2I..2I+2, 2J..2J+2, 2K..2K+2 (0-based) with weights (1, 2, 1)
// per axis, formed separably -- along x per fine row, then y per fine plane,
// then z -- and scaled by 1/64 at the end:
//   X = fw3(t(2I), t(2I+1), t(2I+2)), Y = fw3(X(2J), X(2J+1), X(2J+2)),
//   value = fw3(Y(2K), Y(2K+1), Y(2K+2)) * (rs / 64).
// Every implementation (the z-marching restriction kernel, which reuses the
// plane sums Y of the fine planes two coarse planes share, the persistent
// solve kernel, the fused coarse levels) uses exactly these operations, so
// they agree bit for bit.
template <typename T>
__host__ __device__ __forceinline__ T fw3(T a, T b, T c) {
  return fma(T(2), b, a + c);
}

// Per item, per SDC level: step data of the sweep (Sec. 1.1).
struct ItemSDC {
  double dtS[kMaxNodes - 1][kMaxNodes];  // dt * S[m][j]
  double gS[kMaxNodes - 1];              // dt * sum_j S[m][j] g(t0 + dt tau_j): forcing integral
  double dtm[kMaxNodes - 1];             // dt * (tau_{m+1} - tau_m)
  double dtQ[kMaxNodes][kMaxNodes];      // dt * Q[m][j]  (FAS restriction, fine level)
  double gQ[kMaxNodes];                  // dt * sum_j Q[m][j] g(t0 + dt tau_j)
  double nu;
};

// FAS transfer data between the fine (F) and coarse (G) levels.
struct FasMap {
  int jm[kMaxNodes];                      // fine node of coarse node m
  double L[kMaxNodes][kMaxNodes];         // L[j][m] = l^G_m(tau^F_j): Lagrange in time
};

}  // namespace h3d
