// coarse_fused.cuh -- the bottom of a V-cycle (Sec. 1.2: coarsening down to
// one unknown) as a block-level device routine, shared by the fused coarse
// kernel (coarse_fused.cu) and the persistent solve kernel (persist.cu).
//
// One block runs the whole sub-cycle of one item from a level with N <= 15
// down to the one-unknown grid and back, with every level's right-hand side,
// correction and ping-pong field in shared memory (dense N^3 layout), and
// writes the correction of its top level to global memory.  Each operation
// repeats the arithmetic of the separate kernels in the same order (neighbour
// sums, fused multiply-adds, restriction and prolongation summation order), so
// the result is bitwise the same as the launch sequence.
#pragma once
#include "kernels.cuh"

namespace h3d {

// Shared memory of vcycle_small_body for the levels Ns[0..nlev) (bytes).
size_t vcycle_small_smem(int nlev, const int* Ns, size_t tsize);

namespace {

template <typename T>
__device__ __forceinline__ T sval(const T* f, int N, int i, int j, int k) {
  bool neg = false;
  if (i < 0 || i >= N) {
    if (i == -1 || i == N) return T(0);
    neg = !neg;
    i = i < 0 ? 0 : N - 1;
  }
  if (j < 0 || j >= N) {
    if (j == -1 || j == N) return T(0);
    neg = !neg;
    j = j < 0 ? 0 : N - 1;
  }
  if (k < 0 || k >= N) {
    if (k == -1 || k == N) return T(0);
    neg = !neg;
    k = k < 0 ? 0 : N - 1;
  }
  T v = f[(k * N + j) * N + i];
  return neg ? -v : v;
}

// Neighbour sums in the order of the stencil kernels: ((x) + (y)) + (z).
template <typename T, int ORDER>
__device__ __forceinline__ void nsums(const T* f, int N, int i, int j, int k, T& s1, T& s2) {
  s1 = ((sval(f, N, i - 1, j, k) + sval(f, N, i + 1, j, k)) +
        (sval(f, N, i, j - 1, k) + sval(f, N, i, j + 1, k))) +
       (sval(f, N, i, j, k - 1) + sval(f, N, i, j, k + 1));
  s2 = T(0);
  if (ORDER == 4)
    s2 = ((sval(f, N, i - 2, j, k) + sval(f, N, i + 2, j, k)) +
          (sval(f, N, i, j - 2, k) + sval(f, N, i, j + 2, k))) +
         (sval(f, N, i, j, k - 2) + sval(f, N, i, j, k + 2));
}

template <typename T, int ORDER>
__device__ __forceinline__ T combine_s(T s1, T s2) {
  if (ORDER == 2) return s1;
  return fma(T(16), s1, -s2);
}

template <typename T>
struct SmallArgs {
  int nlev;                   // levels handled (top .. one unknown)
  int N[kMaxLevels];          // sizes, top first
  const Coef<T>* cf[kMaxLevels];  // per level, item 0 of the launch
  const T* b;                 // top-level right-hand side (pitched, grid gtop)
  T* e;                       // top-level correction out (pitched)
  Grid gtop;
  int nu1, nu2;
  const int* active;
};

template <typename T, int ORDER>
__device__ __forceinline__ void vcycle_small_body(const SmallArgs<T>& a, int item, T* base) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // per level: b, e, t (dense)
  T* lb[kMaxLevels];
  T* le[kMaxLevels];
  T* lt[kMaxLevels];
  {
    T* p = base;
    for (int l = 0; l < a.nlev; ++l) {
      const int n3 = a.N[l] * a.N[l] * a.N[l];
      lb[l] = p; p += n3;
      le[l] = p; p += n3;
      lt[l] = p; p += n3;
    }
  }
  // top right-hand side from global memory
  {
    const int N = a.N[0];
    const T* src = a.b + item * a.gtop.fs;
    for (int q = tid; q < N * N * N; q += nt) {
      const int i = q % N, j = (q / N) % N, k = q / (N * N);
      lb[0][q] = __ldcg(src + (long long)k * a.gtop.plane + (long long)j * a.gtop.px + i);
    }
  }
  __syncthreads();
  T* cur[kMaxLevels];
  T* oth[kMaxLevels];
  // down: pre-smoothing from the scaled right-hand side b' (the first
  // iterate, never written), residual, restriction
  for (int l = 0; l < a.nlev; ++l) {
    const int N = a.N[l];
    const Coef<T> c = a.cf[l][item];
    const int n3 = N * N * N;
    if (N == 1) {
      if (tid == 0) le[l][0] = lb[l][0] / c.a11w;
      cur[l] = le[l];
      __syncthreads();
      break;
    }
    T* cu = lb[l];
    T* ot = le[l];
    for (int s = 1; s < a.nu1; ++s) {
      for (int q = tid; q < n3; q += nt) {
        const int i = q % N, j = (q / N) % N, k = q / (N * N);
        T s1, s2;
        nsums<T, ORDER>(cu, N, i, j, k, s1, s2);
        ot[q] = fma(c.al, cu[q], fma(c.be, combine_s<T, ORDER>(s1, s2), lb[l][q]));
      }
      __syncthreads();
      if (cu == lb[l]) {
        cu = ot;
        ot = lt[l];
      } else {
        T* tmp = cu; cu = ot; ot = tmp;
      }
    }
    for (int q = tid; q < n3; q += nt) {
      const int i = q % N, j = (q / N) % N, k = q / (N * N);
      T s1, s2;
      nsums<T, ORDER>(cu, N, i, j, k, s1, s2);
      ot[q] = fma(-c.om, cu[q], fma(c.be, combine_s<T, ORDER>(s1, s2), lb[l][q]));
    }
    __syncthreads();
    // full weighting (fw3) into the next level's scaled right-hand side
    const int Nc = a.N[l + 1];
    const T sc = a.cf[l + 1][item].rs * T(0.015625);
    for (int q = tid; q < Nc * Nc * Nc; q += nt) {
      const int I = q % Nc, J = (q / Nc) % Nc, K = q / (Nc * Nc);
      T y[3];
      for (int cz = 0; cz < 3; ++cz) {
        T x[3];
        for (int cy = 0; cy < 3; ++cy) {
          const T* row = ot + ((2 * K + cz) * N + (2 * J + cy)) * N + 2 * I;
          x[cy] = fw3(row[0], row[1], row[2]);
        }
        y[cz] = fw3(x[0], x[1], x[2]);
      }
      lb[l + 1][q] = fw3(y[0], y[1], y[2]) * sc;
    }
    cur[l] = cu;
    oth[l] = ot;
    __syncthreads();
  }
  // up: prolongation (cell-based, as k_prolong_add; from b' into the free
  // buffer when no pre-smoothing sweep ran) and post-smoothing
  for (int l = a.nlev - 2; l >= 0; --l) {
    const int N = a.N[l], Nc = a.N[l + 1];
    const Coef<T> c = a.cf[l][item];
    const T* ec = cur[l + 1];
    T* cu = cur[l];
    T* ot = oth[l];
    T* dst = cu == lb[l] ? ot : cu;
    const int nc1 = Nc + 1;
    for (int q = tid; q < nc1 * nc1 * nc1; q += nt) {
      const int cx = q % nc1, cy = (q / nc1) % nc1, cz = q / (nc1 * nc1);
      T v[2][2][2];
      for (int z = 0; z < 2; ++z)
        for (int y = 0; y < 2; ++y)
          for (int x = 0; x < 2; ++x) {
            const int ii = cx - 1 + x, jj = cy - 1 + y, kk = cz - 1 + z;
            v[z][y][x] = (ii < 0 || ii >= Nc || jj < 0 || jj >= Nc || kk < 0 || kk >= Nc)
                             ? T(0) : ec[(kk * Nc + jj) * Nc + ii];
          }
      T X[2][2][2], Y[2][2][2];
      for (int z = 0; z < 2; ++z)
        for (int y = 0; y < 2; ++y) {
          X[z][y][0] = v[z][y][0] + v[z][y][1];
          X[z][y][1] = v[z][y][1];
        }
      for (int z = 0; z < 2; ++z)
        for (int mx = 0; mx < 2; ++mx) {
          Y[z][0][mx] = X[z][0][mx] + X[z][1][mx];
          Y[z][1][mx] = X[z][1][mx];
        }
      for (int mz = 0; mz < 2; ++mz) {
        const int fz = 2 * cz + mz;
        if (fz >= N) continue;
        for (int my = 0; my < 2; ++my) {
          const int fy = 2 * cy + my;
          if (fy >= N) continue;
          for (int mx = 0; mx < 2; ++mx) {
            const int fx = 2 * cx + mx;
            if (fx >= N) continue;
            T wv = mz == 0 ? Y[0][my][mx] + Y[1][my][mx] : Y[1][my][mx];
            const int na = (mx == 0) + (my == 0) + (mz == 0);
            const T val = na == 0 ? wv : wv * (na == 1 ? T(0.5) : na == 2 ? T(0.25) : T(0.125));
            const int o = (fz * N + fy) * N + fx;
            dst[o] = cu[o] + val;
          }
        }
      }
    }
    __syncthreads();
    if (cu == lb[l]) {
      cu = dst;
      ot = dst == le[l] ? lt[l] : le[l];
    }
    const int n3 = N * N * N;
    for (int s = 0; s < a.nu2; ++s) {
      for (int q = tid; q < n3; q += nt) {
        const int i = q % N, j = (q / N) % N, k = q / (N * N);
        T s1, s2;
        nsums<T, ORDER>(cu, N, i, j, k, s1, s2);
        ot[q] = fma(c.al, cu[q], fma(c.be, combine_s<T, ORDER>(s1, s2), lb[l][q]));
      }
      __syncthreads();
      T* tmp = cu; cu = ot; ot = tmp;
    }
    cur[l] = cu;
  }
  // top-level correction to global memory
  {
    const int N = a.N[0];
    T* dst = a.e + item * a.gtop.fs;
    for (int q = tid; q < N * N * N; q += nt) {
      const int i = q % N, j = (q / N) % N, k = q / (N * N);
      dst[(long long)k * a.gtop.plane + (long long)j * a.gtop.px + i] = cur[0][q];
    }
  }
}

}  // namespace
}  // namespace h3d
