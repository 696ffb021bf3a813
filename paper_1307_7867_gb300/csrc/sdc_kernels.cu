// sdc_kernels.cu -- spectral-quadrature and FAS kernels (Sec. 1.1).
// All are point-parallel: one thread per grid point of one item, FP64.
#include "kernels.cuh"

namespace h3d {
namespace {

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ void warp_max_to(unsigned long long v, unsigned long long* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicMax(dst, v);
}

inline dim3 point_grid(const Grid& g, int B) {
  return dim3((g.N + 31) / 32, (g.N + 7) / 8, g.N * B);
}

// Quadrature integrals of one sweep and (optionally) the collocation residual
// of the current iterate.  I == nullptr: residual only.
template <int M>
__global__ void k_integrals(Grid g, const double* __restrict__ U, const double* __restrict__ F,
                            const double* __restrict__ tauS, double* __restrict__ I,
                            const ItemSDC* __restrict__ items, const double* __restrict__ phi1d,
                            unsigned long long* res_bits, const int* active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int b = blockIdx.z / g.N;
  const int k = blockIdx.z - b * g.N;
  if (active && !active[b]) return;  // uniform over the block
  unsigned long long mx = 0ull;
  if (i < g.N && j < g.N) {
    const long long idx = (long long)k * g.plane + (long long)j * g.px + i;
    const long long fs = g.fs;
    const double* Ub = U + (long long)b * M * fs + idx;
    const double* Fb = F + (long long)b * M * fs + idx;
    const ItemSDC& it = items[b];
    double Fj[M];
#pragma unroll
    for (int q = 0; q < M; ++q) Fj[q] = Fb[q * fs];
    const double phi = phi1d[i] * phi1d[j] * phi1d[k];
    const double u0 = Ub[0];
    double cum = 0.0;
#pragma unroll
    for (int m = 0; m < M - 1; ++m) {
      double J = it.gS[m] * phi;
#pragma unroll
      for (int q = 0; q < M; ++q) J = fma(it.dtS[m][q], Fj[q], J);
      if (tauS) J += tauS[((long long)b * (M - 1) + m) * fs + idx];
      if (I) {
        double Im = fma(-it.dtm[m], Fj[m + 1], J);
        if (m == 0) Im += u0;
        I[((long long)b * (M - 1) + m) * fs + idx] = Im;
      }
      if (res_bits) {
        cum += J;
        double rv = (u0 + cum) - Ub[(m + 1) * fs];
        unsigned long long bits = abs_bits(rv);
        mx = bits > mx ? bits : mx;
      }
    }
  }
  if (res_bits) warp_max_to(mx, res_bits + b);
}

// Coarse point (I, J, K) (0-based) sits on fine point (2I+1, 2J+1, 2K+1), or on
// the same point when the two grids are equal.
// X (compact fine level): qF_m = R(U_jm - U_0 + X_{m-1}) with X_{m-1} = W^{-1} r
// of coarse node m >= 1 (field m-1 of each item at item stride xs), qF_0 = 0.
template <int MF, int MG>
__global__ void k_fas_inject(Grid gf, Grid gg, int same, const double* __restrict__ UF,
                             const double* __restrict__ FF, double* __restrict__ UG,
                             double* __restrict__ UGr, double* __restrict__ qF,
                             const ItemSDC* __restrict__ itF, const FasMap* __restrict__ map,
                             const double* __restrict__ phif1d, const double* __restrict__ X,
                             long long xs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int b = blockIdx.z / gg.N;
  const int k = blockIdx.z - b * gg.N;
  if (i >= gg.N || j >= gg.N) return;
  const int fi = same ? i : 2 * i + 1, fj = same ? j : 2 * j + 1, fk = same ? k : 2 * k + 1;
  const long long fidx = (long long)fk * gf.plane + (long long)fj * gf.px + fi;
  const long long gidx = (long long)k * gg.plane + (long long)j * gg.px + i;
  const double* UFb = UF + (long long)b * MF * gf.fs + fidx;
  const double* FFb = FF + (long long)b * MF * gf.fs + fidx;
  const ItemSDC& it = itF[b];
  double Fq[MF];
#pragma unroll
  for (int q = 0; q < MF; ++q) Fq[q] = FFb[q * gf.fs];
  const double phi = phif1d[fi] * phif1d[fj] * phif1d[fk];
#pragma unroll
  for (int m = 0; m < MG; ++m) {
    const int jm = map->jm[m];
    const double v = UFb[jm * gf.fs];
    const long long o = ((long long)b * MG + m) * gg.fs + gidx;
    UG[o] = v;
    UGr[o] = v;
    if (X) {
      qF[o] = m == 0 ? 0.0 : (v - UFb[0]) + X[(long long)b * xs + (long long)(m - 1) * gf.fs + fidx];
      continue;
    }
    double q = it.gQ[jm] * phi;
#pragma unroll
    for (int p = 0; p < MF; ++p) q = fma(it.dtQ[jm][p], Fq[p], q);
    qF[o] = q;
  }
}

// Compact fine level, coarse node m (fine node jm): the weighted residual
// r = W U_0 + dt sum_p Q[jm][p] (F_p + W f_p) - W U_jm on the fine grid, into
// R (one field per item) and into X (the W-solve's start value, item stride
// xs); max |r| per item into res_bits.
template <int MF>
__global__ void k_fas_wresid(Grid gf, int jm, const double* __restrict__ WU,
                             const double* __restrict__ FF, const ItemSDC* __restrict__ itF,
                             const double* __restrict__ phif1d, double* __restrict__ R,
                             double* __restrict__ X, long long xs, unsigned long long* res_bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int b = blockIdx.z / gf.N;
  const int k = blockIdx.z - b * gf.N;
  unsigned long long mx = 0ull;
  if (i < gf.N && j < gf.N) {
    const long long idx = (long long)k * gf.plane + (long long)j * gf.px + i;
    const double* Wb = WU + (long long)b * MF * gf.fs + idx;
    const double* Fb = FF + (long long)b * MF * gf.fs + idx;
    const ItemSDC& it = itF[b];
    double q = it.gQ[jm] * (phif1d[i] * phif1d[j] * phif1d[k]);
#pragma unroll
    for (int p = 0; p < MF; ++p) q = fma(it.dtQ[jm][p], Fb[p * gf.fs], q);
    const double r = (Wb[0] + q) - Wb[jm * gf.fs];
    R[(long long)b * gf.fs + idx] = r;
    X[(long long)b * xs + idx] = r;
    mx = abs_bits(r);
  }
  warp_max_to(mx, res_bits + b);
}

template <int MG>
__global__ void k_fas_tau(Grid gg, const double* __restrict__ qF, const double* __restrict__ FG,
                          double* __restrict__ tauS, const ItemSDC* __restrict__ itG,
                          const double* __restrict__ phig1d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int b = blockIdx.z / gg.N;
  const int k = blockIdx.z - b * gg.N;
  if (i >= gg.N || j >= gg.N) return;
  const long long gidx = (long long)k * gg.plane + (long long)j * gg.px + i;
  const ItemSDC& it = itG[b];
  double Fg[MG];
#pragma unroll
  for (int q = 0; q < MG; ++q) Fg[q] = FG[((long long)b * MG + q) * gg.fs + gidx];
  const double phi = phig1d[i] * phig1d[j] * phig1d[k];
  double prev = 0.0;  // tauQ_0 = 0 (Q's first row is zero)
#pragma unroll
  for (int m = 1; m < MG; ++m) {
    double c = it.gQ[m] * phi;
#pragma unroll
    for (int q = 0; q < MG; ++q) c = fma(it.dtQ[m][q], Fg[q], c);
    const double tq = qF[((long long)b * MG + m) * gg.fs + gidx] - c;
    tauS[((long long)b * (MG - 1) + (m - 1)) * gg.fs + gidx] = tq - prev;
    prev = tq;
  }
}

template <int MF, int MG>
__global__ void k_fas_delta(Grid gg, const double* __restrict__ UG, const double* __restrict__ UGr,
                            double* __restrict__ D, const FasMap* __restrict__ map) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int b = blockIdx.z / gg.N;
  const int k = blockIdx.z - b * gg.N;
  if (i >= gg.N || j >= gg.N) return;
  const long long gidx = (long long)k * gg.plane + (long long)j * gg.px + i;
  double dl[MG];
#pragma unroll
  for (int m = 0; m < MG; ++m) {
    const long long o = ((long long)b * MG + m) * gg.fs + gidx;
    dl[m] = UG[o] - UGr[o];
  }
#pragma unroll
  for (int q = 0; q < MF; ++q) {
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < MG; ++m) s += map->L[q][m] * dl[m];
    D[((long long)b * MF + q) * gg.fs + gidx] = s;
  }
}

}  // namespace

cudaError_t launch_integrals(int M, const Grid& g, int B, const double* U, const double* F,
                             const double* tauS, double* I, const ItemSDC* items,
                             const double* phi1d, unsigned long long* res_bits,
                             const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  dim3 grd = point_grid(g, B), blk(32, 8);
  switch (M) {
    case 2: k_integrals<2><<<grd, blk, 0, st>>>(g, U, F, tauS, I, items, phi1d, res_bits, active); break;
    case 3: k_integrals<3><<<grd, blk, 0, st>>>(g, U, F, tauS, I, items, phi1d, res_bits, active); break;
    case 4: k_integrals<4><<<grd, blk, 0, st>>>(g, U, F, tauS, I, items, phi1d, res_bits, active); break;
    case 5: k_integrals<5><<<grd, blk, 0, st>>>(g, U, F, tauS, I, items, phi1d, res_bits, active); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

#define H3D_FAS_CASES(X) \
  X(5, 3) X(5, 2) X(5, 5) X(3, 3) X(3, 2) X(2, 2) X(4, 4) X(4, 2)

cudaError_t launch_fas_inject(int MF, int MG, const Grid& gf, const Grid& gg, int B,
                              const double* UF, const double* FF, double* UG, double* UGr,
                              double* qF, const ItemSDC* itF, const FasMap* map,
                              const double* phif1d, cudaStream_t st, const double* X,
                              long long xs) {
  if (B <= 0) return cudaSuccess;
  int same = gf.N == gg.N;
  dim3 grd = point_grid(gg, B), blk(32, 8);
#define X_(a, b)                                                                        \
  if (MF == a && MG == b) {                                                             \
    k_fas_inject<a, b><<<grd, blk, 0, st>>>(gf, gg, same, UF, FF, UG, UGr, qF, itF, map, \
                                            phif1d, X, xs);                             \
    count_launch();                                                                     \
    return cudaGetLastError();                                                          \
  }
  H3D_FAS_CASES(X_)
#undef X_
  return cudaErrorInvalidValue;
}

cudaError_t launch_fas_wresid(int MF, const Grid& gf, int B, int jm, const double* WU,
                              const double* FF, const ItemSDC* itF, const double* phif1d,
                              double* R, double* X, long long xs, unsigned long long* res_bits,
                              cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  dim3 grd = point_grid(gf, B), blk(32, 8);
  switch (MF) {
    case 2: k_fas_wresid<2><<<grd, blk, 0, st>>>(gf, jm, WU, FF, itF, phif1d, R, X, xs, res_bits); break;
    case 3: k_fas_wresid<3><<<grd, blk, 0, st>>>(gf, jm, WU, FF, itF, phif1d, R, X, xs, res_bits); break;
    case 4: k_fas_wresid<4><<<grd, blk, 0, st>>>(gf, jm, WU, FF, itF, phif1d, R, X, xs, res_bits); break;
    case 5: k_fas_wresid<5><<<grd, blk, 0, st>>>(gf, jm, WU, FF, itF, phif1d, R, X, xs, res_bits); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fas_tau(int MG, const Grid& gg, int B, const double* qF, const double* FG,
                           double* tauS, const ItemSDC* itG, const double* phig1d,
                           cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  dim3 grd = point_grid(gg, B), blk(32, 8);
  switch (MG) {
    case 2: k_fas_tau<2><<<grd, blk, 0, st>>>(gg, qF, FG, tauS, itG, phig1d); break;
    case 3: k_fas_tau<3><<<grd, blk, 0, st>>>(gg, qF, FG, tauS, itG, phig1d); break;
    case 4: k_fas_tau<4><<<grd, blk, 0, st>>>(gg, qF, FG, tauS, itG, phig1d); break;
    case 5: k_fas_tau<5><<<grd, blk, 0, st>>>(gg, qF, FG, tauS, itG, phig1d); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_fas_delta(int MF, int MG, const Grid& gg, int B, const double* UG,
                             const double* UGr, double* D, const FasMap* map, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  dim3 grd = point_grid(gg, B), blk(32, 8);
#define X(a, b)                                                      \
  if (MF == a && MG == b) {                                          \
    k_fas_delta<a, b><<<grd, blk, 0, st>>>(gg, UG, UGr, D, map);     \
    count_launch();                                                  \
    return cudaGetLastError();                                       \
  }
  H3D_FAS_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace h3d
