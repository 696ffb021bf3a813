// mg_kernels.cu -- point-parallel multigrid and layout kernels (Sec. 1.2):
// Jacobi from a zero initial guess and the exact one-unknown solve, full
// weighting restriction, trilinear prolongation, the FP64 update, max-norms
// and the dense <-> pitched copies.  One thread per grid point of one item;
// blockIdx.z = item * N + plane.  (The stencil kernels are in
// stencil_impl.cuh.)
#include <algorithm>

#include "kernels.cuh"

namespace h3d {
namespace {

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

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

// ---- point-parallel kernels: one thread per point, blockIdx.z = item * N + k ----

struct PointIdx {
  int b, i, j, k;
  long long idx;
};

__device__ __forceinline__ bool point_index(const Grid& g, PointIdx& p) {
  p.i = blockIdx.x * blockDim.x + threadIdx.x;
  p.j = blockIdx.y * blockDim.y + threadIdx.y;
  p.b = blockIdx.z / g.N;
  p.k = blockIdx.z - p.b * g.N;
  if (p.i >= g.N || p.j >= g.N) return false;
  p.idx = (long long)p.k * g.plane + (long long)p.j * g.px + p.i;
  return true;
}

inline dim3 point_grid(const Grid& g, int B) {
  return dim3((g.N + 31) / 32, (g.N + 7) / 8, g.N * B);
}

// The one-unknown grid's exact solve from the scaled right-hand side.
template <typename T>
__global__ void k_solve_one(Grid g, const T* __restrict__ r, T* __restrict__ e,
                            const Coef<T>* coef, const int* active) {
  PointIdx p;
  if (!point_index(g, p)) return;
  if (active && !active[p.b]) return;
  long long o = p.b * g.fs + p.idx;
  e[o] = r[o] / coef[p.b].a11w;
}

// Full weighting (fw3 in common.cuh) into the coarse level's scaled
// right-hand side.  A thread owns coarse column (I, J) and marches over a
// chunk of kc coarse planes: the plane sum Y of fine plane 2K+2 closes coarse
// plane K and opens K+1, so each coarse point costs two plane sums (8
// operations each), the z combination and the scaling: 19 operations instead
// of 27 (plus 8 per chunk for its first plane).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(Grid gf, Grid gc, const T* __restrict__ rr,
                                                  T* __restrict__ bc, const Coef<T>* cc, int kc,
                                                  const int* active) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int nkc = (gc.N + kc - 1) / kc;
  const int b = blockIdx.z / nkc;
  const int K0 = (blockIdx.z - b * nkc) * kc, K1 = min(gc.N, K0 + kc);
  if (I >= gc.N || J >= gc.N) return;
  if (active && !active[b]) return;
  const T* f = rr + b * gf.fs + (long long)(2 * J) * gf.px + 2 * I;  // fine (2I, 2J, 0)
  const long long px = gf.px;
  auto plane_sum = [&](int p) {
    const T* q = f + (long long)p * gf.plane;
    const T x0 = fw3(ldg(q), ldg(q + 1), ldg(q + 2));
    const T x1 = fw3(ldg(q + px), ldg(q + px + 1), ldg(q + px + 2));
    const T x2 = fw3(ldg(q + 2 * px), ldg(q + 2 * px + 1), ldg(q + 2 * px + 2));
    return fw3(x0, x1, x2);
  };
  const T sc = cc[b].rs * T(0.015625);
  T* out = bc + b * gc.fs + (long long)J * gc.px + I;
  T ylo = plane_sum(2 * K0);
  for (int K = K0; K < K1; ++K) {
    const T y1 = plane_sum(2 * K + 1), y2 = plane_sum(2 * K + 2);
    out[(long long)K * gc.plane] = fw3(ylo, y1, y2) * sc;
    ylo = y2;
  }
}

// Trilinear prolongation, one thread per coarse cell.  In 1-based indices the
// cell C = 0..Nc spans coarse points C and C+1 (0 and Nc+1 are the Dirichlet
// zeros) and owns the fine points 2C+1 (midway: mean of the two) and 2C+2 (on
// coarse point C+1), per axis; in 0-based fine indices those are 2C and 2C+1,
// so x-pairs are read and written as aligned two-element vectors.  The eight
// corner values are combined axis by axis (x, then y, then z) and scaled by
// 1/2 per averaged axis: 27 arithmetic operations per 8 fine points, no
// divergent branches.
template <typename T>
struct Vec2;
template <>
struct Vec2<double> { using type = double2; };
template <>
struct Vec2<float> { using type = float2; };

template <typename T>
__device__ __forceinline__ T cval(const T* __restrict__ e, const Grid& gc, int i, int j, int k) {
  if (i < 0 || i >= gc.N || j < 0 || j >= gc.N || k < 0 || k >= gc.N) return T(0);
  return ldg(e + (long long)k * gc.plane + (long long)j * gc.px + i);
}

template <typename T>
__global__ void k_prolong_add(Grid gc, Grid gf, const T* __restrict__ ec, long long ecs,
                              const T* src, T* uf, long long ufs, const int* active) {
  using V2 = typename Vec2<T>::type;
  const int nc1 = gc.N + 1;  // cells per axis
  const int cx = blockIdx.x * blockDim.x + threadIdx.x;
  const int cy = blockIdx.y * blockDim.y + threadIdx.y;
  const int b = blockIdx.z / nc1;
  const int cz = blockIdx.z - b * nc1;
  if (cx >= nc1 || cy >= nc1) return;
  if (active && !active[b]) return;
  const T* e = ec + b * ecs;
  // corner values v[z][y][x], 0 = low (coarse 0-based C-1), 1 = high (C)
  T v[2][2][2];
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y)
#pragma unroll
      for (int x = 0; x < 2; ++x) v[z][y][x] = cval(e, gc, cx - 1 + x, cy - 1 + y, cz - 1 + z);
  // x: A = sum of the pair (midpoint, scaled later), E = high value
  T X[2][2][2];  // [z][y][mode x: 0 mid, 1 on-point]
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      X[z][y][0] = v[z][y][0] + v[z][y][1];
      X[z][y][1] = v[z][y][1];
    }
  T Y[2][2][2];  // [z][mode y][mode x]
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int mx = 0; mx < 2; ++mx) {
      Y[z][0][mx] = X[z][0][mx] + X[z][1][mx];
      Y[z][1][mx] = X[z][1][mx];
    }
  const int Nf = gf.N;
  const int fx = 2 * cx, fy0 = 2 * cy, fz0 = 2 * cz;  // 0-based fine index of the mid points
  T* u = uf + b * ufs;
  const T* us = src + b * ufs;
  // src may be uf: every value is loaded before the first store, so that the
  // loads need not wait for stores they might alias (each point is read and
  // written by this thread only)
  V2 o[2][2];
  T o1[2][2];
#pragma unroll
  for (int mz = 0; mz < 2; ++mz)
#pragma unroll
    for (int my = 0; my < 2; ++my) {
      const int fz = fz0 + mz, fy = fy0 + my;
      if (fz >= Nf || fy >= Nf) continue;
      const T* srow = us + (long long)fz * gf.plane + (long long)fy * gf.px;
      if (fx + 1 < Nf) o[mz][my] = *reinterpret_cast<const V2*>(srow + fx);
      else if (fx < Nf) o1[mz][my] = srow[fx];
    }
#pragma unroll
  for (int mz = 0; mz < 2; ++mz) {
    const int fz = fz0 + mz;
    if (fz >= Nf) continue;
#pragma unroll
    for (int my = 0; my < 2; ++my) {
      const int fy = fy0 + my;
      if (fy >= Nf) continue;
      T val[2];
#pragma unroll
      for (int mx = 0; mx < 2; ++mx) {
        T w = mz == 0 ? Y[0][my][mx] + Y[1][my][mx] : Y[1][my][mx];
        const int na = (mx == 0) + (my == 0) + (mz == 0);  // averaged axes
        val[mx] = na == 0 ? w : w * (na == 1 ? T(0.5) : na == 2 ? T(0.25) : T(0.125));
      }
      T* row = u + (long long)fz * gf.plane + (long long)fy * gf.px;
      if (fx + 1 < Nf) {
        V2 r = o[mz][my];
        r.x += val[0];
        r.y += val[1];
        *reinterpret_cast<V2*>(row + fx) = r;
      } else if (fx < Nf) {
        row[fx] = o1[mz][my] + val[0];
      }
    }
  }
}

// Taps of the cubic interpolation along one axis for fine index f (0-based):
// even 1-based fine points take their coarse point, odd ones the 4-point
// midpoint weights (-1, 9, 9, -1) / 16; coarse points 0 and Nc + 1 (1-based)
// are the zero boundary, points beyond are odd reflections.  Always four
// taps (unused ones weigh 0, index kept valid) so that they stay in registers.
__device__ __forceinline__ void cubic_taps(int f, int Nc, int (&ix)[4], double (&w)[4]) {
  const int f1 = f + 1;
  if ((f1 & 1) == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ix[q] = f1 / 2 - 1;
      w[q] = q == 0 ? 1.0 : 0.0;
    }
    return;
  }
  const int I = (f1 - 1) / 2;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int a = I - 1 + q;
    double cw = (q == 1 || q == 2) ? 9.0 / 16.0 : -1.0 / 16.0;
    if (a == 0 || a == Nc + 1) { cw = 0.0; a = 1; }
    if (a < 0) { a = -a; cw = -cw; }
    if (a > Nc + 1) { a = 2 * (Nc + 1) - a; cw = -cw; }
    ix[q] = a - 1;
    w[q] = cw;
  }
}

// Taps of the 6- and 8-point midpoint rules, the Lagrange weights of equally
// spaced points evaluated halfway between the middle two ((3, -25, 150, 150,
// -25, 3) / 256 and (-5, 49, -245, 1225, 1225, -245, 49, -5) / 2048, exact in
// binary): even 1-based fine points take their coarse point, odd ones the NT
// coarse values around the midpoint on the odd extension of the coarse line
// about both boundary points (period 2 (Nc + 1)), which also covers stencils
// that reach past a boundary more than once on small grids.  Always NT taps
// (unused ones weigh 0, index kept valid).
template <int NT>
__host__ __device__ __forceinline__ double mid_weight(int q) {
  if (NT == 6) {
    const double w6[6] = {3.0, -25.0, 150.0, 150.0, -25.0, 3.0};
    return w6[q] / 256.0;
  }
  const double w8[8] = {-5.0, 49.0, -245.0, 1225.0, 1225.0, -245.0, 49.0, -5.0};
  return w8[q] / 2048.0;
}

template <int NT>
__host__ __device__ __forceinline__ void mid_taps(int f, int Nc, int (&ix)[NT], double (&w)[NT]) {
  const int f1 = f + 1;
  if ((f1 & 1) == 0) {
#pragma unroll
    for (int q = 0; q < NT; ++q) {
      ix[q] = f1 / 2 - 1;
      w[q] = q == 0 ? 1.0 : 0.0;
    }
    return;
  }
  const int I = (f1 - 1) / 2;  // the midpoint lies between coarse points I and I + 1 (1-based)
  const int per = 2 * (Nc + 1);
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    double cw = mid_weight<NT>(q);
    int r = (I - NT / 2 + 1 + q) % per;
    if (r < 0) r += per;
    int idx = r - 1;
    if (r == 0 || r == Nc + 1) {
      cw = 0.0;
      idx = 0;
    } else if (r > Nc + 1) {
      cw = -cw;
      idx = per - r - 1;
    }
    ix[q] = idx;
    w[q] = cw;
  }
}

// Taps of the NT-point rule (4: cubic_taps).
template <int NT>
__device__ __forceinline__ void interp_taps(int f, int Nc, int (&ix)[NT], double (&w)[NT]) {
  if constexpr (NT == 4) cubic_taps(f, Nc, ix, w);
  else mid_taps<NT>(f, Nc, ix, w);
}

// uf += P ec (NT-point midpoint rule per axis): one thread per fine point,
// separable sums x, then y, then z (zero-weight taps are skipped).
template <int NT>
__global__ void k_prolong_mid(Grid gc, Grid gf, const double* __restrict__ ec, long long ecs,
                              double* __restrict__ uf, long long ufs) {
  PointIdx p;
  if (!point_index(gf, p)) return;
  int xi[NT], yi[NT], zi[NT];
  double xw[NT], yw[NT], zw[NT];
  interp_taps<NT>(p.i, gc.N, xi, xw);
  interp_taps<NT>(p.j, gc.N, yi, yw);
  interp_taps<NT>(p.k, gc.N, zi, zw);
  const double* e = ec + p.b * ecs;
  double sz = 0.0;
#pragma unroll
  for (int c = 0; c < NT; ++c) {
    if (zw[c] == 0.0) continue;
    double sy = 0.0;
#pragma unroll
    for (int b = 0; b < NT; ++b) {
      if (yw[b] == 0.0) continue;
      const double* row = e + (long long)zi[c] * gc.plane + (long long)yi[b] * gc.px;
      double sx = 0.0;
#pragma unroll
      for (int a = 0; a < NT; ++a)
        if (xw[a] != 0.0) sx = fma(xw[a], __ldg(row + xi[a]), sx);
      sy = fma(yw[b], sx, sy);
    }
    sz = fma(zw[c], sy, sz);
  }
  double* o = uf + p.b * ufs + p.idx;
  *o = *o + sz;
}

// The same interpolation as k_prolong_mid in three one-axis passes through
// dense temporaries (t1: [K][J][Nf], t2: [K][Nf][Nf] per item), with the sums
// in the same order (x, then y, then z), so the result is bitwise the same
// while each fine point costs a few fused multiply-adds instead of up to NT^3.
template <int NT>
__global__ void k_mid_x(Grid gc, int Nf, const double* __restrict__ ec, long long ecs,
                        double* __restrict__ t1, long long t1s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // fine x
  const int J = blockIdx.y * blockDim.y + threadIdx.y;  // coarse y
  const int Nc = gc.N;
  const int b = blockIdx.z / Nc, K = blockIdx.z - b * Nc;
  if (i >= Nf || J >= Nc) return;
  int xi[NT];
  double xw[NT];
  interp_taps<NT>(i, Nc, xi, xw);
  const double* row = ec + b * ecs + (long long)K * gc.plane + (long long)J * gc.px;
  double sx = 0.0;
#pragma unroll
  for (int a = 0; a < NT; ++a)
    if (xw[a] != 0.0) sx = fma(xw[a], __ldg(row + xi[a]), sx);
  t1[b * t1s + ((long long)K * Nc + J) * Nf + i] = sx;
}

template <int NT>
__global__ void k_mid_y(int Nc, int Nf, const double* __restrict__ t1, long long t1s,
                        double* __restrict__ t2, long long t2s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // fine x
  const int j = blockIdx.y * blockDim.y + threadIdx.y;  // fine y
  const int b = blockIdx.z / Nc, K = blockIdx.z - b * Nc;
  if (i >= Nf || j >= Nf) return;
  int yi[NT];
  double yw[NT];
  interp_taps<NT>(j, Nc, yi, yw);
  const double* s = t1 + b * t1s + (long long)K * Nc * Nf + i;
  double sy = 0.0;
#pragma unroll
  for (int q = 0; q < NT; ++q)
    if (yw[q] != 0.0) sy = fma(yw[q], s[(long long)yi[q] * Nf], sy);
  t2[b * t2s + ((long long)K * Nf + j) * Nf + i] = sy;
}

template <int NT>
__global__ void k_mid_z(Grid gf, int Nc, const double* __restrict__ t2, long long t2s,
                        double* __restrict__ uf, long long ufs) {
  PointIdx p;
  if (!point_index(gf, p)) return;
  const int Nf = gf.N;
  int zi[NT];
  double zw[NT];
  interp_taps<NT>(p.k, Nc, zi, zw);
  const double* s = t2 + p.b * t2s + (long long)p.j * Nf + p.i;
  double sz = 0.0;
#pragma unroll
  for (int q = 0; q < NT; ++q)
    if (zw[q] != 0.0) sz = fma(zw[q], s[(long long)zi[q] * Nf * Nf], sz);
  double* o = uf + p.b * ufs + p.idx;
  *o = *o + sz;
}

template <typename T>
__global__ void k_update(Grid g, const T* __restrict__ e, double* __restrict__ u, long long us,
                         const int* active) {
  PointIdx p;
  if (!point_index(g, p)) return;
  if (active && !active[p.b]) return;
  double* o = u + p.b * us + p.idx;
  *o = *o + (double)e[p.b * g.fs + p.idx];
}

__global__ void k_maxabs(Grid g, const double* __restrict__ u, long long us,
                         unsigned long long* norm_bits, const int* active) {
  PointIdx p;
  bool ok = point_index(g, p);
  unsigned long long v = 0ull;
  if (ok && !(active && !active[p.b])) v = abs_bits(u[p.b * us + p.idx]);
  // blockIdx.z fixes the item: every lane of the warp shares b
  int b = blockIdx.z / g.N;
  warp_max_to(v, norm_bits + b);
}

__global__ void k_dense_to_pitched(Grid g, const double* __restrict__ d, double* __restrict__ f,
                                   long long fsd) {
  PointIdx p;
  if (!point_index(g, p)) return;
  long long n = (long long)g.N;
  f[p.b * fsd + p.idx] = d[((p.b * n + p.k) * n + p.j) * n + p.i];
}

__global__ void k_pitched_to_dense(Grid g, const double* __restrict__ f, long long fsd,
                                   double* __restrict__ d) {
  PointIdx p;
  if (!point_index(g, p)) return;
  long long n = (long long)g.N;
  d[((p.b * n + p.k) * n + p.j) * n + p.i] = f[p.b * fsd + p.idx];
}

__global__ void k_copy(Grid g, const double* __restrict__ s, long long ss, double* __restrict__ d,
                       long long ds) {
  PointIdx p;
  if (!point_index(g, p)) return;
  d[p.b * ds + p.idx] = s[p.b * ss + p.idx];
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <typename T>
cudaError_t launch_solve_one(const Grid& g, int B, const T* r, T* e, const Coef<T>* coef,
                             const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_solve_one<T><<<point_grid(g, B), dim3(32, 8), 0, st>>>(g, r, e, coef, active);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, int B, const T* rr, T* bc,
                            const Coef<T>* cc, const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  // coarse planes per thread: in FP64 (bound by the FP64 pipe) long runs that
  // share plane sums, where there are columns enough to fill the GPU; in FP32
  // (bound by memory latency and bandwidth) one plane per thread, for the
  // most loads in flight
  const int kc = sizeof(T) == 8 ? std::max(1, std::min(8, gc.N / 16)) : 1;
  const int nkc = (gc.N + kc - 1) / kc;
  k_restrict<T><<<dim3((gc.N + 31) / 32, (gc.N + 7) / 8, nkc * B), dim3(32, 8), 0, st>>>(
      gf, gc, rr, bc, cc, kc, active);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(const Grid& gc, const Grid& gf, int B, const T* ec,
                               long long ec_stride, const T* src, T* uf, long long uf_stride,
                               const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int nc1 = gc.N + 1;
  k_prolong_add<T><<<dim3((nc1 + 31) / 32, (nc1 + 7) / 8, nc1 * B), dim3(32, 8), 0, st>>>(
      gc, gf, ec, ec_stride, src, uf, uf_stride, active);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_mg_check(int B, const unsigned long long* __restrict__ norm_bits, int* active,
                           const double* __restrict__ tol, int* ncyc, double* last,
                           const int* max_cycles, int* nan_flag, int init) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || !active[b]) return;
  const double n = __longlong_as_double((long long)norm_bits[b]);
  last[b] = n;
  if (!(n <= 1e300)) {
    *nan_flag = 1;
    active[b] = 0;
    return;
  }
  if (!init) ncyc[b] += 1;
  if (n <= tol[b] || (!init && ncyc[b] >= *max_cycles)) active[b] = 0;
}

cudaError_t launch_mg_check(int B, const unsigned long long* norm_bits, int* active,
                            const double* tol, int* ncyc, double* last, const int* max_cycles,
                            int* nan_flag, bool init, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_mg_check<<<(B + 63) / 64, 64, 0, st>>>(B, norm_bits, active, tol, ncyc, last, max_cycles,
                                           nan_flag, init ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

template <int NT>
static cudaError_t prolong_mid(const Grid& gc, const Grid& gf, int B, const double* ec,
                               long long ec_stride, double* uf, long long uf_stride, cudaStream_t st,
                               double* t1, double* t2, long long t_stride) {
  if (!t1 || !t2) {
    k_prolong_mid<NT><<<point_grid(gf, B), dim3(32, 8), 0, st>>>(gc, gf, ec, ec_stride, uf, uf_stride);
    count_launch();
    return cudaGetLastError();
  }
  const int Nc = gc.N, Nf = gf.N;
  const dim3 blk(32, 8);
  k_mid_x<NT><<<dim3((Nf + 31) / 32, (Nc + 7) / 8, Nc * B), blk, 0, st>>>(gc, Nf, ec, ec_stride, t1,
                                                                           t_stride);
  count_launch();
  k_mid_y<NT><<<dim3((Nf + 31) / 32, (Nf + 7) / 8, Nc * B), blk, 0, st>>>(Nc, Nf, t1, t_stride, t2,
                                                                           t_stride);
  count_launch();
  k_mid_z<NT><<<point_grid(gf, B), blk, 0, st>>>(gf, Nc, t2, t_stride, uf, uf_stride);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_prolong_add_mid(int npts, const Grid& gc, const Grid& gf, int B,
                                   const double* ec, long long ec_stride, double* uf,
                                   long long uf_stride, cudaStream_t st, double* t1, double* t2,
                                   long long t_stride) {
  if (B <= 0) return cudaSuccess;
  switch (npts) {
    case 4: return prolong_mid<4>(gc, gf, B, ec, ec_stride, uf, uf_stride, st, t1, t2, t_stride);
    case 6: return prolong_mid<6>(gc, gf, B, ec, ec_stride, uf, uf_stride, st, t1, t2, t_stride);
    case 8: return prolong_mid<8>(gc, gf, B, ec, ec_stride, uf, uf_stride, st, t1, t2, t_stride);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_update(const Grid& g, int B, const T* e, double* u64, long long u64_stride,
                          const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_update<T><<<point_grid(g, B), dim3(32, 8), 0, st>>>(g, e, u64, u64_stride, active);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_maxabs(const Grid& g, int B, const double* u, long long u_stride,
                          unsigned long long* norm_bits, const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_maxabs<<<point_grid(g, B), dim3(32, 8), 0, st>>>(g, u, u_stride, norm_bits, active);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_dense_to_pitched(const Grid& g, int B, const double* dense, double* f,
                                    long long f_stride, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_dense_to_pitched<<<point_grid(g, B), dim3(32, 8), 0, st>>>(g, dense, f, f_stride);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pitched_to_dense(const Grid& g, int B, const double* f, long long f_stride,
                                    double* dense, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_pitched_to_dense<<<point_grid(g, B), dim3(32, 8), 0, st>>>(g, f, f_stride, dense);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_copy(const Grid& g, int B, const double* src, long long src_stride,
                        double* dst, long long dst_stride, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_copy<<<point_grid(g, B), dim3(32, 8), 0, st>>>(g, src, src_stride, dst, dst_stride);
  count_launch();
  return cudaGetLastError();
}

#define H3D_INST(T)                                                                            \
  template cudaError_t launch_solve_one<T>(const Grid&, int, const T*, T*, const Coef<T>*,     \
                                           const int*, cudaStream_t);                           \
  template cudaError_t launch_restrict<T>(const Grid&, const Grid&, int, const T*, T*,         \
                                          const Coef<T>*, const int*, cudaStream_t);            \
  template cudaError_t launch_prolong_add<T>(const Grid&, const Grid&, int, const T*, long long,\
                                             const T*, T*, long long, const int*, cudaStream_t);\
  template cudaError_t launch_update<T>(const Grid&, int, const T*, double*, long long,        \
                                        const int*, cudaStream_t);
H3D_INST(double)
H3D_INST(float)
#undef H3D_INST

}  // namespace h3d
