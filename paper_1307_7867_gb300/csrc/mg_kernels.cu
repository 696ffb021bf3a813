// mg_kernels.cu -- stencil and multigrid kernels (Sec. 1 method of lines,
// Sec. 1.2 multigrid), templated on the storage type (double / float) and on
// the stencil order (2: 7 points, 4: 13-point wide stencil).
//
// Stencil kernels march along z: each thread owns one (x, y) column of a
// zc-plane chunk and keeps the column's z-neighbours in a register queue, so
// every plane of the input is fetched from DRAM once per chunk; the x/y
// neighbours of the current plane come from L1 (the neighbouring threads of
// the block load the same rows).  Boundary rule of every stencil read:
// indices -1 and N are the Dirichlet zeros; the wide stencil's ghosts -2 and
// N+1 are -u(0) and -u(N-1) (odd reflection).
#include "kernels.cuh"

namespace h3d {
namespace {

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Value at (i, j, k) with the boundary rule; each index within [-2, N+1].
template <typename T>
__device__ __forceinline__ T at(const T* __restrict__ u, const Grid& g, int i, int j, int k) {
  const int N = g.N;
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
  T v = ldg(u + (long long)k * g.plane + (long long)j * g.px + i);
  return neg ? -v : v;
}

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Max over the warp of 64-bit patterns; lane 0 adds it to *dst.
__device__ __forceinline__ void warp_max_to(unsigned long long v, unsigned long long* dst) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0 && v != 0ull) atomicMax(dst, v);
}

// The z-marching driver.  Op supplies src(b) (the field whose stencil is
// taken), init(b) (per-item coefficients) and apply(b, idx, u, s1, s2) with
// u the centre value, s1 the sum of the 6 nearest neighbours and s2 the sum of
// the 6 second neighbours (order 4 only).  apply returns a value whose
// absolute maximum is accumulated when norm_bits != nullptr.
template <typename T, int ORDER, typename Op>
__global__ void __launch_bounds__(256) k_zmarch(Grid g, int nzc, int zc, const int* active,
                                                unsigned long long* norm_bits, Op op) {
  constexpr int R = ORDER == 2 ? 1 : 2;
  const int b = blockIdx.z / nzc;
  if (active && !active[b]) return;  // uniform over the block
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int z0 = (blockIdx.z - b * nzc) * zc;
  const int z1 = min(g.N, z0 + zc);
  unsigned long long mx = 0ull;
  if (i < g.N && j < g.N) {
    Op o = op;
    o.init(b);
    const T* __restrict__ u = o.src(b);
    T q[2 * R + 1];
#pragma unroll
    for (int d = -R; d <= R; ++d) q[R + d] = at(u, g, i, j, z0 + d);
    const bool inner = i >= R && i < g.N - R && j >= R && j < g.N - R;
    const long long px = g.px;
    for (int k = z0; k < z1; ++k) {
      const long long idx = (long long)k * g.plane + (long long)j * px + i;
      T s1, s2 = T(0);
      if (inner) {
        const T* c = u + idx;
        s1 = ((ldg(c - 1) + ldg(c + 1)) + (ldg(c - px) + ldg(c + px))) + (q[R - 1] + q[R + 1]);
        if (R == 2)
          s2 = ((ldg(c - 2) + ldg(c + 2)) + (ldg(c - 2 * px) + ldg(c + 2 * px))) + (q[0] + q[2 * R]);
      } else {
        s1 = ((at(u, g, i - 1, j, k) + at(u, g, i + 1, j, k)) +
              (at(u, g, i, j - 1, k) + at(u, g, i, j + 1, k))) + (q[R - 1] + q[R + 1]);
        if (R == 2)
          s2 = ((at(u, g, i - 2, j, k) + at(u, g, i + 2, j, k)) +
                (at(u, g, i, j - 2, k) + at(u, g, i, j + 2, k))) + (q[0] + q[2 * R]);
      }
      double rv = (double)o.apply(b, idx, q[R], s1, s2);
      if (norm_bits) {
        unsigned long long bits = abs_bits(rv);
        mx = bits > mx ? bits : mx;
      }
#pragma unroll
      for (int d = 0; d < 2 * R; ++d) q[d] = q[d + 1];
      if (k + 1 < z1) q[2 * R] = at(u, g, i, j, k + R + 1);
    }
  }
  if (norm_bits) warp_max_to(mx, norm_bits + b);
}

template <typename T, int ORDER>
__device__ __forceinline__ T combine(T s1, T s2) {
  if (ORDER == 2) return s1;
  return fma(T(16), s1, -s2);
}

// ---- operators ----

template <int ORDER>
struct OpLap {
  const double* u; long long us;
  double* out; long long os;
  const double* alpha;
  const double* add_src; double* add_dst; long long as;
  double a;
  __device__ const double* src(int b) const { return u + b * us; }
  __device__ void init(int b) { a = alpha[b]; }
  __device__ double apply(int b, long long idx, double c, double s1, double s2) {
    double L = ORDER == 2 ? fma(-6.0, c, s1) : fma(-90.0, c, fma(16.0, s1, -s2));
    out[b * os + idx] = a * L;
    if (add_src) add_dst[b * as + idx] = c + add_src[b * as + idx];
    return 0.0;
  }
};

template <int ORDER, typename TR>
struct OpResid64 {
  const double* u; long long us;
  const double* bb; long long bs;
  const Coef<double>* coef;
  TR* r; TR* e0; const Coef<TR>* coef_r; long long rs;
  double d, e; TR wd;
  __device__ const double* src(int b) const { return u + b * us; }
  __device__ void init(int b) {
    d = coef[b].d; e = coef[b].e;
    wd = e0 ? coef_r[b].wd : TR(0);
  }
  __device__ double apply(int b, long long idx, double c, double s1, double s2) {
    double S = combine<double, ORDER>(s1, s2);
    double res = fma(-d, c, fma(e, S, bb[b * bs + idx]));
    TR rt = (TR)res;
    r[b * rs + idx] = rt;
    if (e0) e0[b * rs + idx] = wd * rt;
    return res;
  }
};

template <typename T, int ORDER>
struct OpJacobi {
  const T* e; const T* r; T* out; long long fs;
  double* u64; long long u64s;
  const Coef<T>* coef;
  T d, ec, wd;
  __device__ const T* src(int b) const { return e + b * fs; }
  __device__ void init(int b) { d = coef[b].d; ec = coef[b].e; wd = coef[b].wd; }
  __device__ T apply(int b, long long idx, T c, T s1, T s2) {
    T S = combine<T, ORDER>(s1, s2);
    T res = fma(-d, c, fma(ec, S, r[b * fs + idx]));
    T v = fma(wd, res, c);
    if (u64) {
      double* p = u64 + b * u64s + idx;
      *p = *p + (double)v;
    } else {
      out[b * fs + idx] = v;
    }
    return T(0);
  }
};

template <typename T, int ORDER>
struct OpResid {
  const T* e; const T* r; T* rr; long long fs;
  const Coef<T>* coef;
  T d, ec;
  __device__ const T* src(int b) const { return e + b * fs; }
  __device__ void init(int b) { d = coef[b].d; ec = coef[b].e; }
  __device__ T apply(int b, long long idx, T c, T s1, T s2) {
    T S = combine<T, ORDER>(s1, s2);
    rr[b * fs + idx] = fma(-d, c, fma(ec, S, r[b * fs + idx]));
    return T(0);
  }
};

template <typename T, int ORDER, typename Op>
cudaError_t run_zmarch(const Grid& g, int B, const int* active, unsigned long long* norm_bits,
                       const Op& op, Shape sh, cudaStream_t st) {
  if (B <= 0 || g.N <= 0) return cudaSuccess;
  int zc = sh.zc > 0 ? sh.zc : 16;
  if (zc > g.N) zc = g.N;
  int nzc = (g.N + zc - 1) / zc;
  dim3 blk(sh.bx, sh.by, 1);
  dim3 grd((g.N + sh.bx - 1) / sh.bx, (g.N + sh.by - 1) / sh.by, nzc * B);
  k_zmarch<T, ORDER, Op><<<grd, blk, 0, st>>>(g, nzc, zc, active, norm_bits, op);
  count_launch();
  return cudaGetLastError();
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

template <typename T>
__global__ void k_jacobi_zero(Grid g, const T* __restrict__ r, T* __restrict__ e,
                              const Coef<T>* coef, int exact, const int* active) {
  PointIdx p;
  if (!point_index(g, p)) return;
  if (active && !active[p.b]) return;
  long long o = p.b * g.fs + p.idx;
  if (exact) e[o] = r[o] / coef[p.b].a11;
  else e[o] = coef[p.b].wd * r[o];
}

// Full weighting at the coarse point (I, J, K) <- fine (2I+1, 2J+1, 2K+1) in
// 0-based indices, weights (1/4, 1/2, 1/4) per axis, summed z, y, x in order.
template <typename T>
__global__ void k_restrict(Grid gf, Grid gc, const T* __restrict__ rr, T* __restrict__ bc,
                           const int* active) {
  PointIdx p;
  if (!point_index(gc, p)) return;
  if (active && !active[p.b]) return;
  const T w[3] = {T(0.25), T(0.5), T(0.25)};
  const T* f = rr + p.b * gf.fs;
  const int fi = 2 * p.i + 1, fj = 2 * p.j + 1, fk = 2 * p.k + 1;
  T s = T(0);
#pragma unroll
  for (int c = -1; c <= 1; ++c)
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
      const T* row = f + (long long)(fk + c) * gf.plane + (long long)(fj + b) * gf.px + fi;
      T wcb = w[c + 1] * w[b + 1];
#pragma unroll
      for (int a = -1; a <= 1; ++a) s = fma(wcb * w[a + 1], ldg(row + a), s);
    }
  bc[p.b * gc.fs + p.idx] = s;
}

// Trilinear prolongation: fine (0-based) index i corresponds to the 1-based
// fine index i+1; even 1-based indices sit on coarse points, odd ones average
// the two coarse neighbours (zero outside).
template <typename T>
__global__ void k_prolong_add(Grid gc, Grid gf, const T* __restrict__ ec, long long ecs,
                              T* __restrict__ uf, long long ufs, const int* active) {
  PointIdx p;
  if (!point_index(gf, p)) return;
  if (active && !active[p.b]) return;
  const T* e = ec + p.b * ecs;
  int ia[2], ja[2], ka[2], ni, nj, nk;
  // 1-based fine index I = i + 1; coarse 1-based neighbours I/2 or (I-1)/2,(I+1)/2; to 0-based: -1
  {
    int I = p.i + 1;
    if ((I & 1) == 0) { ia[0] = I / 2 - 1; ni = 1; } else { ia[0] = (I - 1) / 2 - 1; ia[1] = (I + 1) / 2 - 1; ni = 2; }
    int J = p.j + 1;
    if ((J & 1) == 0) { ja[0] = J / 2 - 1; nj = 1; } else { ja[0] = (J - 1) / 2 - 1; ja[1] = (J + 1) / 2 - 1; nj = 2; }
    int K = p.k + 1;
    if ((K & 1) == 0) { ka[0] = K / 2 - 1; nk = 1; } else { ka[0] = (K - 1) / 2 - 1; ka[1] = (K + 1) / 2 - 1; nk = 2; }
  }
  const int Nc = gc.N;
  const T scale = T(1) / T(ni * nj * nk);
  T s = T(0);
  for (int c = 0; c < nk; ++c) {
    int kk = ka[c];
    if (kk < 0 || kk >= Nc) continue;
    for (int b = 0; b < nj; ++b) {
      int jj = ja[b];
      if (jj < 0 || jj >= Nc) continue;
      const T* row = e + (long long)kk * gc.plane + (long long)jj * gc.px;
      for (int a = 0; a < ni; ++a) {
        int ii = ia[a];
        if (ii < 0 || ii >= Nc) continue;
        s += ldg(row + ii) * scale;
      }
    }
  }
  T* o = uf + p.b * ufs + p.idx;
  *o = *o + s;
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

cudaError_t launch_lap(int order, const Grid& g, int B, const double* u, long long u_stride,
                       double* out, long long out_stride, const double* alpha,
                       const double* add_src, double* add_dst, long long add_stride,
                       const int* active, Shape sh, cudaStream_t st) {
  if (order == 2) {
    OpLap<2> op{u, u_stride, out, out_stride, alpha, add_src, add_dst, add_stride, 0.0};
    return run_zmarch<double, 2>(g, B, active, nullptr, op, sh, st);
  }
  OpLap<4> op{u, u_stride, out, out_stride, alpha, add_src, add_dst, add_stride, 0.0};
  return run_zmarch<double, 4>(g, B, active, nullptr, op, sh, st);
}

template <typename TR>
cudaError_t launch_resid64(int order, const Grid& g, int B, const double* u, long long u_stride,
                           const double* b, long long b_stride, const Coef<double>* coef,
                           TR* r_out, TR* e0_out, const Coef<TR>* coef_r,
                           unsigned long long* norm_bits, const int* active, Shape sh,
                           cudaStream_t st) {
  if (order == 2) {
    OpResid64<2, TR> op{u, u_stride, b, b_stride, coef, r_out, e0_out, coef_r, g.fs, 0.0, 0.0, TR(0)};
    return run_zmarch<double, 2>(g, B, active, norm_bits, op, sh, st);
  }
  OpResid64<4, TR> op{u, u_stride, b, b_stride, coef, r_out, e0_out, coef_r, g.fs, 0.0, 0.0, TR(0)};
  return run_zmarch<double, 4>(g, B, active, norm_bits, op, sh, st);
}

template <typename T>
cudaError_t launch_jacobi(int order, const Grid& g, int B, const T* e, const T* r, T* out,
                          double* u64, long long u64_stride, const Coef<T>* coef,
                          const int* active, Shape sh, cudaStream_t st) {
  if (order == 2) {
    OpJacobi<T, 2> op{e, r, out, g.fs, u64, u64_stride, coef, T(0), T(0), T(0)};
    return run_zmarch<T, 2>(g, B, active, nullptr, op, sh, st);
  }
  OpJacobi<T, 4> op{e, r, out, g.fs, u64, u64_stride, coef, T(0), T(0), T(0)};
  return run_zmarch<T, 4>(g, B, active, nullptr, op, sh, st);
}

template <typename T>
cudaError_t launch_resid(int order, const Grid& g, int B, const T* e, const T* r, T* rr,
                         const Coef<T>* coef, const int* active, Shape sh, cudaStream_t st) {
  if (order == 2) {
    OpResid<T, 2> op{e, r, rr, g.fs, coef, T(0), T(0)};
    return run_zmarch<T, 2>(g, B, active, nullptr, op, sh, st);
  }
  OpResid<T, 4> op{e, r, rr, g.fs, coef, T(0), T(0)};
  return run_zmarch<T, 4>(g, B, active, nullptr, op, sh, st);
}

template <typename T>
cudaError_t launch_jacobi_zero(const Grid& g, int B, const T* r, T* e, const Coef<T>* coef,
                               bool exact, const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_jacobi_zero<T><<<point_grid(g, B), dim3(32, 8), 0, st>>>(g, r, e, coef, exact ? 1 : 0,
                                                              active);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, int B, const T* rr, T* bc,
                            const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_restrict<T><<<point_grid(gc, B), dim3(32, 8), 0, st>>>(gf, gc, rr, bc, active);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(const Grid& gc, const Grid& gf, int B, const T* ec,
                               long long ec_stride, T* uf, long long uf_stride,
                               const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  k_prolong_add<T><<<point_grid(gf, B), dim3(32, 8), 0, st>>>(gc, gf, ec, ec_stride, uf,
                                                              uf_stride, active);
  count_launch();
  return cudaGetLastError();
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
  template cudaError_t launch_resid64<T>(int, const Grid&, int, const double*, long long,      \
                                         const double*, long long, const Coef<double>*, T*, T*, \
                                         const Coef<T>*, unsigned long long*, const int*, Shape, \
                                         cudaStream_t);                                         \
  template cudaError_t launch_jacobi<T>(int, const Grid&, int, const T*, const T*, T*, double*, \
                                        long long, const Coef<T>*, const int*, Shape,          \
                                        cudaStream_t);                                          \
  template cudaError_t launch_resid<T>(int, const Grid&, int, const T*, const T*, T*,          \
                                       const Coef<T>*, const int*, Shape, cudaStream_t);        \
  template cudaError_t launch_jacobi_zero<T>(const Grid&, int, const T*, T*, const Coef<T>*,   \
                                             bool, const int*, cudaStream_t);                   \
  template cudaError_t launch_restrict<T>(const Grid&, const Grid&, int, const T*, T*,         \
                                          const int*, cudaStream_t);                            \
  template cudaError_t launch_prolong_add<T>(const Grid&, const Grid&, int, const T*, long long,\
                                             T*, long long, const int*, cudaStream_t);          \
  template cudaError_t launch_update<T>(const Grid&, int, const T*, double*, long long,        \
                                        const int*, cudaStream_t);
H3D_INST(double)
H3D_INST(float)
#undef H3D_INST

}  // namespace h3d
