// mg_kernels.cu -- point-parallel multigrid and layout kernels (Sec. 1.2):
// Jacobi from a zero initial guess and the exact one-unknown solve, full
// weighting restriction, trilinear prolongation, the FP64 update, max-norms
// and the dense <-> pitched copies.  One thread per grid point of one item;
// blockIdx.z = item * N + plane.  (The stencil kernels are in
// stencil_kernels.cu.)
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
