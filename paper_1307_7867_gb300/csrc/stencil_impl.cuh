// stencil_impl.cuh -- the 7-point, 13-point (wide) and 19-point (compact)
// stencil kernels of the spatial operator (Sec. 1, method of lines) and of the
// multigrid smoother and residuals (Sec. 1.2), templated on the storage type
// and stencil order, with their launcher templates; stencil_f64.cu and
// stencil_f32.cu instantiate them.
//
// The drivers share one operator interface:
//  * k_tile (grids with N >= 32): a block owns a 32 x TY tile of x-y points
//    and marches along z through a chunk of planes.  The planes it needs
//    (z-R .. z+R, R = 1 or 2) live in a shared-memory ring that cp.async
//    fills D planes ahead in 16-byte chunks, so HBM streams while the block
//    computes; every neighbour is read from shared memory and each thread
//    computes RY rows (independent FP64 chains for the FP64 pipe).  Cells
//    outside the domain are never loaded: the few points next to a boundary
//    replace those neighbours in registers (fix_axis).
//  * k_tile4 (FP32 Jacobi and residual): as k_tile with four x points per
//    thread and 16-byte shared and global accesses.
//  * k_zq4 / k_zq4p (FP32 Jacobi and residual, 7-point and wide): as k_tile4
//    with each thread's own points of the planes k-R .. k+R in a register
//    queue; planes by cp.async or TMA (mbarrier per ring slot), k_zq4p as a
//    producer/consumer pipeline without block barriers.
//  * k_zmarch (small grids): one (x, y) column per thread, z-neighbours in a
//    register queue, x/y neighbours through L1.
// Boundary rule of every stencil read: indices -1 and N are the Dirichlet
// zeros; the wide stencil's ghosts -2 and N+1 are -u(0) and -u(N-1) (odd
// reflection).
//
// Operator interface: src(b) is the field whose stencil is taken, init(b)
// loads per-item coefficients, load(b, idx) the per-point extra operands
// (issued before the plane barrier), apply(b, idx, u, s1, s2, ex) produces the
// outputs from the centre u, the sum s1 of the 6 nearest and s2 of the 6
// second neighbours, and returns the value whose max |.| is accumulated when
// the launch asks for a norm.
#pragma once
#include <cuda.h>  // CUtensorMap (the tensor map of the TMA loader)
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "kernels.cuh"

namespace h3d {
namespace {

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Value at (i, j, k) under the boundary rule, for indices in [-2, N+1].
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

// The boundary rule for the neighbours, along one axis, of a point at
// coordinate p of that axis (the tiled kernels never load cells outside the
// domain; their ring slots hold stale data and are replaced here): indices -1
// and N read 0, the wide stencil's ghosts -2 and N+1 read minus the point
// itself (they occur only for p = 0 and p = N - 1).
template <typename T, int R>
__device__ __forceinline__ void fix_axis(int p, int N, T c, T& m1, T& p1, T& m2, T& p2) {
  if (p == 0) m1 = T(0);
  if (p == N - 1) p1 = T(0);
  if (R == 2) {
    if (p == 0) m2 = -c;
    else if (p == 1) m2 = T(0);
    if (p == N - 1) p2 = -c;
    else if (p == N - 2) p2 = T(0);
  }
}

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

__device__ __forceinline__ void cp_async16(unsigned s, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// mbarrier and TMA (tensor memory access) primitives of the FP32 plane loader.
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for phase `parity` of the barrier to complete; gives up (false) after
// about one second of SM clock cycles, so that a lost copy cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}
// Orders this thread's earlier shared-memory accesses before later copies of
// the async proxy (TMA) into the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// One box of a 4-D tensor map (x, y, z, item) into shared memory, completing
// `bytes` on the barrier.  x must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int x, int y, int z,
                                            int b, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(b), "r"(bar)
      : "memory");
}

template <typename T, int ORDER>
__host__ __device__ __forceinline__ T combine(T s1, T s2) {
  if (ORDER == 2) return s1;
  return fma(T(16), s1, -s2);
}

// b - A u at one point from the centre c and the neighbour sums s1, s2 (for
// the compact stencil: faces and edges, A u = d c - e s1 - e2 s2).
template <typename T, int ORDER>
__device__ __forceinline__ T a_res(T d, T e, T e2, T c, T s1, T s2, T b) {
  if (ORDER == kCompact) return fma(-d, c, fma(e, s1, fma(e2, s2, b)));
  return fma(-d, c, fma(e, combine<T, ORDER>(s1, s2), b));
}

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------

// F = alpha_b L u (and, when ADD, the next substep's rhs add_dst = u + add_src).
// Compact stencil: F = alpha_b (-24 u + 2 S1 + S2) with alpha = nu / (6 h^2);
// the weighted field W u = (6 u + S1) / 12 is written to wu (when given) and
// replaces u in the rhs, add_dst = W u + add_src.
// Operators take 32-bit offsets within the item (fields are < 2^31 elements);
// init(b) resolves the item's base pointers once.  Optional outputs are
// template parameters so that unused FP64 work is not executed.
template <int ORDER, bool ADD>
struct OpLap {
  using T = double;
  struct Ex { double add; };
  const double* u; long long us;
  double* out; long long os;
  const double* alpha;
  const double* add_src; double* add_dst; long long as;
  double a;
  double* o_;
  const double* as_;
  double* ad_;
  double* wu;  // compact stencil: optional W u output, stride us
  double* wu_;
  __device__ const double* src(int b) const { return u + b * us; }
  __device__ void init(int b) {
    a = alpha[b];
    o_ = out + b * os;
    if (ADD) {
      as_ = add_src + b * as;
      ad_ = add_dst + b * as;
    }
    if (ORDER == kCompact) wu_ = wu ? wu + b * us : nullptr;
  }
  __device__ Ex load(int idx) const {
    Ex x;
    if (ADD) x.add = as_[idx];
    return x;
  }
  __device__ double apply(int idx, double c, double s1, double s2, const Ex& ex) {
    if (ORDER == kCompact) {
      o_[idx] = a * fma(-24.0, c, fma(2.0, s1, s2));
      const double w = fma(6.0, c, s1) * (1.0 / 12.0);
      if (wu_) wu_[idx] = w;
      if (ADD) ad_[idx] = w + ex.add;
      return 0.0;
    }
    double L = ORDER == 2 ? fma(-6.0, c, s1) : fma(-90.0, c, fma(16.0, s1, -s2));
    o_[idx] = a * L;
    if (ADD) ad_[idx] = c + ex.add;
    return 0.0;
  }
};

// r = b - A u in FP64 (its max |.| is the stop rule's norm), stored as the
// scaled right-hand side of the error equation b' = wd (TR) r, which is also
// the first Jacobi iterate from zero.
template <int ORDER, typename TR>
struct OpResid64 {
  using T = double;
  struct Ex { double b; };
  const double* u; long long us;
  const double* bb; long long bs;
  const Coef<double>* coef;
  TR* bp; const Coef<TR>* coef_r; long long rs;
  double d, e; TR wd;
  const double* b_;
  TR* bp_;
  double e2;
  __device__ const double* src(int b) const { return u + b * us; }
  __device__ void init(int b) {
    d = coef[b].d;
    e = coef[b].e;
    e2 = coef[b].e2;
    wd = coef_r[b].wd;
    b_ = bb + b * bs;
    bp_ = bp + b * rs;
  }
  __device__ Ex load(int idx) const { return Ex{b_[idx]}; }
  __device__ double apply(int idx, double c, double s1, double s2, const Ex& ex) {
    double res = a_res<double, ORDER>(d, e, e2, c, s1, s2, ex.b);
    bp_[idx] = wd * (TR)res;
    return res;
  }
};

// One damped-Jacobi sweep on the error equation with the scaled right-hand
// side r = b' = wd b: v = e + wd (b - A e) = al e + be S + b' (compact:
// + be2 S2), one multiply-add fewer than forming the residual first; stored
// (UPD = false) or added to the FP64 solution u64 (UPD = true).  UPD is a
// template parameter so that the stored variant contains no FP64 instruction
// at all (a runtime branch is if-converted and would run the FP64 add
// everywhere).
template <typename T, int ORDER>
__host__ __device__ __forceinline__ T jacobi_point(T al, T be, T be2, T c, T s1, T s2, T bp) {
  if (ORDER == kCompact) return fma(al, c, fma(be, s1, fma(be2, s2, bp)));
  return fma(al, c, fma(be, combine<T, ORDER>(s1, s2), bp));
}
// t' = wd (b - A e) = b' - om e + be S (compact: + be2 S2), the residual the
// restriction takes on the scaled levels.
template <typename T, int ORDER>
__host__ __device__ __forceinline__ T resid_point(T om, T be, T be2, T c, T s1, T s2, T bp) {
  if (ORDER == kCompact) return fma(-om, c, fma(be, s1, fma(be2, s2, bp)));
  return fma(-om, c, fma(be, combine<T, ORDER>(s1, s2), bp));
}

template <typename TT, int ORDER, bool UPD>
struct OpJacobi {
  using T = TT;
  struct Ex { T r; double u; };
  const T* e; const T* r; T* out; long long fs;
  double* u64; long long u64s;
  const Coef<T>* coef;
  T al, be, be2;
  const T* r_;
  T* o_;
  double* u_;
  __device__ const T* src(int b) const { return e + b * fs; }
  __host__ __device__ const T* src_base() const { return e; }
  __host__ __device__ long long src_stride() const { return fs; }
  __device__ void init(int b) {
    al = coef[b].al;
    be = coef[b].be;
    be2 = coef[b].be2;
    r_ = r + b * fs;
    if (UPD) u_ = u64 + b * u64s;
    else o_ = out + b * fs;
  }
  __device__ Ex load(int idx) const {
    Ex x;
    x.r = r_[idx];
    if (UPD) x.u = u_[idx];
    return x;
  }
  __device__ double apply(int idx, T c, T s1, T s2, const Ex& ex) {
    T v = jacobi_point<T, ORDER>(al, be, be2, c, s1, s2, ex.r);
    if (UPD) u_[idx] = ex.u + (double)v;
    else o_[idx] = v;
    return 0.0;
  }
  // Four consecutive x points (FP32 storage, k_tile4): idx is a multiple of
  // 4, n >= 1 of the four are inside the grid.  Same arithmetic per point as
  // apply().
  static constexpr bool kVec4 = sizeof(TT) == 4;
  // registers k_tile4 keeps without spilling
  static constexpr int kRegFloor = ORDER == kCompact ? 128 : UPD ? 96 : 64;
  struct Ex4 { float4 r; double2 u01, u23; };
  __device__ Ex4 load4(int idx) const {
    Ex4 x;
    x.r = *reinterpret_cast<const float4*>(r_ + idx);
    if (UPD) {
      x.u01 = *reinterpret_cast<const double2*>(u_ + idx);
      x.u23 = *reinterpret_cast<const double2*>(u_ + idx + 2);
    }
    return x;
  }
  __device__ void apply4(int idx, int n, const float (&c)[4], const float (&s1)[4],
                         const float (&s2)[4], const Ex4& ex) {
    const float rr[4] = {ex.r.x, ex.r.y, ex.r.z, ex.r.w};
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = jacobi_point<float, ORDER>(al, be, be2, c[q], s1[q], s2[q], rr[q]);
    if (UPD) {
      const double w[4] = {ex.u01.x + (double)v[0], ex.u01.y + (double)v[1],
                           ex.u23.x + (double)v[2], ex.u23.y + (double)v[3]};
      if (n >= 4) {
        *reinterpret_cast<double2*>(u_ + idx) = make_double2(w[0], w[1]);
        *reinterpret_cast<double2*>(u_ + idx + 2) = make_double2(w[2], w[3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < n) u_[idx + q] = w[q];
      }
    } else if (n >= 4) {
      *reinterpret_cast<float4*>(o_ + idx) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < n) o_[idx + q] = v[q];
    }
  }
};

// rr = t' = wd (b - A e) from the scaled right-hand side r = b'
template <typename TT, int ORDER>
struct OpResid {
  using T = TT;
  struct Ex { T r; };
  const T* e; const T* r; T* rr; long long fs;
  const Coef<T>* coef;
  T om, be;
  const T* r_;
  T* o_;
  T be2;
  __device__ const T* src(int b) const { return e + b * fs; }
  __host__ __device__ const T* src_base() const { return e; }
  __host__ __device__ long long src_stride() const { return fs; }
  __device__ void init(int b) {
    om = coef[b].om;
    be = coef[b].be;
    be2 = coef[b].be2;
    r_ = r + b * fs;
    o_ = rr + b * fs;
  }
  __device__ Ex load(int idx) const { return Ex{r_[idx]}; }
  __device__ double apply(int idx, T c, T s1, T s2, const Ex& ex) {
    o_[idx] = resid_point<T, ORDER>(om, be, be2, c, s1, s2, ex.r);
    return 0.0;
  }
  static constexpr bool kVec4 = sizeof(TT) == 4;
  static constexpr int kRegFloor = ORDER == kCompact ? 128 : 64;
  struct Ex4 { float4 r; };
  __device__ Ex4 load4(int idx) const { return Ex4{*reinterpret_cast<const float4*>(r_ + idx)}; }
  __device__ void apply4(int idx, int n, const float (&c)[4], const float (&s1)[4],
                         const float (&s2)[4], const Ex4& ex) {
    const float rr[4] = {ex.r.x, ex.r.y, ex.r.z, ex.r.w};
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = resid_point<float, ORDER>(om, be, be2, c[q], s1[q], s2[q], rr[q]);
    if (n >= 4) {
      *reinterpret_cast<float4*>(o_ + idx) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < n) o_[idx + q] = v[q];
    }
  }
};

// ---------------------------------------------------------------------------
// drivers
// ---------------------------------------------------------------------------

template <int ORDER, bool NORM, typename Op>
__global__ void __launch_bounds__(128) k_zmarch(Grid g, int nzc, int zc, const int* active,
                                                unsigned long long* norm_bits, Op op) {
  using T = typename Op::T;
  constexpr int R = ORDER == 4 ? 2 : 1;
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
    const int plane = (int)g.plane;
    int idx = z0 * plane + j * g.px + i;
    for (int k = z0; k < z1; ++k, idx += plane) {
      typename Op::Ex ex = o.load(idx);
      T s1 = ((at(u, g, i - 1, j, k) + at(u, g, i + 1, j, k)) +
              (at(u, g, i, j - 1, k) + at(u, g, i, j + 1, k))) + (q[R - 1] + q[R + 1]);
      T s2 = T(0);
      if (R == 2)
        s2 = ((at(u, g, i - 2, j, k) + at(u, g, i + 2, j, k)) +
              (at(u, g, i, j - 2, k) + at(u, g, i, j + 2, k))) + (q[0] + q[2 * R]);
      if (ORDER == kCompact)  // the 12 edge neighbours, grouped xy, xz, yz
        s2 = (((at(u, g, i - 1, j - 1, k) + at(u, g, i + 1, j - 1, k)) +
               (at(u, g, i - 1, j + 1, k) + at(u, g, i + 1, j + 1, k))) +
              ((at(u, g, i - 1, j, k - 1) + at(u, g, i + 1, j, k - 1)) +
               (at(u, g, i - 1, j, k + 1) + at(u, g, i + 1, j, k + 1)))) +
             ((at(u, g, i, j - 1, k - 1) + at(u, g, i, j + 1, k - 1)) +
              (at(u, g, i, j - 1, k + 1) + at(u, g, i, j + 1, k + 1)));
      double rv = o.apply(idx, q[R], s1, s2, ex);
      if (NORM) {
        unsigned long long bits = abs_bits(rv);
        mx = bits > mx ? bits : mx;
      }
#pragma unroll
      for (int d = 0; d < 2 * R; ++d) q[d] = q[d + 1];
      if (k + 1 < z1) q[2 * R] = at(u, g, i, j, k + R + 1);
    }
  }
  if (NORM) warp_max_to(mx, norm_bits + b);
}

template <typename T>
__host__ __device__ constexpr int halo_x() { return 16 / (int)sizeof(T); }

// Ring of 2R + D + 1 planes: the D planes in flight, the 2R + 1 planes being
// read, and the slot refilled during the current plane.
template <typename T, int ORDER, int TYT, int RY, int D>
constexpr int tile_smem_bytes() {
  return (2 * (ORDER == 4 ? 2 : 1) + D + 1) * (TYT * RY + 2 * (ORDER == 4 ? 2 : 1)) *
         (32 + 2 * halo_x<T>()) * (int)sizeof(T);
}

__device__ __forceinline__ int ring_next(int s, int nb) { return s + 1 == nb ? 0 : s + 1; }
__device__ __forceinline__ int ring_prev(int s, int nb) { return s == 0 ? nb - 1 : s - 1; }

template <int ORDER, int TYT, int RY, int D, bool NORM, typename Op>
__global__ void __launch_bounds__(32 * TYT) k_tile(Grid g, int nzc, int zc, const int* active,
                                                   unsigned long long* norm_bits, Op op) {
  using T = typename Op::T;
  constexpr int R = ORDER == 4 ? 2 : 1;
  constexpr int TX = 32, TY = TYT * RY;
  constexpr int XH = halo_x<T>();
  constexpr int SX = TX + 2 * XH, SY = TY + 2 * R, NB = 2 * R + D + 1;
  constexpr int CH = SX / XH;  // 16-byte chunks per shared row
  constexpr int NT = 32 * TYT;
  constexpr int PS = SY * SX;  // elements per shared plane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);
  const int b = blockIdx.z / nzc;
  if (active && !active[b]) return;  // uniform over the block
  const int N = g.N;
  const int plane = (int)g.plane;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = (blockIdx.z - b * nzc) * zc, z1 = min(N, z0 + zc);
  Op o = op;
  o.init(b);
  const T* __restrict__ u = o.src(b);
  const int tid = threadIdx.y * 32 + threadIdx.x;

  // Plane z into ring slot `slot` by 16-byte cp.async chunks.  Only chunks of
  // rows and planes inside the domain whose 16 bytes lie within the allocated
  // row (x < px) are copied; the stencil replaces every neighbour outside the
  // domain by the boundary rule (fix_axis), so nothing else is ever read.
  // A thread's chunks are the same for every plane: offsets computed once.
  constexpr int NCH = (SY * CH + NT - 1) / NT;
  int soff[NCH], goff[NCH];
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int c = tid + q * NT;
    const int ry = c / CH, cx = c - ry * CH;
    const int cgy = y0 - R + ry, cgx = x0 - XH + cx * XH;
    const bool ok = c < SY * CH && cgy >= 0 && cgy < N && cgx >= 0 && cgx + XH <= g.px;
    soff[q] = ok ? ry * SX + cx * XH : -1;
    goff[q] = cgy * g.px + cgx;
  }
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  auto issue = [&](int z, int slot) {
    if (z >= 0 && z < N && z <= z1 - 1 + R) {
      const unsigned dst = ring_s + (unsigned)(slot * PS) * (unsigned)sizeof(T);
      const T* uz = u + z * plane;
#pragma unroll
      for (int q = 0; q < NCH; ++q)
        if (soff[q] >= 0) cp_async16(dst + (unsigned)soff[q] * (unsigned)sizeof(T), uz + goff[q]);
    }
    cp_async_commit();
  };

#pragma unroll 1
  for (int q = 0; q < 2 * R + D; ++q) issue(z0 - R + q, q);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = x0 + tx;
  const int jb = y0 + ty * RY;
  const int sbase = (R + ty * RY) * SX + XH + tx;
  const bool xedge = i < R || i >= N - R;
  int idx0 = z0 * plane + jb * g.px + i;
  int cs = R;                // ring slot of plane k
  int fs_ = 2 * R + D;       // slot that receives plane k + R + D
  unsigned long long mx = 0ull;
  for (int k = z0; k < z1; ++k, idx0 += plane) {
    typename Op::Ex ex[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r)
      if (i < N && jb + r < N) ex[r] = o.load(idx0 + r * g.px);
    cp_async_wait<D - 1>();
    // one barrier per plane: after it every thread has finished plane k - 1,
    // so the slot of plane k - R - 1 can be refilled while plane k is computed
    __syncthreads();
    issue(k + R + D, fs_);
    fs_ = ring_next(fs_, NB);
    const int sm1 = ring_prev(cs, NB), sp1 = ring_next(cs, NB);
    const int sm2 = ring_prev(sm1, NB), sp2 = ring_next(sp1, NB);
    const T* P0 = ring + cs * PS + sbase;
    const T* Pm1 = ring + sm1 * PS + sbase;
    const T* Pp1 = ring + sp1 * PS + sbase;
    const T* Pm2 = ring + sm2 * PS + sbase;
    const T* Pp2 = ring + sp2 * PS + sbase;
    const bool zedge = k < R || k >= N - R;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const int o0 = r * SX;
      const int j = jb + r;
      const T c = P0[o0];
      T xm1 = P0[o0 - 1], xp1 = P0[o0 + 1], ym1 = P0[o0 - SX], yp1 = P0[o0 + SX];
      T zm1 = Pm1[o0], zp1 = Pp1[o0];
      T xm2 = T(0), xp2 = T(0), ym2 = T(0), yp2 = T(0), zm2 = T(0), zp2 = T(0);
      if (R == 2) {
        xm2 = P0[o0 - 2]; xp2 = P0[o0 + 2]; ym2 = P0[o0 - 2 * SX]; yp2 = P0[o0 + 2 * SX];
        zm2 = Pm2[o0]; zp2 = Pp2[o0];
      }
      const bool yedge = j < R || j >= N - R;
      if (xedge) fix_axis<T, R>(i, N, c, xm1, xp1, xm2, xp2);
      if (yedge) fix_axis<T, R>(j, N, c, ym1, yp1, ym2, yp2);
      if (zedge) fix_axis<T, R>(k, N, c, zm1, zp1, zm2, zp2);
      T s1 = ((xm1 + xp1) + (ym1 + yp1)) + (zm1 + zp1);
      T s2 = T(0);
      if (R == 2) s2 = ((xm2 + xp2) + (ym2 + yp2)) + (zm2 + zp2);
      if (ORDER == kCompact) {
        // edge neighbours e<axes>_<sign of first axis><sign of second axis>
        T exy_mm = P0[o0 - SX - 1], exy_pm = P0[o0 - SX + 1];
        T exy_mp = P0[o0 + SX - 1], exy_pp = P0[o0 + SX + 1];
        T exz_mm = Pm1[o0 - 1], exz_pm = Pm1[o0 + 1], exz_mp = Pp1[o0 - 1], exz_pp = Pp1[o0 + 1];
        T eyz_mm = Pm1[o0 - SX], eyz_pm = Pm1[o0 + SX], eyz_mp = Pp1[o0 - SX], eyz_pp = Pp1[o0 + SX];
        if (xedge) {
          if (i == 0) exy_mm = exy_mp = exz_mm = exz_mp = T(0);
          if (i == N - 1) exy_pm = exy_pp = exz_pm = exz_pp = T(0);
        }
        if (yedge) {
          if (j == 0) exy_mm = exy_pm = eyz_mm = eyz_mp = T(0);
          if (j == N - 1) exy_mp = exy_pp = eyz_pm = eyz_pp = T(0);
        }
        if (zedge) {
          if (k == 0) exz_mm = exz_pm = eyz_mm = eyz_pm = T(0);
          if (k == N - 1) exz_mp = exz_pp = eyz_mp = eyz_pp = T(0);
        }
        s2 = (((exy_mm + exy_pm) + (exy_mp + exy_pp)) + ((exz_mm + exz_pm) + (exz_mp + exz_pp))) +
             ((eyz_mm + eyz_pm) + (eyz_mp + eyz_pp));
      }
      if (i < N && j < N) {
        double rv = o.apply(idx0 + r * g.px, c, s1, s2, ex[r]);
        if (NORM) {
          unsigned long long bits = abs_bits(rv);
          mx = bits > mx ? bits : mx;
        }
      }
    }
    cs = sp1;
  }
  cp_async_wait<0>();
  if (NORM) warp_max_to(mx, norm_bits + b);
}

// One tiled launch: TYT warps per block, RY rows per thread, D planes of
// prefetch.  Rings above 48 KB need the shared-memory opt-in (set once).
template <int ORDER, int TYT, int RY, int D, bool NORM, typename Op>
cudaError_t launch_tile(const Grid& g, int B, int nzc, int zc, const int* active,
                        unsigned long long* norm_bits, const Op& op, cudaStream_t st) {
  using T = typename Op::T;
  constexpr int smem = tile_smem_bytes<T, ORDER, TYT, RY, D>();
  if (smem > 48 * 1024) {
    static std::atomic<bool> set{false};  // set once per process (one device)
    if (!set.load()) {
      cudaError_t e = cudaFuncSetAttribute(k_tile<ORDER, TYT, RY, D, NORM, Op>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      set.store(true);
    }
  }
  dim3 blk(32, TYT, 1);
  dim3 grd((g.N + 31) / 32, (g.N + TYT * RY - 1) / (TYT * RY), nzc * B);
  k_tile<ORDER, TYT, RY, D, NORM, Op><<<grd, blk, smem, st>>>(g, nzc, zc, active, norm_bits, op);
  return cudaSuccess;
}

// FP32 tile with four x points per thread: a warp covers 128 consecutive x
// points of one row, so every neighbour read is a 16-byte (centre, y, z) or
// 8-byte (x halo) shared-memory access shared by four points, and the
// per-point loads and stores are float4.  Ring and loader as k_tile (the
// 16-byte x halo is exactly one chunk); the boundary cells of the x and y
// halo are written into the ring instead of being fixed per point.  The sums
// per point are formed in the same order as k_tile and k_zmarch, so the
// results are bitwise identical.
template <int ORDER, int TYT, int RY, int D>
constexpr int tile4_smem() {
  return (2 * (ORDER == 4 ? 2 : 1) + D + 1) * (TYT * RY + 2 * (ORDER == 4 ? 2 : 1)) * (128 + 8) * 4;
}
// Blocks per SM that the ring allows, but no more than keeps the operator's
// register floor (kRegFloor) available: the register cap that keeps them
// resident together.
template <int ORDER, int TYT, int RY, int D, int REGS>
constexpr int tile4_min_blocks() {
  return (232448 / tile4_smem<ORDER, TYT, RY, D>()) < (65536 / (32 * TYT * REGS))
             ? (232448 / tile4_smem<ORDER, TYT, RY, D>())
             : (65536 / (32 * TYT * REGS));
}

template <int ORDER, int TYT, int RY, int D, typename Op>
__global__ void __launch_bounds__(32 * TYT, (tile4_min_blocks<ORDER, TYT, RY, D, Op::kRegFloor>()))
    k_tile4(Grid g, int nzc, int zc, const int* active, Op op) {
  using T = typename Op::T;
  static_assert(sizeof(T) == 4, "k_tile4 is the FP32 path");
  constexpr int R = ORDER == 4 ? 2 : 1;
  constexpr int TX = 128, TY = TYT * RY;
  constexpr int XH = 4;
  constexpr int SX = TX + 2 * XH, SY = TY + 2 * R, NB = 2 * R + D + 1;
  constexpr int CH = SX / XH;
  constexpr int NT = 32 * TYT;
  constexpr int PS = SY * SX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* ring = reinterpret_cast<float*>(smem_raw);
  const int b = blockIdx.z / nzc;
  if (active && !active[b]) return;  // uniform over the block
  const int N = g.N;
  const int plane = (int)g.plane;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = (blockIdx.z - b * nzc) * zc, z1 = min(N, z0 + zc);
  Op o = op;
  o.init(b);
  const float* __restrict__ u = o.src(b);
  const int tid = threadIdx.y * 32 + threadIdx.x;

  constexpr int NCH = (SY * CH + NT - 1) / NT;
  int soff[NCH], goff[NCH];
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int c = tid + q * NT;
    const int ry = c / CH, cx = c - ry * CH;
    const int cgy = y0 - R + ry, cgx = x0 - XH + cx * XH;
    const bool ok = c < SY * CH && cgy >= 0 && cgy < N && cgx >= 0 && cgx + XH <= g.px;
    soff[q] = ok ? ry * SX + cx * XH : -1;
    goff[q] = cgy * g.px + cgx;
  }
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  auto issue = [&](int z, int slot) {
    if (z >= 0 && z < N && z <= z1 - 1 + R) {
      const unsigned dst = ring_s + (unsigned)(slot * PS) * 4u;
      const float* uz = u + z * plane;
#pragma unroll
      for (int q = 0; q < NCH; ++q)
        if (soff[q] >= 0) cp_async16(dst + (unsigned)soff[q] * 4u, uz + goff[q]);
    }
    cp_async_commit();
  };

#pragma unroll 1
  for (int q = 0; q < 2 * R + D; ++q) issue(z0 - R + q, q);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = x0 + 4 * tx;
  const int jb = y0 + ty * RY;
  const int sbase = (R + ty * RY) * SX + XH + 4 * tx;
  const int nx = N - i;  // points of the thread's four inside the grid
  // Boundary cells of a plane held in the ring (x and y out of the domain)
  // are written with the boundary rule once the plane has arrived, so the
  // stencil reads them like any neighbour: indices -1 and N are 0, the wide
  // stencil's ghosts -2 and N+1 minus the cell at 0 and N-1.  Corners (out in
  // x and y) are never read by these axis-aligned stencils.
  const int cxN = XH + N - x0;  // ring column of x = N
  const bool xlo = x0 == 0, xhi = cxN < SX;
  const int ryN = N - (y0 - R);  // ring row of y = N
  const bool ylo = y0 < R, yhi = ryN < SY;
  auto fill = [&](int z, int slot) {
    if (z < 0 || z >= N || !(xlo || xhi || ylo || yhi)) return;
    float* P = ring + slot * PS;
    if (xlo || xhi)
      for (int r = tid; r < SY; r += NT) {
        const int y = y0 - R + r;
        if (y < 0 || y >= N) continue;
        float* row = P + r * SX;
        if (xlo) {
          if (R == 2) row[XH - 2] = -row[XH];
          row[XH - 1] = 0.f;
        }
        if (xhi) {
          if (R == 2 && cxN + 1 < SX) row[cxN + 1] = -row[cxN - 1];
          row[cxN] = 0.f;
        }
      }
    if (ylo || yhi)
      for (int c = tid; c < SX; c += NT) {
        if (ylo) {  // rows y = -1 and -2 sit at ring rows R - 1 and R - 2
          if (R == 2) P[c] = -P[R * SX + c];
          P[(R - 1) * SX + c] = 0.f;
        }
        if (yhi) {
          if (R == 2 && ryN + 1 < SY) P[(ryN + 1) * SX + c] = -P[(ryN - 1) * SX + c];
          P[ryN * SX + c] = 0.f;
        }
      }
  };
  int idx0 = z0 * plane + jb * g.px + i;
  int cs = R;
  int fs_ = 2 * R + D;
  for (int k = z0; k < z1; ++k, idx0 += plane) {
    typename Op::Ex4 ex[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r)
      if (nx > 0 && jb + r < N) ex[r] = o.load4(idx0 + r * g.px);
    cp_async_wait<D - 1>();
    __syncthreads();
    // planes up to k + R have arrived: complete the boundary cells of plane
    // k + R (read as a centre plane R iterations later, after a barrier); the
    // first iteration completes planes k - R .. k + R (slots 0 .. 2R) and
    // waits for that.  The compact stencil also reads the boundary cells of
    // the planes k -+ 1 (edge neighbours), so it waits after every fill.
    if (k == z0) {
      for (int q = 0; q <= 2 * R; ++q) fill(z0 - R + q, q);
      __syncthreads();
    } else {
      int sl = cs;
      for (int q = 0; q < R; ++q) sl = ring_next(sl, NB);
      fill(k + R, sl);
      if (ORDER == kCompact && (xlo || xhi || ylo || yhi)) __syncthreads();  // uniform
    }
    issue(k + R + D, fs_);
    fs_ = ring_next(fs_, NB);
    const int sm1 = ring_prev(cs, NB), sp1 = ring_next(cs, NB);
    const int sm2 = ring_prev(sm1, NB), sp2 = ring_next(sp1, NB);
    const float* P0 = ring + cs * PS + sbase;
    const float* Pm1 = ring + sm1 * PS + sbase;
    const float* Pp1 = ring + sp1 * PS + sbase;
    const float* Pm2 = ring + sm2 * PS + sbase;
    const float* Pp2 = ring + sp2 * PS + sbase;
    // centre float4 of rows jb - R .. jb + RY - 1 + R in plane k
    float4 col[RY + 2 * R];
#pragma unroll
    for (int q = 0; q < RY + 2 * R; ++q) col[q] = *reinterpret_cast<const float4*>(P0 + (q - R) * SX);
    const bool zedge = k < R || k >= N - R;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const int o0 = r * SX;
      const int j = jb + r;
      const float4 cc = col[r + R];
      const float c[4] = {cc.x, cc.y, cc.z, cc.w};
      // x: a[2..3] = x-2, x-1; a[4..7] = the four points; a[8..9] = x+4, x+5
      float a[10];
      if (R == 2) {
        const float2 lh = *reinterpret_cast<const float2*>(P0 + o0 - 2);
        const float2 rh = *reinterpret_cast<const float2*>(P0 + o0 + 4);
        a[2] = lh.x; a[3] = lh.y; a[8] = rh.x; a[9] = rh.y;
      } else {
        a[2] = 0.f; a[3] = P0[o0 - 1]; a[8] = P0[o0 + 4]; a[9] = 0.f;
      }
      a[4] = c[0]; a[5] = c[1]; a[6] = c[2]; a[7] = c[3];
      const float4 ym1 = col[r + R - 1], yp1 = col[r + R + 1];
      const float4 zm1 = *reinterpret_cast<const float4*>(Pm1 + o0);
      const float4 zp1 = *reinterpret_cast<const float4*>(Pp1 + o0);
      float xm1v[4], xp1v[4], ym1v[4] = {ym1.x, ym1.y, ym1.z, ym1.w}, yp1v[4] = {yp1.x, yp1.y, yp1.z, yp1.w};
      float zm1v[4] = {zm1.x, zm1.y, zm1.z, zm1.w}, zp1v[4] = {zp1.x, zp1.y, zp1.z, zp1.w};
      float xm2v[4] = {0.f, 0.f, 0.f, 0.f}, xp2v[4] = {0.f, 0.f, 0.f, 0.f};
      float ym2v[4] = {0.f, 0.f, 0.f, 0.f}, yp2v[4] = {0.f, 0.f, 0.f, 0.f};
      float zm2v[4] = {0.f, 0.f, 0.f, 0.f}, zp2v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xm1v[q] = a[3 + q];
        xp1v[q] = a[5 + q];
      }
      if (R == 2) {
        const float4 ym2 = col[r + R - 2], yp2 = col[r + R + 2];
        const float4 zm2 = *reinterpret_cast<const float4*>(Pm2 + o0);
        const float4 zp2 = *reinterpret_cast<const float4*>(Pp2 + o0);
        ym2v[0] = ym2.x; ym2v[1] = ym2.y; ym2v[2] = ym2.z; ym2v[3] = ym2.w;
        yp2v[0] = yp2.x; yp2v[1] = yp2.y; yp2v[2] = yp2.z; yp2v[3] = yp2.w;
        zm2v[0] = zm2.x; zm2v[1] = zm2.y; zm2v[2] = zm2.z; zm2v[3] = zm2.w;
        zp2v[0] = zp2.x; zp2v[1] = zp2.y; zp2v[2] = zp2.z; zp2v[3] = zp2.w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xm2v[q] = a[2 + q];
          xp2v[q] = a[6 + q];
        }
      }
      if (zedge) {
#pragma unroll
        for (int q = 0; q < 4; ++q) fix_axis<float, R>(k, N, c[q], zm1v[q], zp1v[q], zm2v[q], zp2v[q]);
      }
      float s1[4], s2[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s1[q] = ((xm1v[q] + xp1v[q]) + (ym1v[q] + yp1v[q])) + (zm1v[q] + zp1v[q]);
        s2[q] = R == 2 ? ((xm2v[q] + xp2v[q]) + (ym2v[q] + yp2v[q])) + (zm2v[q] + zp2v[q]) : 0.f;
      }
      if (ORDER == kCompact) {
        // the 12 edge neighbours: x windows (x-1 .. x+4) of rows y-1 and y+1
        // in plane k and of row y in planes k-1 and k+1, and the centres of
        // rows y-1 and y+1 in planes k-1 and k+1; boundary cells of planes in
        // the domain are in the ring, planes outside are zeroed here
        float bm[6], bp[6], zmw[6], zpw[6];
        bm[0] = P0[o0 - SX - 1]; bm[5] = P0[o0 - SX + 4];
        bp[0] = P0[o0 + SX - 1]; bp[5] = P0[o0 + SX + 4];
        zmw[0] = Pm1[o0 - 1]; zmw[5] = Pm1[o0 + 4];
        zpw[0] = Pp1[o0 - 1]; zpw[5] = Pp1[o0 + 4];
        bm[1] = ym1.x; bm[2] = ym1.y; bm[3] = ym1.z; bm[4] = ym1.w;
        bp[1] = yp1.x; bp[2] = yp1.y; bp[3] = yp1.z; bp[4] = yp1.w;
        zmw[1] = zm1.x; zmw[2] = zm1.y; zmw[3] = zm1.z; zmw[4] = zm1.w;
        zpw[1] = zp1.x; zpw[2] = zp1.y; zpw[3] = zp1.z; zpw[4] = zp1.w;
        const float4 yzmm = *reinterpret_cast<const float4*>(Pm1 + o0 - SX);
        const float4 yzpm = *reinterpret_cast<const float4*>(Pm1 + o0 + SX);
        const float4 yzmp = *reinterpret_cast<const float4*>(Pp1 + o0 - SX);
        const float4 yzpp = *reinterpret_cast<const float4*>(Pp1 + o0 + SX);
        float eyz_mm[4] = {yzmm.x, yzmm.y, yzmm.z, yzmm.w}, eyz_pm[4] = {yzpm.x, yzpm.y, yzpm.z, yzpm.w};
        float eyz_mp[4] = {yzmp.x, yzmp.y, yzmp.z, yzmp.w}, eyz_pp[4] = {yzpp.x, yzpp.y, yzpp.z, yzpp.w};
        if (zedge) {
          if (k == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) zmw[q] = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) eyz_mm[q] = eyz_pm[q] = 0.f;
          }
          if (k == N - 1) {
#pragma unroll
            for (int q = 0; q < 6; ++q) zpw[q] = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) eyz_mp[q] = eyz_pp[q] = 0.f;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          s2[q] = (((bm[q] + bm[q + 2]) + (bp[q] + bp[q + 2])) + ((zmw[q] + zmw[q + 2]) + (zpw[q] + zpw[q + 2]))) +
                  ((eyz_mm[q] + eyz_pm[q]) + (eyz_mp[q] + eyz_pp[q]));
      }
      if (nx > 0 && j < N) o.apply4(idx0 + r * g.px, nx, c, s1, s2, ex[r]);
    }
    cs = sp1;
  }
  cp_async_wait<0>();
}

template <int ORDER, int TYT, int RY, int D, typename Op>
cudaError_t launch_tile4(const Grid& g, int B, int nzc, int zc, const int* active, const Op& op,
                         cudaStream_t st) {
  constexpr int smem = tile4_smem<ORDER, TYT, RY, D>();
  if (smem > 48 * 1024) {
    static std::atomic<bool> set{false};  // set once per process (one device)
    if (!set.load()) {
      cudaError_t e = cudaFuncSetAttribute(k_tile4<ORDER, TYT, RY, D, Op>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      set.store(true);
    }
  }
  dim3 blk(32, TYT, 1);
  dim3 grd((g.N + 127) / 128, (g.N + TYT * RY - 1) / (TYT * RY), nzc * B);
  k_tile4<ORDER, TYT, RY, D, Op><<<grd, blk, smem, st>>>(g, nzc, zc, active, op);
  return cudaSuccess;
}

// FP32 tile with the z neighbours in registers (7-point and wide stencils):
// as k_tile4 (a warp covers 128 consecutive x points of one row, four per
// thread, float4 accesses), but each thread keeps its own four points of the
// planes k-R .. k+R in a register queue, so that the ring in shared memory
// only has to hold the plane being computed (for the x and y neighbours), the
// planes up to k+R (whose own points enter the queue) and the D planes in
// flight: R + D + 1 planes instead of 2R + D + 1, and four fewer 16-byte
// shared reads per row.  The ring size is a multiple of the queue length
// 2R + 1 and the z loop is unrolled by it, so ring slots and queue entries
// are compile-time registers.  Boundary cells in x and y are written into
// the ring as in k_tile4, those in z replaced in registers.  Planes arrive
// either by
// 16-byte cp.async copies of every thread (TMA = 0) or as one TMA box per
// plane issued by one thread, completing on an mbarrier per ring slot
// (TMA = 1; waits bounded, a lost copy sets g_zq_timeout and the block
// returns).  The per-point sums are formed as in k_tile4, so the results are
// bitwise identical.
__device__ int g_zq_timeout;

template <int ORDER, int DEEP>
__host__ __device__ constexpr int zq_depth() {  // prefetch depth: R + D + 1 must be a multiple of 2R + 1
  return ORDER == 4 ? (DEEP ? 7 : 2) : (DEEP ? 7 : 4);
}
template <int ORDER, int TYT>
__host__ __device__ constexpr int zq_slot_floats() {  // one plane of the ring, 128-byte aligned
  return ((TYT + 2 * (ORDER == 4 ? 2 : 1)) * (128 + 8) + 31) / 32 * 32;
}
template <int ORDER, int TYT, int DEEP>
__host__ __device__ constexpr int zq_smem() {
  return ((ORDER == 4 ? 2 : 1) + zq_depth<ORDER, DEEP>() + 1) * zq_slot_floats<ORDER, TYT>() * 4 + 128;
}
template <int ORDER, int TYT, int DEEP, int REGS>
constexpr int zq_min_blocks() {
  return (232448 / zq_smem<ORDER, TYT, DEEP>()) < (65536 / (32 * TYT * REGS))
             ? (232448 / zq_smem<ORDER, TYT, DEEP>())
             : (65536 / (32 * TYT * REGS));
}
// registers the queue kernel keeps without spilling: the wide stencil's
// queue and y neighbours take 16 more than k_tile4's floor
template <int ORDER, int TMA, typename Op>
constexpr int zq_reg_floor() {
  return ORDER != 4 ? Op::kRegFloor : Op::kRegFloor >= 80 ? Op::kRegFloor : 80;
}

template <int ORDER, int TYT, int DEEP, int TMA, typename Op>
__global__ void __launch_bounds__(32 * TYT, (zq_min_blocks<ORDER, TYT, DEEP, zq_reg_floor<ORDER, TMA, Op>()>()))
    k_zq4(Grid g, int nzc, int zc, const int* active, Op op, const __grid_constant__ CUtensorMap tmap) {
  using T = typename Op::T;
  static_assert(sizeof(T) == 4, "k_zq4 is the FP32 path");
  static_assert(ORDER == 2 || ORDER == 4, "k_zq4: 7-point and wide stencils");
  constexpr int R = ORDER == 4 ? 2 : 1;
  constexpr int D = zq_depth<ORDER, DEEP>();
  constexpr int NB = R + D + 1;  // ring slots
  constexpr int QL = 2 * R + 1;  // queue length
  static_assert(NB % QL == 0, "ring size must be a multiple of the queue length");
  constexpr int TX = 128, TY = TYT;
  constexpr int XH = 4;
  constexpr int SX = TX + 2 * XH, SY = TY + 2 * R;
  constexpr int CH = SX / XH;
  constexpr int NT = 32 * TYT;
  constexpr int PS = zq_slot_floats<ORDER, TYT>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[NB];
  float* ring = reinterpret_cast<float*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int b = blockIdx.z / nzc;
  if (active && !active[b]) return;  // uniform over the block
  const int N = g.N;
  const int plane = (int)g.plane;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = (blockIdx.z - b * nzc) * zc, z1 = min(N, z0 + zc);
  Op o = op;
  o.init(b);
  const float* __restrict__ u = o.src(b);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  const unsigned bar_s = (unsigned)__cvta_generic_to_shared(bars);

  constexpr int NCH = TMA ? 1 : (SY * CH + NT - 1) / NT;
  int soff[NCH], goff[NCH];
  if (!TMA) {
#pragma unroll
    for (int q = 0; q < NCH; ++q) {
      const int c = tid + q * NT;
      const int ry = c / CH, cx = c - ry * CH;
      const int cgy = y0 - R + ry, cgx = x0 - XH + cx * XH;
      const bool ok = c < SY * CH && cgy >= 0 && cgy < N && cgx >= 0 && cgx + XH <= g.px;
      soff[q] = ok ? ry * SX + cx * XH : -1;
      goff[q] = cgy * g.px + cgx;
    }
  } else if (tid == 0) {
#pragma unroll
    for (int q = 0; q < NB; ++q) mbar_init(bar_s + 8u * q, 1);
    mbar_init_fence();
  }
  if (TMA) __syncthreads();
  // plane p lives in slot (p - z0 + R) mod NB.  cp.async: one commit group per
  // plane, empty for planes outside the domain or past the chunk, so that group
  // counts match.  TMA: thread 0 arms the slot's barrier with the box's bytes
  // and issues the box, or only arrives for a plane that is not copied, so that
  // every slot completes one barrier phase per plane it is assigned.
  auto issue = [&](int z, int slot) {
    const bool copy = z >= 0 && z < N && z <= z1 - 1 + R;
    if (TMA) {
      if (tid == 0) {
        const unsigned bar = bar_s + 8u * slot;
        if (copy) {
          fence_proxy_async_smem();
          mbar_expect_tx(bar, (unsigned)(SY * SX * 4));
          tma_load_4d(ring_s + (unsigned)(slot * PS) * 4u, &tmap, x0 - XH, y0 - R, z, b, bar);
        } else {
          mbar_arrive(bar);
        }
      }
    } else {
      if (copy) {
        const unsigned dst = ring_s + (unsigned)(slot * PS) * 4u;
        const float* uz = u + z * plane;
#pragma unroll
        for (int q = 0; q < NCH; ++q)
          if (soff[q] >= 0) cp_async16(dst + (unsigned)soff[q] * 4u, uz + goff[q]);
      }
      cp_async_commit();
    }
  };
  // TMA: waits for plane p (fill number (p - z0 + R) / NB of its slot); false
  // if the copy never completed
  auto arrived = [&](int p, int slot) -> bool {
    if (!TMA) return true;
    const unsigned parity = (unsigned)((p - z0 + R) / NB) & 1u;
    return mbar_wait_bounded(bar_s + 8u * slot, parity);
  };
  // after a lost copy: thread 0 waits (bounded) for every slot's last
  // fill, records the fault, and the whole block returns
  auto give_up = [&](int last_issued) {
    if (tid == 0) {
      atomicExch(&g_zq_timeout, 1);
      for (int p = last_issued; p > last_issued - NB && p >= z0 - R; --p)
        mbar_wait_bounded(bar_s + 8u * ((p - z0 + R) % NB), (unsigned)((p - z0 + R) / NB) & 1u);
    }
  };

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = x0 + 4 * tx;
  const int j = y0 + ty;
  const int sbase = (R + ty) * SX + XH + 4 * tx;
  const int nx = N - i;  // points of the thread's four inside the grid
  auto own = [&](int slot) { return *reinterpret_cast<const float4*>(ring + slot * PS + sbase); };
  // boundary cells of a plane in the ring, as in k_tile4: x and y indices -1
  // and N read 0, the wide stencil's ghosts -2 and N+1 minus the cell at 0
  // and N-1 (corners are never read by these stencils).  With the TMA loader
  // the writing threads then order their writes before the slot's next copy.
  const int cxN = XH + N - x0;
  const bool xlo = x0 == 0, xhi = cxN < SX;
  const int ryN = N - (y0 - R);
  const bool ylo = y0 < R, yhi = ryN < SY;
  const bool edge = xlo || xhi || ylo || yhi;  // the same for the whole block
  auto fill = [&](int z, int slot) {
    if (z < 0 || z >= N || !edge) return;
    float* P = ring + slot * PS;
    if (xlo || xhi)
      for (int r = tid; r < SY; r += NT) {
        const int y = y0 - R + r;
        if (y < 0 || y >= N) continue;
        float* row = P + r * SX;
        if (xlo) {
          if (R == 2) row[XH - 2] = -row[XH];
          row[XH - 1] = 0.f;
        }
        if (xhi) {
          if (R == 2 && cxN + 1 < SX) row[cxN + 1] = -row[cxN - 1];
          row[cxN] = 0.f;
        }
      }
    if (ylo || yhi)
      for (int c = tid; c < SX; c += NT) {
        if (ylo) {
          if (R == 2) P[c] = -P[R * SX + c];
          P[(R - 1) * SX + c] = 0.f;
        }
        if (yhi) {
          if (R == 2 && ryN + 1 < SY) P[(ryN + 1) * SX + c] = -P[(ryN - 1) * SX + c];
          P[ryN * SX + c] = 0.f;
        }
      }
    if (TMA) fence_proxy_async_smem();
  };

  // prologue: the first NB planes (z0-R .. z0+D); the queue takes the own
  // points of z0-R .. z0+R-1; planes z0 .. z0+R get their boundary cells
#pragma unroll 1
  for (int q = 0; q < NB; ++q) issue(z0 - R + q, q);
  if (TMA) {
    bool ok = true;
#pragma unroll
    for (int q = 0; q <= 2 * R; ++q) ok = arrived(z0 - R + q, q) && ok;
    if (__syncthreads_or(!ok)) {
      give_up(z0 + D);
      return;
    }
  } else {
    cp_async_wait<D - R>();  // planes up to z0+R have arrived
    __syncthreads();
  }
  float4 qv[QL];
#pragma unroll
  for (int q = 0; q < 2 * R; ++q) qv[q] = own(q);
#pragma unroll
  for (int q = 0; q <= R; ++q) fill(z0 + q, R + q);
  __syncthreads();
  // slots 0 .. R-2 (planes z0-R .. z0-2) are free: the planes after z0+D
#pragma unroll
  for (int q = 0; q + 1 < R; ++q) issue(z0 + D + 1 + q, q);

  int idx0 = z0 * plane + j * g.px + i;
  const bool live = nx > 0 && j < N;
  for (int kb = z0; kb < z1; kb += NB) {
#pragma unroll
    for (int uu = 0; uu < NB; ++uu) {
      const int k = kb + uu;
      if (k >= z1) break;  // uniform
      const int sc = (uu + R) % NB;           // slot of plane k
      const int sn = (uu + 2 * R) % NB;       // slot of plane k+R
      const int sf = (uu + R + NB - 1) % NB;  // slot of plane k-1 (refilled)
      typename Op::Ex4 ex;
      if (live) ex = o.load4(idx0);
      if (TMA) {
        const bool ok = arrived(k + R, sn);
        if (__syncthreads_or(!ok)) {
          give_up(k + R + D - 1);
          return;
        }
      } else {
        cp_async_wait<D - 1>();
        __syncthreads();
      }
      // plane k+R has arrived: its own points enter the queue and its
      // boundary cells are completed (read as a current plane R iterations
      // later, after a barrier); plane k-1 is no longer read (after the
      // barrier), its slot takes plane k+R+D
      qv[(uu + 2 * R) % QL] = own(sn);
      if (k > z0) fill(k + R, sn);  // the prologue completed plane z0+R
      issue(k + R + D, sf);
      const float* P0 = ring + sc * PS + sbase;
      const float4 cc = qv[(uu + R) % QL];
      const float c[4] = {cc.x, cc.y, cc.z, cc.w};
      // x: a[2..3] = x-2, x-1; a[4..7] = the four points; a[8..9] = x+4, x+5
      float a[10];
      if (R == 2) {
        const float2 lh = *reinterpret_cast<const float2*>(P0 - 2);
        const float2 rh = *reinterpret_cast<const float2*>(P0 + 4);
        a[2] = lh.x; a[3] = lh.y; a[8] = rh.x; a[9] = rh.y;
      } else {
        a[2] = 0.f; a[3] = P0[-1]; a[8] = P0[4]; a[9] = 0.f;
      }
      a[4] = c[0]; a[5] = c[1]; a[6] = c[2]; a[7] = c[3];
      const float4 ym1 = *reinterpret_cast<const float4*>(P0 - SX);
      const float4 yp1 = *reinterpret_cast<const float4*>(P0 + SX);
      const float4 zm1 = qv[(uu + R - 1) % QL], zp1 = qv[(uu + R + 1) % QL];
      float xm1v[4], xp1v[4], ym1v[4] = {ym1.x, ym1.y, ym1.z, ym1.w}, yp1v[4] = {yp1.x, yp1.y, yp1.z, yp1.w};
      float zm1v[4] = {zm1.x, zm1.y, zm1.z, zm1.w}, zp1v[4] = {zp1.x, zp1.y, zp1.z, zp1.w};
      float xm2v[4] = {0.f, 0.f, 0.f, 0.f}, xp2v[4] = {0.f, 0.f, 0.f, 0.f};
      float ym2v[4] = {0.f, 0.f, 0.f, 0.f}, yp2v[4] = {0.f, 0.f, 0.f, 0.f};
      float zm2v[4] = {0.f, 0.f, 0.f, 0.f}, zp2v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xm1v[q] = a[3 + q];
        xp1v[q] = a[5 + q];
      }
      if (R == 2) {
        const float4 ym2 = *reinterpret_cast<const float4*>(P0 - 2 * SX);
        const float4 yp2 = *reinterpret_cast<const float4*>(P0 + 2 * SX);
        const float4 zm2 = qv[(uu + R - 2 + QL) % QL], zp2 = qv[(uu + R + 2) % QL];
        ym2v[0] = ym2.x; ym2v[1] = ym2.y; ym2v[2] = ym2.z; ym2v[3] = ym2.w;
        yp2v[0] = yp2.x; yp2v[1] = yp2.y; yp2v[2] = yp2.z; yp2v[3] = yp2.w;
        zm2v[0] = zm2.x; zm2v[1] = zm2.y; zm2v[2] = zm2.z; zm2v[3] = zm2.w;
        zp2v[0] = zp2.x; zp2v[1] = zp2.y; zp2v[2] = zp2.z; zp2v[3] = zp2.w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xm2v[q] = a[2 + q];
          xp2v[q] = a[6 + q];
        }
      }
      if (k < R || k >= N - R) {
#pragma unroll
        for (int q = 0; q < 4; ++q) fix_axis<float, R>(k, N, c[q], zm1v[q], zp1v[q], zm2v[q], zp2v[q]);
      }
      float s1[4], s2[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s1[q] = ((xm1v[q] + xp1v[q]) + (ym1v[q] + yp1v[q])) + (zm1v[q] + zp1v[q]);
        s2[q] = R == 2 ? ((xm2v[q] + xp2v[q]) + (ym2v[q] + yp2v[q])) + (zm2v[q] + zp2v[q]) : 0.f;
      }
      if (live) o.apply4(idx0, nx, c, s1, s2, ex);
      idx0 += plane;
    }
  }
  if (!TMA) cp_async_wait<0>();
}

// k_zq4 as a producer/consumer pipeline without block barriers: one extra
// warp issues the TMA box of every plane once the ring slot it goes to has
// been released, and each compute warp waits only for the slot's "full"
// barrier and releases the slot (one arrival per warp on its "empty"
// barrier) after its last read, so warps drift apart by up to the prefetch
// depth instead of meeting at every plane.  The ring holds plain copies (the
// out-of-domain cells read the TMA zero fill) and every boundary value is
// set in registers: x at the two edge lanes, y for whole warps, z at the
// edge planes.  Waits are bounded like k_zq4's; a warp that gives up sets
// g_zq_timeout and returns, the producer then waits (bounded) for the copies
// it issued.  The sums per point are those of k_tile4, so the results are
// bitwise identical.
template <int ORDER, int TYT, int DEEP>
constexpr int zqp_min_blocks() {  // register floor 96: no spills in any variant
  return (232448 / zq_smem<ORDER, TYT, DEEP>()) < (65536 / (32 * (TYT + 1) * 96))
             ? (232448 / zq_smem<ORDER, TYT, DEEP>())
             : (65536 / (32 * (TYT + 1) * 96));
}

template <int ORDER, int TYT, int DEEP, typename Op>
__global__ void __launch_bounds__(32 * (TYT + 1), (zqp_min_blocks<ORDER, TYT, DEEP>()))
    k_zq4p(Grid g, int nzc, int zc, const int* active, Op op, const __grid_constant__ CUtensorMap tmap) {
  static_assert(sizeof(typename Op::T) == 4, "k_zq4p is the FP32 path");
  static_assert(ORDER == 2 || ORDER == 4, "k_zq4p: 7-point and wide stencils");
  constexpr int R = ORDER == 4 ? 2 : 1;
  constexpr int D = zq_depth<ORDER, DEEP>();
  constexpr int NB = R + D + 1;
  constexpr int QL = 2 * R + 1;
  static_assert(NB % QL == 0, "ring size must be a multiple of the queue length");
  constexpr int TX = 128, TY = TYT, XH = 4;
  constexpr int SX = TX + 2 * XH, SY = TY + 2 * R;
  constexpr int PS = zq_slot_floats<ORDER, TYT>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long full[NB], empty[NB];
  float* ring = reinterpret_cast<float*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int b = blockIdx.z / nzc;
  if (active && !active[b]) return;  // uniform over the block
  const int N = g.N;
  const int plane = (int)g.plane;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = (blockIdx.z - b * nzc) * zc, z1 = min(N, z0 + zc);
  const int warp = threadIdx.y, lane = threadIdx.x;
  const unsigned ring_s = (unsigned)__cvta_generic_to_shared(ring);
  const unsigned full_s = (unsigned)__cvta_generic_to_shared(full);
  const unsigned empty_s = (unsigned)__cvta_generic_to_shared(empty);
  if (warp == 0 && lane == 0) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      mbar_init(full_s + 8u * q, 1);
      mbar_init(empty_s + 8u * q, TYT);
    }
    mbar_init_fence();
  }
  __syncthreads();
  // fill f of the ring holds plane z0 - R + f in slot f mod NB; phase f / NB
  // of that slot's barriers belongs to it
  const int last = z1 - 1 + R;  // the last plane a compute warp reads
  if (warp == TYT) {  // the producer
    if (lane == 0) {
      int f = 0;
      bool ok = true;
      for (; z0 - R + f <= last; ++f) {
        const int p = z0 - R + f, s = f % NB;
        if (f >= NB && !mbar_wait_bounded(empty_s + 8u * s, (unsigned)(f / NB - 1) & 1u)) {
          ok = false;
          break;
        }
        const unsigned bar = full_s + 8u * s;
        if (p >= 0 && p < N) {
          fence_proxy_async_smem();
          mbar_expect_tx(bar, (unsigned)(SY * SX * 4));
          tma_load_4d(ring_s + (unsigned)(s * PS) * 4u, &tmap, x0 - XH, y0 - R, p, b, bar);
        } else {
          mbar_arrive(bar);
        }
      }
      if (!ok) {  // wait for the copies already issued, then leave
        atomicExch(&g_zq_timeout, 1);
        for (int q = f - 1; q >= 0 && q > f - 1 - NB; --q)
          mbar_wait_bounded(full_s + 8u * (q % NB), (unsigned)(q / NB) & 1u);
      }
    }
    return;
  }

  Op o = op;
  o.init(b);
  const int i = x0 + 4 * lane;
  const int j = y0 + warp;
  const int sbase = (R + warp) * SX + XH + 4 * lane;
  const int nx = N - i;
  auto own = [&](int slot) { return *reinterpret_cast<const float4*>(ring + slot * PS + sbase); };
  auto wait_full = [&](int p) {
    const int f = p - z0 + R;
    return mbar_wait_bounded(full_s + 8u * (f % NB), (unsigned)(f / NB) & 1u);
  };
  auto release = [&](int slot) {
    __syncwarp();
    if (lane == 0) mbar_arrive(empty_s + 8u * slot);
  };
  float4 qv[QL];
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 2 * R; ++q) {
    ok = wait_full(z0 - R + q) && ok;
    qv[q] = own(q);
  }
  if (!ok) {
    atomicExch(&g_zq_timeout, 1);
    return;
  }
#pragma unroll
  for (int q = 0; q < R; ++q) release(q);  // planes z0-R .. z0-1 only feed the queue

  int idx0 = z0 * plane + j * g.px + i;
  const bool live = nx > 0 && j < N;
  const bool yedge = j < R || j >= N - R;  // the same for the whole warp
  for (int kb = z0; kb < z1; kb += NB) {
#pragma unroll
    for (int uu = 0; uu < NB; ++uu) {
      const int k = kb + uu;
      if (k >= z1) break;  // uniform
      const int sc = (uu + R) % NB;      // slot of plane k
      const int sn = (uu + 2 * R) % NB;  // slot of plane k+R
      typename Op::Ex4 ex;
      if (live) ex = o.load4(idx0);
      if (!wait_full(k + R)) {
        atomicExch(&g_zq_timeout, 1);
        return;
      }
      qv[(uu + 2 * R) % QL] = own(sn);
      const float* P0 = ring + sc * PS + sbase;
      const float4 cc = qv[(uu + R) % QL];
      const float c[4] = {cc.x, cc.y, cc.z, cc.w};
      float a[10];
      if (R == 2) {
        const float2 lh = *reinterpret_cast<const float2*>(P0 - 2);
        const float2 rh = *reinterpret_cast<const float2*>(P0 + 4);
        a[2] = lh.x; a[3] = lh.y; a[8] = rh.x; a[9] = rh.y;
      } else {
        a[2] = 0.f; a[3] = P0[-1]; a[8] = P0[4]; a[9] = 0.f;
      }
      a[4] = c[0]; a[5] = c[1]; a[6] = c[2]; a[7] = c[3];
      // x boundary: index -1 and N read 0, the wide stencil's ghosts -2 and
      // N+1 minus the cell at 0 and N-1
      if (i == 0) {
        a[3] = 0.f;
        if (R == 2) a[2] = -c[0];
      }
      if (nx > 0 && nx <= 4) {
        const float cl = nx == 1 ? c[0] : nx == 2 ? c[1] : nx == 3 ? c[2] : c[3];
#pragma unroll
        for (int t = 5; t <= 9; ++t) {
          if (t == 4 + nx) a[t] = 0.f;
          if (R == 2 && t == 5 + nx) a[t] = -cl;
        }
      }
      const float4 ym1 = *reinterpret_cast<const float4*>(P0 - SX);
      const float4 yp1 = *reinterpret_cast<const float4*>(P0 + SX);
      const float4 zm1 = qv[(uu + R - 1) % QL], zp1 = qv[(uu + R + 1) % QL];
      float xm1v[4], xp1v[4], ym1v[4] = {ym1.x, ym1.y, ym1.z, ym1.w}, yp1v[4] = {yp1.x, yp1.y, yp1.z, yp1.w};
      float zm1v[4] = {zm1.x, zm1.y, zm1.z, zm1.w}, zp1v[4] = {zp1.x, zp1.y, zp1.z, zp1.w};
      float xm2v[4] = {0.f, 0.f, 0.f, 0.f}, xp2v[4] = {0.f, 0.f, 0.f, 0.f};
      float ym2v[4] = {0.f, 0.f, 0.f, 0.f}, yp2v[4] = {0.f, 0.f, 0.f, 0.f};
      float zm2v[4] = {0.f, 0.f, 0.f, 0.f}, zp2v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xm1v[q] = a[3 + q];
        xp1v[q] = a[5 + q];
      }
      if (R == 2) {
        const float4 ym2 = *reinterpret_cast<const float4*>(P0 - 2 * SX);
        const float4 yp2 = *reinterpret_cast<const float4*>(P0 + 2 * SX);
        const float4 zm2 = qv[(uu + R - 2 + QL) % QL], zp2 = qv[(uu + R + 2) % QL];
        ym2v[0] = ym2.x; ym2v[1] = ym2.y; ym2v[2] = ym2.z; ym2v[3] = ym2.w;
        yp2v[0] = yp2.x; yp2v[1] = yp2.y; yp2v[2] = yp2.z; yp2v[3] = yp2.w;
        zm2v[0] = zm2.x; zm2v[1] = zm2.y; zm2v[2] = zm2.z; zm2v[3] = zm2.w;
        zp2v[0] = zp2.x; zp2v[1] = zp2.y; zp2v[2] = zp2.z; zp2v[3] = zp2.w;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xm2v[q] = a[2 + q];
          xp2v[q] = a[6 + q];
        }
      }
      release(sc);  // plane k's slot is read for the last time above
      if (yedge) {
#pragma unroll
        for (int q = 0; q < 4; ++q) fix_axis<float, R>(j, N, c[q], ym1v[q], yp1v[q], ym2v[q], yp2v[q]);
      }
      if (k < R || k >= N - R) {
#pragma unroll
        for (int q = 0; q < 4; ++q) fix_axis<float, R>(k, N, c[q], zm1v[q], zp1v[q], zm2v[q], zp2v[q]);
      }
      float s1[4], s2[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s1[q] = ((xm1v[q] + xp1v[q]) + (ym1v[q] + yp1v[q])) + (zm1v[q] + zp1v[q]);
        s2[q] = R == 2 ? ((xm2v[q] + xp2v[q]) + (ym2v[q] + yp2v[q])) + (zm2v[q] + zp2v[q]) : 0.f;
      }
      if (live) o.apply4(idx0, nx, c, s1, s2, ex);
      idx0 += plane;
    }
  }
}

// The driver's tensor-map encoder, looked up once through the runtime (the
// library does not link against the driver library itself).
inline PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  }();
  return fn;
}

// zc > 0: planes per z-chunk; zc = -w: the chunk length for which the grid
// fills w whole waves of the GPU (152 SMs x the blocks one SM holds).
// TMA = 0: k_zq4 with cp.async, 1: k_zq4 with TMA, 2: k_zq4p (TMA, producer
// warp, no block barriers).
template <int ORDER, int TYT, int DEEP, int TMA, typename Op>
cudaError_t launch_zq4(const Grid& g, int B, int zc, const int* active, const Op& op, cudaStream_t st) {
  constexpr int smem = zq_smem<ORDER, TYT, DEEP>();
  constexpr int R = ORDER == 4 ? 2 : 1;
  constexpr int threads = 32 * (TYT + (TMA == 2 ? 1 : 0));
  void (*kern)(Grid, int, int, const int*, Op, const CUtensorMap);
  if constexpr (TMA == 2) kern = k_zq4p<ORDER, TYT, DEEP, Op>;
  else kern = k_zq4<ORDER, TYT, DEEP, TMA, Op>;
  if (smem > 48 * 1024) {
    static std::atomic<bool> set{false};  // set once per process (one device)
    if (!set.load()) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      set.store(true);
    }
  }
  const int tiles = ((g.N + 127) / 128) * ((g.N + TYT - 1) / TYT) * B;
  if (zc <= 0) {
    static std::atomic<int> slots{0};  // resident blocks on the whole GPU (one device)
    if (slots.load() == 0) {
      int dev = 0, sms = 0, bps = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, smem);
      if (e != cudaSuccess) return e;
      slots.store(std::max(1, sms * bps));
    }
    const int waves = zc < 0 ? -zc : 1;
    const int nfit = std::max(1, waves * slots.load() / tiles);
    zc = (g.N + nfit - 1) / nfit;
  }
  zc = std::min(zc, g.N);
  const int nzc = (g.N + zc - 1) / zc;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  if (TMA) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return cudaErrorNotSupported;
    // dimensions x (pitch), y, z, item; the box is one plane of the tile with
    // its halo, (128 + 8) x (TYT + 2R), starting at x0 - 4 (16-byte aligned)
    const cuuint64_t dims[4] = {(cuuint64_t)g.px, (cuuint64_t)g.N, (cuuint64_t)g.N, (cuuint64_t)B};
    const cuuint64_t strides[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.plane * 4,
                                   (cuuint64_t)op.src_stride() * 4};
    const cuuint32_t box[4] = {128 + 8, (cuuint32_t)(TYT + 2 * R), 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)op.src_base(), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  dim3 blk(32, threads / 32, 1);
  dim3 grd((g.N + 127) / 128, (g.N + TYT - 1) / TYT, nzc * B);
  kern<<<grd, blk, smem, st>>>(g, nzc, zc, active, op, map);
  return cudaSuccess;
}

template <typename Op, typename = void>
struct has_vec4 : std::false_type {};
template <typename Op>
struct has_vec4<Op, std::void_t<decltype(Op::kVec4)>> : std::integral_constant<bool, Op::kVec4> {};

template <int ORDER, bool NORM, typename Op>
cudaError_t run_stencil(const Grid& g, int B, const int* active, unsigned long long* norm_bits,
                        const Op& op, Shape sh, cudaStream_t st) {
  if (B <= 0 || g.N <= 0) return cudaSuccess;
  int kind = sh.kind;
  if (kind == 0) kind = g.N >= 32 ? 3 : 1;
  int zc = sh.zc > 0 ? sh.zc : 16;
  if (zc > g.N) zc = g.N;
  const int nzc = (g.N + zc - 1) / zc;
  cudaError_t e = cudaSuccess;
  switch (kind) {
    case 1: {
      dim3 blk(32, 4, 1);
      dim3 grd((g.N + 31) / 32, (g.N + 3) / 4, nzc * B);
      k_zmarch<ORDER, NORM, Op><<<grd, blk, 0, st>>>(g, nzc, zc, active, norm_bits, op);
      break;
    }
    case 2: e = launch_tile<ORDER, 4, 2, 3, NORM>(g, B, nzc, zc, active, norm_bits, op, st); break;
    case 4: e = launch_tile<ORDER, 4, 4, 3, NORM>(g, B, nzc, zc, active, norm_bits, op, st); break;
    case 5: e = launch_tile<ORDER, 4, 2, 6, NORM>(g, B, nzc, zc, active, norm_bits, op, st); break;
    case 6: e = launch_tile<ORDER, 8, 2, 6, NORM>(g, B, nzc, zc, active, norm_bits, op, st); break;
    case 7: case 8: case 9: case 10: case 11: case 12: case 13: case 14:
      if constexpr (has_vec4<Op>::value && !NORM) {
        switch (kind) {
          case 7: e = launch_tile4<ORDER, 4, 2, 3>(g, B, nzc, zc, active, op, st); break;
          case 8: e = launch_tile4<ORDER, 8, 1, 3>(g, B, nzc, zc, active, op, st); break;
          case 9: e = launch_tile4<ORDER, 4, 4, 3>(g, B, nzc, zc, active, op, st); break;
          case 10: e = launch_tile4<ORDER, 8, 2, 3>(g, B, nzc, zc, active, op, st); break;
          case 11: e = launch_tile4<ORDER, 4, 2, 6>(g, B, nzc, zc, active, op, st); break;
          case 12: e = launch_tile4<ORDER, 8, 1, 6>(g, B, nzc, zc, active, op, st); break;
          case 13: e = launch_tile4<ORDER, 4, 2, 10>(g, B, nzc, zc, active, op, st); break;
          default: e = launch_tile4<ORDER, 2, 2, 6>(g, B, nzc, zc, active, op, st); break;
        }
        break;
      }
      [[fallthrough]];
    case 15: case 16: case 17: case 18: case 19: case 20: case 21: case 22: case 23: case 24:
    case 25: case 26:
      if constexpr (has_vec4<Op>::value && !NORM && ORDER != kCompact) {
        if (kind >= 15) {
          const int zr = sh.zc;  // the launcher resolves wave-fitted chunks (zc < 0)
          switch (kind) {
            case 15: e = launch_zq4<ORDER, 8, 0, 0>(g, B, zr, active, op, st); break;
            case 16: e = launch_zq4<ORDER, 4, 0, 0>(g, B, zr, active, op, st); break;
            case 17: e = launch_zq4<ORDER, 8, 1, 0>(g, B, zr, active, op, st); break;
            case 18: e = launch_zq4<ORDER, 16, 0, 0>(g, B, zr, active, op, st); break;
            case 19: e = launch_zq4<ORDER, 8, 0, 1>(g, B, zr, active, op, st); break;
            case 20: e = launch_zq4<ORDER, 4, 0, 1>(g, B, zr, active, op, st); break;
            case 21: e = launch_zq4<ORDER, 8, 1, 1>(g, B, zr, active, op, st); break;
            case 22: e = launch_zq4<ORDER, 16, 0, 1>(g, B, zr, active, op, st); break;
            case 23: e = launch_zq4<ORDER, 8, 1, 2>(g, B, zr, active, op, st); break;
            case 24: e = launch_zq4<ORDER, 4, 1, 2>(g, B, zr, active, op, st); break;
            case 25: e = launch_zq4<ORDER, 8, 0, 2>(g, B, zr, active, op, st); break;
            default: e = launch_zq4<ORDER, 16, 0, 2>(g, B, zr, active, op, st); break;
          }
          break;
        }
      }
      [[fallthrough]];
    default: e = launch_tile<ORDER, 8, 2, 3, NORM>(g, B, nzc, zc, active, norm_bits, op, st); break;
  }
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

template <typename TR>
cudaError_t launch_resid64(int order, const Grid& g, int B, const double* u, long long u_stride,
                           const double* b, long long b_stride, const Coef<double>* coef,
                           TR* bp_out, const Coef<TR>* coef_r,
                           unsigned long long* norm_bits, const int* active, Shape sh,
                           cudaStream_t st) {
  if (order == kCompact) {
    OpResid64<kCompact, TR> op{u, u_stride, b, b_stride, coef, bp_out, coef_r, g.fs, 0.0, 0.0, TR(0)};
    return norm_bits ? run_stencil<kCompact, true>(g, B, active, norm_bits, op, sh, st)
                     : run_stencil<kCompact, false>(g, B, active, nullptr, op, sh, st);
  }
  if (order == 2) {
    OpResid64<2, TR> op{u, u_stride, b, b_stride, coef, bp_out, coef_r, g.fs, 0.0, 0.0, TR(0)};
    return norm_bits ? run_stencil<2, true>(g, B, active, norm_bits, op, sh, st)
                     : run_stencil<2, false>(g, B, active, nullptr, op, sh, st);
  }
  OpResid64<4, TR> op{u, u_stride, b, b_stride, coef, bp_out, coef_r, g.fs, 0.0, 0.0, TR(0)};
  return norm_bits ? run_stencil<4, true>(g, B, active, norm_bits, op, sh, st)
                   : run_stencil<4, false>(g, B, active, nullptr, op, sh, st);
}

template <typename T>
cudaError_t launch_jacobi(int order, const Grid& g, int B, const T* e, const T* r, T* out,
                          double* u64, long long u64_stride, const Coef<T>* coef,
                          const int* active, Shape sh, cudaStream_t st) {
  if (order == kCompact) {
    if (u64) {
      OpJacobi<T, kCompact, true> op{e, r, out, g.fs, u64, u64_stride, coef, T(0), T(0), T(0)};
      return run_stencil<kCompact, false>(g, B, active, nullptr, op, sh, st);
    }
    OpJacobi<T, kCompact, false> op{e, r, out, g.fs, u64, u64_stride, coef, T(0), T(0), T(0)};
    return run_stencil<kCompact, false>(g, B, active, nullptr, op, sh, st);
  }
  if (u64) {
    if (order == 2) {
      OpJacobi<T, 2, true> op{e, r, out, g.fs, u64, u64_stride, coef, T(0), T(0), T(0)};
      return run_stencil<2, false>(g, B, active, nullptr, op, sh, st);
    }
    OpJacobi<T, 4, true> op{e, r, out, g.fs, u64, u64_stride, coef, T(0), T(0), T(0)};
    return run_stencil<4, false>(g, B, active, nullptr, op, sh, st);
  }
  if (order == 2) {
    OpJacobi<T, 2, false> op{e, r, out, g.fs, u64, u64_stride, coef, T(0), T(0), T(0)};
    return run_stencil<2, false>(g, B, active, nullptr, op, sh, st);
  }
  OpJacobi<T, 4, false> op{e, r, out, g.fs, u64, u64_stride, coef, T(0), T(0), T(0)};
  return run_stencil<4, false>(g, B, active, nullptr, op, sh, st);
}

template <typename T>
cudaError_t launch_resid(int order, const Grid& g, int B, const T* e, const T* r, T* rr,
                         const Coef<T>* coef, const int* active, Shape sh, cudaStream_t st) {
  if (order == kCompact) {
    OpResid<T, kCompact> op{e, r, rr, g.fs, coef, T(0), T(0)};
    return run_stencil<kCompact, false>(g, B, active, nullptr, op, sh, st);
  }
  if (order == 2) {
    OpResid<T, 2> op{e, r, rr, g.fs, coef, T(0), T(0)};
    return run_stencil<2, false>(g, B, active, nullptr, op, sh, st);
  }
  OpResid<T, 4> op{e, r, rr, g.fs, coef, T(0), T(0)};
  return run_stencil<4, false>(g, B, active, nullptr, op, sh, st);
}

}  // namespace h3d
