// stencil_kernels.cu -- the 7-point and 13-point (wide) stencil kernels of the
// spatial operator (Sec. 1, method of lines) and of the multigrid smoother and
// residuals (Sec. 1.2), templated on the storage type and stencil order.
//
// Two drivers share one operator interface:
//  * k_tile (grids with N >= 32): a block owns a 32 x TY tile of x-y points
//    and marches along z through a chunk of planes.  The planes it needs
//    (z-R .. z+R, R = 1 or 2) live in a shared-memory ring that cp.async
//    fills D planes ahead in 16-byte chunks, so HBM streams while the block
//    computes; every neighbour is read from shared memory and each thread
//    computes RY rows (independent FP64 chains for the FP64 pipe).  Cells of
//    the tile halo that fall outside the domain are written with plain loads
//    under the boundary rule.
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

// As at(), and 0 for indices beyond the ghost layer (never used by a stencil).
template <typename T>
__device__ __forceinline__ T at_any(const T* __restrict__ u, const Grid& g, int i, int j, int k) {
  const int N = g.N;
  if (i < -2 || i > N + 1 || j < -2 || j > N + 1 || k < -2 || k > N + 1) return T(0);
  return at(u, g, i, j, k);
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

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

template <typename T, int ORDER>
__device__ __forceinline__ T combine(T s1, T s2) {
  if (ORDER == 2) return s1;
  return fma(T(16), s1, -s2);
}

// ---------------------------------------------------------------------------
// operators
// ---------------------------------------------------------------------------

// F = alpha_b L u (and, when ADD, the next substep's rhs add_dst = u + add_src).
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
  __device__ const double* src(int b) const { return u + b * us; }
  __device__ void init(int b) {
    a = alpha[b];
    o_ = out + b * os;
    if (ADD) {
      as_ = add_src + b * as;
      ad_ = add_dst + b * as;
    }
  }
  __device__ Ex load(int idx) const {
    Ex x;
    if (ADD) x.add = as_[idx];
    return x;
  }
  __device__ double apply(int idx, double c, double s1, double s2, const Ex& ex) {
    double L = ORDER == 2 ? fma(-6.0, c, s1) : fma(-90.0, c, fma(16.0, s1, -s2));
    o_[idx] = a * L;
    if (ADD) ad_[idx] = c + ex.add;
    return 0.0;
  }
};

// r = b - A u in FP64, stored as TR; e0 = wd r (first Jacobi iterate from zero).
template <int ORDER, typename TR>
struct OpResid64 {
  using T = double;
  struct Ex { double b; };
  const double* u; long long us;
  const double* bb; long long bs;
  const Coef<double>* coef;
  TR* r; TR* e0; const Coef<TR>* coef_r; long long rs;
  double d, e; TR wd;
  const double* b_;
  TR* r_;
  TR* e0_;
  __device__ const double* src(int b) const { return u + b * us; }
  __device__ void init(int b) {
    d = coef[b].d;
    e = coef[b].e;
    wd = e0 ? coef_r[b].wd : TR(0);
    b_ = bb + b * bs;
    r_ = r + b * rs;
    e0_ = e0 ? e0 + b * rs : nullptr;
  }
  __device__ Ex load(int idx) const { return Ex{b_[idx]}; }
  __device__ double apply(int idx, double c, double s1, double s2, const Ex& ex) {
    double S = combine<double, ORDER>(s1, s2);
    double res = fma(-d, c, fma(e, S, ex.b));
    TR rt = (TR)res;
    r_[idx] = rt;
    if (e0_) e0_[idx] = wd * rt;
    return res;
  }
};

// Damped Jacobi on the error equation: v = e + wd (r - A e); stored (UPD =
// false) or added to the FP64 solution u64 (UPD = true).  UPD is a template
// parameter so that the stored variant contains no FP64 instruction at all
// (a runtime branch is if-converted and would run the FP64 add everywhere).
template <typename TT, int ORDER, bool UPD>
struct OpJacobi {
  using T = TT;
  struct Ex { T r; double u; };
  const T* e; const T* r; T* out; long long fs;
  double* u64; long long u64s;
  const Coef<T>* coef;
  T d, ec, wd;
  const T* r_;
  T* o_;
  double* u_;
  __device__ const T* src(int b) const { return e + b * fs; }
  __device__ void init(int b) {
    d = coef[b].d;
    ec = coef[b].e;
    wd = coef[b].wd;
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
    T S = combine<T, ORDER>(s1, s2);
    T res = fma(-d, c, fma(ec, S, ex.r));
    T v = fma(wd, res, c);
    if (UPD) u_[idx] = ex.u + (double)v;
    else o_[idx] = v;
    return 0.0;
  }
};

// rr = r - A e
template <typename TT, int ORDER>
struct OpResid {
  using T = TT;
  struct Ex { T r; };
  const T* e; const T* r; T* rr; long long fs;
  const Coef<T>* coef;
  T d, ec;
  const T* r_;
  T* o_;
  __device__ const T* src(int b) const { return e + b * fs; }
  __device__ void init(int b) {
    d = coef[b].d;
    ec = coef[b].e;
    r_ = r + b * fs;
    o_ = rr + b * fs;
  }
  __device__ Ex load(int idx) const { return Ex{r_[idx]}; }
  __device__ double apply(int idx, T c, T s1, T s2, const Ex& ex) {
    T S = combine<T, ORDER>(s1, s2);
    o_[idx] = fma(-d, c, fma(ec, S, ex.r));
    return 0.0;
  }
};

// ---------------------------------------------------------------------------
// drivers
// ---------------------------------------------------------------------------

template <int ORDER, bool NORM, typename Op>
__global__ void __launch_bounds__(128) k_zmarch(Grid g, int nzc, int zc, const int* active,
                                                unsigned long long* norm_bits, Op op) {
  using T = typename Op::T;
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
  return (2 * (ORDER == 2 ? 1 : 2) + D + 1) * (TYT * RY + 2 * (ORDER == 2 ? 1 : 2)) *
         (32 + 2 * halo_x<T>()) * (int)sizeof(T);
}

__device__ __forceinline__ int ring_next(int s, int nb) { return s + 1 == nb ? 0 : s + 1; }
__device__ __forceinline__ int ring_prev(int s, int nb) { return s == 0 ? nb - 1 : s - 1; }

template <int ORDER, int TYT, int RY, int D, bool NORM, typename Op>
__global__ void __launch_bounds__(32 * TYT) k_tile(Grid g, int nzc, int zc, const int* active,
                                                   unsigned long long* norm_bits, Op op) {
  using T = typename Op::T;
  constexpr int R = ORDER == 2 ? 1 : 2;
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

  // Plane z into ring slot `slot`: interior 16-byte chunks by cp.async, the
  // rest (domain halo, ghost planes) by plain loads under the boundary rule.
  // A thread's chunks are the same for every plane: offsets computed once.
  constexpr int NCH = (SY * CH + NT - 1) / NT;
  int soff[NCH], cgx[NCH], cgy[NCH], goff[NCH];
  bool fast[NCH];
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int c = tid + q * NT;
    const int ry = c / CH, cx = c - ry * CH;
    cgy[q] = y0 - R + ry;
    cgx[q] = x0 - XH + cx * XH;
    soff[q] = c < SY * CH ? ry * SX + cx * XH : -1;
    goff[q] = cgy[q] * g.px + cgx[q];
    fast[q] = cgy[q] >= 0 && cgy[q] < N && cgx[q] >= 0 && cgx[q] + XH <= N;
  }
  auto issue = [&](int z, int slot) {
    if (z <= z1 - 1 + R) {
      T* dst = ring + slot * PS;
      const bool zin = z >= 0 && z < N;
      const T* uz = u + z * plane;
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        if (soff[q] < 0) continue;
        T* d = dst + soff[q];
        if (zin && fast[q]) {
          cp_async16(d, uz + goff[q]);
        } else {
#pragma unroll
          for (int e = 0; e < XH; ++e) d[e] = at_any(u, g, cgx[q] + e, cgy[q], z);
        }
      }
    }
    cp_async_commit();
  };

#pragma unroll 1
  for (int q = 0; q < 2 * R + D; ++q) issue(z0 - R + q, q);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = x0 + tx;
  const int jb = y0 + ty * RY;
  const int sbase = (R + ty * RY) * SX + XH + tx;
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
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const int o0 = r * SX;
      const T c = P0[o0];
      T s1 = ((P0[o0 - 1] + P0[o0 + 1]) + (P0[o0 - SX] + P0[o0 + SX])) + (Pm1[o0] + Pp1[o0]);
      T s2 = T(0);
      if (R == 2)
        s2 = ((P0[o0 - 2] + P0[o0 + 2]) + (P0[o0 - 2 * SX] + P0[o0 + 2 * SX])) + (Pm2[o0] + Pp2[o0]);
      if (i < N && jb + r < N) {
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
    static bool set = false;
    if (!set) {
      cudaError_t e = cudaFuncSetAttribute(k_tile<ORDER, TYT, RY, D, NORM, Op>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      set = true;
    }
  }
  dim3 blk(32, TYT, 1);
  dim3 grd((g.N + 31) / 32, (g.N + TYT * RY - 1) / (TYT * RY), nzc * B);
  k_tile<ORDER, TYT, RY, D, NORM, Op><<<grd, blk, smem, st>>>(g, nzc, zc, active, norm_bits, op);
  return cudaSuccess;
}

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

cudaError_t launch_lap(int order, const Grid& g, int B, const double* u, long long u_stride,
                       double* out, long long out_stride, const double* alpha,
                       const double* add_src, double* add_dst, long long add_stride,
                       const int* active, Shape sh, cudaStream_t st) {
  if (add_src) {
    if (order == 2) {
      OpLap<2, true> op{u, u_stride, out, out_stride, alpha, add_src, add_dst, add_stride, 0.0};
      return run_stencil<2, false>(g, B, active, nullptr, op, sh, st);
    }
    OpLap<4, true> op{u, u_stride, out, out_stride, alpha, add_src, add_dst, add_stride, 0.0};
    return run_stencil<4, false>(g, B, active, nullptr, op, sh, st);
  }
  if (order == 2) {
    OpLap<2, false> op{u, u_stride, out, out_stride, alpha, add_src, add_dst, add_stride, 0.0};
    return run_stencil<2, false>(g, B, active, nullptr, op, sh, st);
  }
  OpLap<4, false> op{u, u_stride, out, out_stride, alpha, add_src, add_dst, add_stride, 0.0};
  return run_stencil<4, false>(g, B, active, nullptr, op, sh, st);
}

template <typename TR>
cudaError_t launch_resid64(int order, const Grid& g, int B, const double* u, long long u_stride,
                           const double* b, long long b_stride, const Coef<double>* coef,
                           TR* r_out, TR* e0_out, const Coef<TR>* coef_r,
                           unsigned long long* norm_bits, const int* active, Shape sh,
                           cudaStream_t st) {
  if (order == 2) {
    OpResid64<2, TR> op{u, u_stride, b, b_stride, coef, r_out, e0_out, coef_r, g.fs, 0.0, 0.0, TR(0)};
    return norm_bits ? run_stencil<2, true>(g, B, active, norm_bits, op, sh, st)
                     : run_stencil<2, false>(g, B, active, nullptr, op, sh, st);
  }
  OpResid64<4, TR> op{u, u_stride, b, b_stride, coef, r_out, e0_out, coef_r, g.fs, 0.0, 0.0, TR(0)};
  return norm_bits ? run_stencil<4, true>(g, B, active, norm_bits, op, sh, st)
                   : run_stencil<4, false>(g, B, active, nullptr, op, sh, st);
}

template <typename T>
cudaError_t launch_jacobi(int order, const Grid& g, int B, const T* e, const T* r, T* out,
                          double* u64, long long u64_stride, const Coef<T>* coef,
                          const int* active, Shape sh, cudaStream_t st) {
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
  if (order == 2) {
    OpResid<T, 2> op{e, r, rr, g.fs, coef, T(0), T(0)};
    return run_stencil<2, false>(g, B, active, nullptr, op, sh, st);
  }
  OpResid<T, 4> op{e, r, rr, g.fs, coef, T(0), T(0)};
  return run_stencil<4, false>(g, B, active, nullptr, op, sh, st);
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
                                       const Coef<T>*, const int*, Shape, cudaStream_t);
H3D_INST(double)
H3D_INST(float)
#undef H3D_INST

}  // namespace h3d
