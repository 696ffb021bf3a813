// persist.cu -- a whole multigrid solve (Sec. 1.2: residual, V-cycles, stop
// rule) of a small grid as one persistent cooperative kernel.
//
// On grids of up to 31^3 points each kernel of a V-cycle runs for a few
// microseconds, and the launch sequence costs about 14 launches per cycle, so
// launch and tail latency set the solve time.  Here one cooperative launch
// runs the solve from the first FP64 residual to the last stop check:
//  * the levels with N >= 15 run grid-wide, each operation (Jacobi sweep,
//    residual, restriction into the next level's scaled right-hand side,
//    which is also its first iterate, prolongation, the FP64 residual and its
//    norm) followed by a grid barrier;
//    a block takes chunks of 256 consecutive points of one item;
//  * the levels with N <= 7 run in one block per item, in shared memory
//    (vcycle_small_body, the code of the fused coarse kernel);
//  * after each FP64 residual every block applies the stop rule to every item
//    itself (the same rule as launch_mg_check), so that all blocks agree on
//    which items go on without another barrier; block 0 writes the per-item
//    cycle counts, last norms and flags for the host.
// Every point is computed with the operations of the separate kernels in the
// same order (neighbour sums, fused multiply-adds, restriction and
// prolongation sums), so solutions and cycle counts are bitwise those of the
// launch sequence.
//
// Data that another block wrote during the launch is read through L2
// (ld.global.cg), never through the non-coherent read-only path.  The grid
// barrier is one arrival counter; a waiting block gives up after about one
// second, sets an error word that every other waiting block sees, and all
// blocks return; the host then reports HEAT3D_ETIMEOUT.  The cooperative
// launch guarantees that all blocks are resident at once.

#include <algorithm>

#include "../../include/heat3d.h"
#include "coarse_fused.cuh"
#include "stencil_impl.cuh"

namespace h3d {
namespace {

constexpr int kPersistThreads = 256;
constexpr unsigned long long kBarrierNs = 1000000000ull;  // give up after 1 s
constexpr unsigned kBarrierSpins = 1u << 23;              // second bound on the spin

struct alignas(16) PersistCtl {
  unsigned count;  // arrivals so far in this launch (never reset within it)
  unsigned err;    // 1: a barrier timed out
  unsigned pad[2];
};

template <typename T>
struct PersistArgs {
  MgPersist<T> p;
  int kb;              // first level run by one block per item
  SmallArgs<T> small;  // levels kb .. nlev-1 for vcycle_small_body
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a bounded wait; false when it timed out here or in
// another block (every block then leaves the kernel).  Barrier g of the
// launch completes when the arrival counter reaches g * gridDim.x: each block
// adds one (after a fence that publishes the block's writes) and polls the
// counter with acquire loads, so no reset or separate release write sits on
// the critical path.
__device__ bool grid_barrier(PersistCtl* ctl, unsigned& gen) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = (gen + 1) * gridDim.x;
    __threadfence();
    atomicAdd(&ctl->count, 1u);
    unsigned long long t0 = 0ull;
    for (unsigned it = 1; ld_acquire(&ctl->count) < target; ++it) {
      if ((it & 15) == 0) {
        if (t0 == 0ull) t0 = now_ns();
        if (*(volatile unsigned*)&ctl->err || it >= kBarrierSpins || now_ns() - t0 > kBarrierNs) {
          atomicExch(&ctl->err, 1u);
          ok = 0;
          break;
        }
      }
      __nanosleep(32);
    }
    ++gen;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Value at (i, j, k) under the boundary rule of the stencil kernels (indices
// -1 and N read 0; the wide stencil's -2 and N+1 read -u(0) and -u(N-1)),
// loaded through L2.
template <typename T>
__device__ __forceinline__ T atc(const T* u, const Grid& g, int i, int j, int k) {
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
  T v = __ldcg(u + (long long)k * g.plane + (long long)j * g.px + i);
  return neg ? -v : v;
}

// Neighbour sums in the order of the stencil kernels: ((x) + (y)) + (z).
template <typename T, int ORDER>
__device__ __forceinline__ void nsums_c(const T* f, const Grid& g, int i, int j, int k, T& s1,
                                        T& s2) {
  s1 = ((atc(f, g, i - 1, j, k) + atc(f, g, i + 1, j, k)) +
        (atc(f, g, i, j - 1, k) + atc(f, g, i, j + 1, k))) +
       (atc(f, g, i, j, k - 1) + atc(f, g, i, j, k + 1));
  s2 = T(0);
  if (ORDER == 4)
    s2 = ((atc(f, g, i - 2, j, k) + atc(f, g, i + 2, j, k)) +
          (atc(f, g, i, j - 2, k) + atc(f, g, i, j + 2, k))) +
         (atc(f, g, i, j, k - 2) + atc(f, g, i, j, k + 2));
}

// f(b, i, j, k) for every point of an n^3 index space of each item b with
// act[b] set.  A block takes chunks of blockDim.x consecutive points of one
// item, so the item is uniform over the block.
template <typename F>
__device__ __forceinline__ void for_points(int n, int B, const int* act, F&& f) {
  const int n3 = n * n * n, cpi = (n3 + blockDim.x - 1) / blockDim.x;
  for (int c = blockIdx.x; c < B * cpi; c += gridDim.x) {
    const int b = c / cpi;
    if (!act[b]) continue;
    const int q = (c - b * cpi) * blockDim.x + threadIdx.x;
    if (q < n3) f(b, q % n, (q / n) % n, q / (n * n));
  }
}

// As for_points; f returns the bits of a value whose max |.| per item is
// accumulated into dst[b] (block maximum, one atomic per chunk).
template <typename F>
__device__ __forceinline__ void for_points_max(int n, int B, const int* act,
                                               unsigned long long* red, unsigned long long* dst,
                                               F&& f) {
  const int n3 = n * n * n, cpi = (n3 + blockDim.x - 1) / blockDim.x;
  for (int c = blockIdx.x; c < B * cpi; c += gridDim.x) {
    const int b = c / cpi;
    if (!act[b]) continue;  // uniform over the block
    const int q = (c - b * cpi) * blockDim.x + threadIdx.x;
    unsigned long long v = 0ull;
    if (q < n3) v = f(b, q % n, (q / n) % n, q / (n * n));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = 0ull;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
      if (m != 0ull) atomicMax(dst + b, m);
    }
    __syncthreads();
  }
}

template <typename T, int ORDER>
__global__ void __launch_bounds__(kPersistThreads) k_mg_persist(PersistArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long red[kPersistThreads / 32];
  const MgPersist<T>& a = A.p;
  const int B = a.B;
  int* act = reinterpret_cast<int*>(smem_raw);  // this block's copy of the active flags
  T* bsm = reinterpret_cast<T*>(smem_raw + ((size_t)B * sizeof(int) + 15) / 16 * 16);
  PersistCtl* ctl = reinterpret_cast<PersistCtl*>(a.ctl);
  unsigned gen = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) act[b] = __ldcg(a.active + b);
  __syncthreads();

  // r = b - A u in FP64, b' = wd (T) r, max |r| per item into slot
  auto resid64 = [&](int slot) {
    const Grid& g = a.g[0];
    for_points_max(g.N, B, act, red, a.norm2 + (size_t)slot * B,
                   [&](int b, int i, int j, int k) -> unsigned long long {
                     const long long idx = (long long)k * g.plane + (long long)j * g.px + i;
                     const double* ub = a.u + b * a.us;
                     double s1, s2;
                     nsums_c<double, ORDER>(ub, g, i, j, k, s1, s2);
                     const Coef<double> c = a.c64[b];
                     const double res = a_res<double, ORDER>(c.d, c.e, c.e2, __ldcg(ub + idx), s1,
                                                             s2, __ldcg(a.rhs + b * a.bs + idx));
                     a.b[0][b * g.fs + idx] = a.cf[0][b].wd * (T)res;
                     return abs_bits(res);
                   });
  };
  // damped Jacobi on level k: dst = src + wd (b - A src) = al src + be S + b',
  // or u += that (upd)
  auto jacobi = [&](int k, const T* src, T* dst, bool upd) {
    const Grid& g = a.g[k];
    for_points(g.N, B, act, [&](int b, int i, int j, int kk) {
      const long long idx = (long long)kk * g.plane + (long long)j * g.px + i;
      const T* f = src + b * g.fs;
      T s1, s2;
      nsums_c<T, ORDER>(f, g, i, j, kk, s1, s2);
      const Coef<T> c = a.cf[k][b];
      const T v = jacobi_point<T, ORDER>(c.al, c.be, c.be2, __ldcg(f + idx), s1, s2,
                                         __ldcg(a.b[k] + b * g.fs + idx));
      if (upd) {
        double* up = a.u + b * a.us + idx;
        *up = __ldcg(up) + (double)v;
      } else {
        dst[b * g.fs + idx] = v;
      }
    });
  };
  // dst = t' = wd (b - A src) = b' - om src + be S on level k
  auto resid = [&](int k, const T* src, T* dst) {
    const Grid& g = a.g[k];
    for_points(g.N, B, act, [&](int b, int i, int j, int kk) {
      const long long idx = (long long)kk * g.plane + (long long)j * g.px + i;
      const T* f = src + b * g.fs;
      T s1, s2;
      nsums_c<T, ORDER>(f, g, i, j, kk, s1, s2);
      const Coef<T> c = a.cf[k][b];
      dst[b * g.fs + idx] = resid_point<T, ORDER>(c.om, c.be, c.be2, __ldcg(f + idx), s1, s2,
                                                  __ldcg(a.b[k] + b * g.fs + idx));
    });
  };
  // full weighting of rr (level k) into b' of level k+1 (fw3, times rs / 64)
  auto restrict_to = [&](int k, const T* rr) {
    const Grid& gf = a.g[k];
    const Grid& gc = a.g[k + 1];
    for_points(gc.N, B, act, [&](int b, int i, int j, int kk) {
      const T* f = rr + b * gf.fs + (long long)(2 * kk) * gf.plane + (long long)(2 * j) * gf.px + 2 * i;
      T y[3];
#pragma unroll
      for (int cz = 0; cz < 3; ++cz) {
        T x[3];
#pragma unroll
        for (int cy = 0; cy < 3; ++cy) {
          const T* row = f + (long long)cz * gf.plane + (long long)cy * gf.px;
          x[cy] = fw3(__ldcg(row), __ldcg(row + 1), __ldcg(row + 2));
        }
        y[cz] = fw3(x[0], x[1], x[2]);
      }
      const long long o = b * gc.fs + (long long)kk * gc.plane + (long long)j * gc.px + i;
      a.b[k + 1][o] = fw3(y[0], y[1], y[2]) * (a.cf[k + 1][b].rs * T(0.015625));
    });
  };
  // uf (level k) = src + trilinear prolongation of ec (level k+1), one coarse
  // cell per thread (src may be uf)
  auto prolong = [&](int k, const T* ec, const T* src, T* uf) {
    const Grid& gf = a.g[k];
    const Grid& gc = a.g[k + 1];
    const int Nc = gc.N, Nf = gf.N;
    for_points(Nc + 1, B, act, [&](int b, int cx, int cy, int cz) {
      const T* e = ec + b * gc.fs;
      T v[2][2][2];
#pragma unroll
      for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int y = 0; y < 2; ++y)
#pragma unroll
          for (int x = 0; x < 2; ++x) {
            const int ii = cx - 1 + x, jj = cy - 1 + y, kk = cz - 1 + z;
            v[z][y][x] = (ii < 0 || ii >= Nc || jj < 0 || jj >= Nc || kk < 0 || kk >= Nc)
                             ? T(0)
                             : __ldcg(e + (long long)kk * gc.plane + (long long)jj * gc.px + ii);
          }
      T X[2][2][2], Y[2][2][2];
#pragma unroll
      for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          X[z][y][0] = v[z][y][0] + v[z][y][1];
          X[z][y][1] = v[z][y][1];
        }
#pragma unroll
      for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int mx = 0; mx < 2; ++mx) {
          Y[z][0][mx] = X[z][0][mx] + X[z][1][mx];
          Y[z][1][mx] = X[z][1][mx];
        }
      T* u = uf + b * gf.fs;
      const T* us = src + b * gf.fs;
      // all loads before the first store (src may be uf; each point is read
      // and written by this thread only)
      T o[2][2][2];
#pragma unroll
      for (int mz = 0; mz < 2; ++mz)
#pragma unroll
        for (int my = 0; my < 2; ++my)
#pragma unroll
          for (int mx = 0; mx < 2; ++mx) {
            const int fz = 2 * cz + mz, fy = 2 * cy + my, fx = 2 * cx + mx;
            if (fz < Nf && fy < Nf && fx < Nf)
              o[mz][my][mx] = __ldcg(us + (long long)fz * gf.plane + (long long)fy * gf.px + fx);
          }
#pragma unroll
      for (int mz = 0; mz < 2; ++mz) {
        const int fz = 2 * cz + mz;
        if (fz >= Nf) continue;
#pragma unroll
        for (int my = 0; my < 2; ++my) {
          const int fy = 2 * cy + my;
          if (fy >= Nf) continue;
#pragma unroll
          for (int mx = 0; mx < 2; ++mx) {
            const int fx = 2 * cx + mx;
            if (fx >= Nf) continue;
            const T wv = mz == 0 ? Y[0][my][mx] + Y[1][my][mx] : Y[1][my][mx];
            const int na = (mx == 0) + (my == 0) + (mz == 0);
            const T val = na == 0 ? wv : wv * (na == 1 ? T(0.5) : na == 2 ? T(0.25) : T(0.125));
            u[(long long)fz * gf.plane + (long long)fy * gf.px + fx] = o[mz][my][mx] + val;
          }
        }
      }
    });
  };
  // u += e (level 0)
  auto update = [&](const T* e) {
    const Grid& g = a.g[0];
    for_points(g.N, B, act, [&](int b, int i, int j, int kk) {
      const long long idx = (long long)kk * g.plane + (long long)j * g.px + i;
      double* up = a.u + b * a.us + idx;
      *up = __ldcg(up) + (double)__ldcg(e + b * g.fs + idx);
    });
  };
  // the levels from kb down, one block per item
  auto bottom = [&]() {
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
      if (!act[b]) continue;
      vcycle_small_body<T, ORDER>(A.small, b, bsm);
      __syncthreads();
    }
  };
  // stop rule after the residual in `slot` (launch_mg_check): every block
  // updates its own flags, block 0 also the global per-item records
  auto check = [&](int slot, bool init, int cyc) {
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
      if (!act[b]) continue;
      const double n = __longlong_as_double((long long)__ldcg(a.norm2 + (size_t)slot * B + b));
      int on = 1;
      const bool nan = !(n <= 1e300);
      if (nan) on = 0;
      else if (n <= a.tol[b] || (!init && cyc + 1 >= a.max_cycles)) on = 0;
      if (blockIdx.x == 0) {
        a.last[b] = n;
        if (nan) *a.nan_flag = 1;
        else if (!init) a.ncyc[b] = cyc + 1;
        if (!on) a.active[b] = 0;
      }
      act[b] = on;
    }
    __syncthreads();
  };

  // one V(nu1, nu2) cycle on the error equation (the steps of the launch
  // sequence; warm: start from the previous cycle's correction res0, final:
  // add the correction to u in the last post-smoothing sweep)
  T* res0 = nullptr;
  auto vcycle = [&](bool warm, bool final) -> bool {
    T* cur[kMaxLevels];
    T* oth[kMaxLevels];
    for (int k = 0; k < A.kb; ++k) {
      // b' (a.b[k]) is the first iterate and is never written in the cycle
      T* c = a.b[k];
      T* o = a.e[k];
      int first = 1;
      if (k == 0 && warm) {
        c = res0;
        o = c == a.e[0] ? a.t[0] : a.e[0];
        first = 0;
      }
      for (int s = first; s < a.nu1; ++s) {
        jacobi(k, c, o, false);
        if (!grid_barrier(ctl, gen)) return false;
        if (c == a.b[k]) {
          c = o;
          o = o == a.e[k] ? a.t[k] : a.e[k];
        } else {
          T* tmp = c; c = o; o = tmp;
        }
      }
      resid(k, c, o);
      if (!grid_barrier(ctl, gen)) return false;
      restrict_to(k, o);
      if (!grid_barrier(ctl, gen)) return false;
      cur[k] = c;
      oth[k] = o;
    }
    bottom();
    if (!grid_barrier(ctl, gen)) return false;
    for (int k = A.kb - 1; k >= 0; --k) {
      const T* ce = k + 1 == A.kb ? a.e[A.kb] : cur[k + 1];
      T* c = cur[k];
      T* o = oth[k];
      T* dst = c == a.b[k] ? o : c;
      prolong(k, ce, c, dst);
      if (!grid_barrier(ctl, gen)) return false;
      if (c == a.b[k]) {
        c = dst;
        o = dst == a.e[k] ? a.t[k] : a.e[k];
      }
      bool added = false;
      for (int s = 0; s < a.nu2; ++s) {
        const bool upd = k == 0 && final && s == a.nu2 - 1;
        jacobi(k, c, o, upd);
        if (!grid_barrier(ctl, gen)) return false;
        if (upd) {
          added = true;
          break;
        }
        T* tmp = c; c = o; o = tmp;
      }
      if (k == 0 && final && !added) {
        update(c);
        if (!grid_barrier(ctl, gen)) return false;
      }
      if (k == 0 && !final) res0 = c;
      cur[k] = c;
    }
    return true;
  };

  resid64(0);
  if (!grid_barrier(ctl, gen)) return;
  check(0, true, 0);
  for (int cyc = 0; cyc < a.max_cycles; ++cyc) {
    int any = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) any |= act[b];
    if (!__syncthreads_or(any)) break;
    // the norm slot of this cycle's residual was last read two checks ago
    const int slot = (cyc + 1) & 1;
    if (blockIdx.x == 0)
      for (int b = threadIdx.x; b < B; b += blockDim.x) a.norm2[(size_t)slot * B + b] = 0ull;
    for (int q = 0; q < a.inner; ++q)
      if (!vcycle(q > 0, q == a.inner - 1)) return;
    resid64(slot);
    if (!grid_barrier(ctl, gen)) return;
    check(slot, false, cyc);
  }
}

// Self-test of the bounded barrier: every block but `absent` waits on one
// barrier; *out = 1 when a wait gave up.
__global__ void k_barrier_selftest(PersistCtl* ctl, int absent, int* out) {
  if ((int)blockIdx.x == absent) return;  // this block never arrives
  unsigned gen = 0;
  const bool ok = grid_barrier(ctl, gen);
  if (threadIdx.x == 0 && !ok) atomicExch(out, 1);
}

template <typename T, int ORDER>
cudaError_t launch_order(const PersistArgs<T>& A, int nblk, size_t smem, cudaStream_t st) {
  auto kern = k_mg_persist<T, ORDER>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
  if ((err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return err;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistThreads, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  nblk = std::max(1, std::min(nblk, per_sm * nsm));
  PersistArgs<T> arg = A;
  void* args[] = {&arg};
  err = cudaLaunchCooperativeKernel((const void*)kern, dim3(nblk), dim3(kPersistThreads), args,
                                    smem, st);
  count_launch();
  return err;
}

}  // namespace

bool mg_persist_supported(int order, int N) {
  return (order == 2 || order == 4) && N >= 15 && N <= kPersistMaxN;
}

template <typename T>
cudaError_t launch_mg_persist(int order, const MgPersist<T>& p, cudaStream_t st) {
  if (p.B <= 0) return cudaSuccess;
  if (!mg_persist_supported(order, p.g[0].N) || p.nlev < 2 || p.nlev > kMaxLevels ||
      p.g[p.nlev - 1].N != 1 || p.nu1 < 1 || p.nu2 < 0 || p.inner < 1 || p.max_cycles < 1)
    return cudaErrorInvalidValue;
  PersistArgs<T> A{};
  A.p = p;
  A.kb = 1;
  while (A.kb < p.nlev && p.g[A.kb].N > 7) ++A.kb;
  SmallArgs<T>& s = A.small;
  s.nlev = p.nlev - A.kb;
  int Ns[kMaxLevels];
  for (int l = 0; l < s.nlev; ++l) {
    Ns[l] = s.N[l] = p.g[A.kb + l].N;
    s.cf[l] = p.cf[A.kb + l];
  }
  s.b = p.b[A.kb];
  s.e = p.e[A.kb];
  s.gtop = p.g[A.kb];
  s.nu1 = p.nu1;
  s.nu2 = p.nu2;
  s.active = nullptr;
  const size_t smem = ((size_t)p.B * sizeof(int) + 15) / 16 * 16 + vcycle_small_smem(s.nlev, Ns, sizeof(T));
  cudaError_t err = cudaMemsetAsync(p.ctl, 0, sizeof(PersistCtl), st);
  if (err == cudaSuccess) err = cudaMemsetAsync(p.norm2, 0, sizeof(unsigned long long) * 2 * p.B, st);
  if (err != cudaSuccess) return err;
  const int N = p.g[0].N;
  const int nblk = p.B * ((N * N * N + kPersistThreads - 1) / kPersistThreads);
  return order == 2 ? launch_order<T, 2>(A, nblk, smem, st) : launch_order<T, 4>(A, nblk, smem, st);
}

template cudaError_t launch_mg_persist<double>(int, const MgPersist<double>&, cudaStream_t);
template cudaError_t launch_mg_persist<float>(int, const MgPersist<float>&, cudaStream_t);

}  // namespace h3d

extern "C" int heat3d_selftest_barrier(void* stream, int absent_block) {
  using namespace h3d;
  if (absent_block < -1 || absent_block >= 4) return HEAT3D_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  void* buf = nullptr;
  if (cudaMalloc(&buf, 32) != cudaSuccess) return HEAT3D_ECUDA;
  PersistCtl* ctl = (PersistCtl*)buf;
  int* out = (int*)((char*)buf + 16);
  int flag = 0;
  cudaError_t err = cudaMemsetAsync(buf, 0, 32, st);
  if (err == cudaSuccess) {
    void* args[] = {&ctl, &absent_block, &out};
    err = cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(4), dim3(32), args, 0, st);
    count_launch();
  }
  if (err == cudaSuccess) err = cudaMemcpyAsync(&flag, out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (err != cudaSuccess) return HEAT3D_ECUDA;
  return flag ? HEAT3D_ETIMEOUT : HEAT3D_OK;
}
