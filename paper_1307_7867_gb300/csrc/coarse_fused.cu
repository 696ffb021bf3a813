// coarse_fused.cu -- the bottom of a V-cycle (Sec. 1.2: coarsening down to
// one unknown) in one kernel.
//
// Multigrid levels with N <= 15 hold at most 15^3 points; run as separate
// launches they are latency-bound (about 19 launches per V-cycle for the
// levels 15, 7, 3, 1).  Here one block per item runs the whole sub-cycle from
// such a level down with every level in shared memory (vcycle_small_body in
// coarse_fused.cuh), bitwise the same as the launch sequence.
#include "coarse_fused.cuh"

namespace h3d {
namespace {

template <typename T, int ORDER>
__global__ void __launch_bounds__(512) k_vcycle_small(SmallArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int item = blockIdx.x;
  if (a.active && !a.active[item]) return;
  vcycle_small_body<T, ORDER>(a, item, reinterpret_cast<T*>(smem_raw));
}

}  // namespace

size_t vcycle_small_smem(int nlev, const int* Ns, size_t tsize) {
  size_t n = 0;
  for (int l = 0; l < nlev; ++l) n += 3 * (size_t)Ns[l] * Ns[l] * Ns[l];
  return n * tsize;
}

template <typename T>
cudaError_t launch_vcycle_small(int order, int nlev, const int* Ns, const Coef<T>* const* cf,
                                int B, const T* b, T* e, const Grid& gtop, int nu1, int nu2,
                                const int* active, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  if (nlev < 1 || nlev > kMaxLevels) return cudaErrorInvalidValue;
  SmallArgs<T> a{};
  a.nlev = nlev;
  for (int l = 0; l < nlev; ++l) {
    a.N[l] = Ns[l];
    a.cf[l] = cf[l];
  }
  a.b = b;
  a.e = e;
  a.gtop = gtop;
  a.nu1 = nu1;
  a.nu2 = nu2;
  a.active = active;
  const size_t smem = vcycle_small_smem(nlev, Ns, sizeof(T));
  cudaError_t err;
  if (order == 2) {
    err = cudaFuncSetAttribute(k_vcycle_small<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_vcycle_small<T, 2><<<B, 512, smem, st>>>(a);
  } else {
    err = cudaFuncSetAttribute(k_vcycle_small<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_vcycle_small<T, 4><<<B, 512, smem, st>>>(a);
  }
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_vcycle_small<double>(int, int, const int*, const Coef<double>* const*, int,
                                                 const double*, double*, const Grid&, int, int,
                                                 const int*, cudaStream_t);
template cudaError_t launch_vcycle_small<float>(int, int, const int*, const Coef<float>* const*, int,
                                                const float*, float*, const Grid&, int, int,
                                                const int*, cudaStream_t);

}  // namespace h3d
