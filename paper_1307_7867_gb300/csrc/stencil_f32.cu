// stencil_f32.cu -- FP32 instantiations of the stencil launchers (kernels in
// stencil_impl.cuh).
#include "stencil_impl.cuh"

namespace h3d {

#define H3D_INST(T)                                                                            \
  template cudaError_t launch_resid64<T>(int, const Grid&, int, const double*, long long,      \
                                         const double*, long long, const Coef<double>*, T*,     \
                                         const Coef<T>*, unsigned long long*, const int*, Shape, \
                                         cudaStream_t);                                         \
  template cudaError_t launch_jacobi<T>(int, const Grid&, int, const T*, const T*, T*, double*, \
                                        long long, const Coef<T>*, const int*, Shape,          \
                                        cudaStream_t);                                          \
  template cudaError_t launch_resid<T>(int, const Grid&, int, const T*, const T*, T*,          \
                                       const Coef<T>*, const int*, Shape, cudaStream_t);
H3D_INST(float)
#undef H3D_INST

// Reads and clears the flag the FP32 tile sets when a TMA plane copy never
// completed (the kernel then returns without finishing its tile).
cudaError_t loader_timeouts_take(cudaStream_t st, int* flag) {
  *flag = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(flag, g_zq_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && *flag) {
    const int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_zq_timeout, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return e;
}

}  // namespace h3d
