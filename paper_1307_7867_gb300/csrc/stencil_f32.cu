// stencil_f32.cu -- FP32 instantiations of the stencil launchers (kernels in
// stencil_impl.cuh).
#include "stencil_impl.cuh"

namespace h3d {

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
H3D_INST(float)
#undef H3D_INST

}  // namespace h3d
