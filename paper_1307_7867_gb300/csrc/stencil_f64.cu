// stencil_f64.cu -- FP64 instantiations of the stencil launchers and the
// operator launcher (kernels in stencil_impl.cuh); split from the FP32 ones
// so that the two compile in parallel.
#include "stencil_impl.cuh"

namespace h3d {

cudaError_t launch_lap(int order, const Grid& g, int B, const double* u, long long u_stride,
                       double* out, long long out_stride, const double* alpha,
                       const double* add_src, double* add_dst, long long add_stride,
                       const int* active, Shape sh, cudaStream_t st, double* wu_out) {
  if (order == kCompact) {
    if (add_src) {
      OpLap<kCompact, true> op{u, u_stride, out, out_stride, alpha, add_src, add_dst, add_stride, 0.0};
      op.wu = wu_out;
      return run_stencil<kCompact, false>(g, B, active, nullptr, op, sh, st);
    }
    OpLap<kCompact, false> op{u, u_stride, out, out_stride, alpha, add_src, add_dst, add_stride, 0.0};
    op.wu = wu_out;
    return run_stencil<kCompact, false>(g, B, active, nullptr, op, sh, st);
  }
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
H3D_INST(double)
#undef H3D_INST

}  // namespace h3d
