// probe.cu -- FP64 FMA throughput of this GPU, the roofline denominator of the
// FP64 stencil kernels (they are bound by the FP64 pipe, not by HBM).
//
// Every thread runs kChains independent FMA chains x = x * a + b (a just
// below 1, so the values stay bounded), enough warps per SM to hide the
// pipe's latency; the result is FMAs per second over the timed launch.
#include "runtime.cuh"
#include "stencil_impl.cuh"

namespace {

constexpr int kChains = 8;
__device__ double g_probe_sink;

__global__ void __launch_bounds__(512) k_fp64_fma_probe(int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = 1e-3 * (threadIdx.x + q);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += x[q];
  if (s == -1.0) g_probe_sink = s;  // never true: keeps the chains live
}

// One block waits on an mbarrier with the bounded wait of the TMA plane
// loader; the barrier completes only if `arrive` is set.  out = number of
// threads whose wait gave up.
__global__ void k_mbar_selftest(int arrive, int* out) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned b = (unsigned)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    h3d::mbar_init(b, 1);
    h3d::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0 && arrive) h3d::mbar_arrive(b);
  if (!h3d::mbar_wait_bounded(b, 0)) atomicAdd(out, 1);
}

__device__ int g_mbar_selftest_out;

}  // namespace

extern "C" int heat3d_selftest_mbarrier(void* stream, int arrive) {
  cudaStream_t st = (cudaStream_t)stream;
  int* out = nullptr;
  if (cudaGetSymbolAddress((void**)&out, g_mbar_selftest_out) != cudaSuccess) return HEAT3D_ECUDA;
  int failed = 0;
  cudaError_t err = cudaMemsetAsync(out, 0, sizeof(int), st);
  if (err == cudaSuccess) {
    k_mbar_selftest<<<1, 64, 0, st>>>(arrive ? 1 : 0, out);
    h3d::count_launch();
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaMemcpyAsync(&failed, out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return HEAT3D_ECUDA;
  return failed ? HEAT3D_ETIMEOUT : HEAT3D_OK;
}

extern "C" int heat3d_fp64_probe(void* stream, double* fma_per_s) {
  if (!fma_per_s) return HEAT3D_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HEAT3D_ECUDA;
  const int threads = 512, blocks = 4 * sms, iters = 8192;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // first launch warms up
    err = cudaEventRecord(e0, st);
    k_fp64_fma_probe<<<blocks, threads, 0, st>>>(iters, 0.9999999, 1e-7);
    h3d::count_launch();
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) return HEAT3D_ECUDA;
  *fma_per_s = (double)blocks * threads * kChains * (double)iters / (best * 1e-3);
  return HEAT3D_OK;
}
