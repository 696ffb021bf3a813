// noalloc.cu -- mg_vcycle_noalloc: the multigrid solve of mg_vcycle for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine): code that
// runs while another component owns every byte of device memory (a host
// framework with its own pool, a plugin handed only input and output
// buffers), real-time loops whose memory budget is fixed before they start,
// and libraries that may not allocate behind their caller's back.  This entry
// point takes its scratch from a file-scope static device array instead of a
// caller-bound workspace, so a call needs nothing but the caller's rhs and u.
//
// Limits and rules:
//  - Grids up to N = 63 (kNoAllocMaxN) interior points per axis, N = 2^k - 1;
//    the array is kNoAllocScratchBytes (32 MiB) and every GPU that loads this
//    library keeps it until the process exits.
//  - The first call on a device, with that device current, looks the array's
//    device address up with cudaGetSymbolAddress (host code cannot use the
//    array's name as a device pointer) and builds the host-side solver state.
//  - Every call is synchronous: it waits for its stream to finish before it
//    returns (host buffers are read and written on that stream), so no call
//    can be part of a CUDA graph: a call made while its stream is being
//    captured returns HEAT3D_EINVAL before it touches the stream, and the
//    capture stays valid.
//  - All calls on a device share the array and it keeps the last call's
//    contents; the solver clears what must start at zero (the residual norms
//    each solve, the whole array when the grid, stencil or precision changes).
//    Calls that overlap on the GPU (different streams or threads, in flight at
//    the same time) race on the array and give wrong results: serialise them.
//  - The failure message is kept per host thread.
#include <stdio.h>

#include <mutex>

#include "runtime.cuh"

namespace {

constexpr int kNoAllocMaxN = 63;
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceState {
  bool ready = false;
  void* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  heat3d_ctx* ctx = nullptr;
  int N = 0, order = 0, precision = -1;
};

std::mutex g_mu;
DeviceState g_dev[kMaxDevices];
thread_local char g_err[256] = "";

int fail(int code, const char* msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
  return code;
}

}  // namespace

extern "C" {

int mg_vcycle_noalloc(int N, int order, int precision, double c, const double* rhs, double* u,
                      int max_cycles, double tol, void* stream, heat3d_stats* stats) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (N < 1 || ((N + 1) & N) != 0) return fail(HEAT3D_EINVAL, "N must be 2^k - 1");
  if (N > kNoAllocMaxN) return fail(HEAT3D_EINVAL, "N exceeds the no-allocation limit of 63");
  if ((order != 2 && order != 4) || (precision != HEAT3D_FP64 && precision != HEAT3D_MIXED) ||
      !rhs || !u || max_cycles < 0 || !(c >= 0))
    return fail(HEAT3D_EINVAL, "bad arguments");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess ||
      cap != cudaStreamCaptureStatusNone)
    return fail(HEAT3D_EINVAL,
                "mg_vcycle_noalloc is synchronous and cannot run while its stream is captured");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(HEAT3D_ECUDA, "no current CUDA device");
  DeviceState& s = g_dev[dev];
  if (!s.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(HEAT3D_ECUDA, "cudaGetSymbolAddress failed for the scratch array");
    s.scratch = p;
    s.ready = true;
  }
  if (!s.ctx || s.N != N || s.order != order || s.precision != precision) {
    if (s.ctx) {
      heat3d_destroy(s.ctx);
      s.ctx = nullptr;
    }
    heat3d_config cfg;
    heat3d_config_default(&cfg);
    cfg.nlevels = 1;
    cfg.levels[0] = heat3d_level{N, order, 2};
    cfg.precision = precision;
    cfg.batch = 1;
    cfg.device = dev;
    cfg.stream = stream;
    cfg.autotune = 0;    // tuning would create timing events
    cfg.use_graphs = 0;  // graphs would be instantiated (a resource allocation)
    size_t need = 0;
    char msg[256] = "";
    int rc0 = h3d_workspace_size_msg(&cfg, &need, msg, sizeof(msg));
    if (rc0 != HEAT3D_OK) return fail(rc0, msg);
    if (need > kNoAllocScratchBytes)
      return fail(HEAT3D_ENOMEM, "solver state does not fit in the no-allocation scratch array");
    rc0 = heat3d_init(&cfg, &s.ctx);
    if (rc0 != HEAT3D_OK) return fail(rc0, "context set-up failed");
    int rc = heat3d_bind_workspace(s.ctx, s.scratch, kNoAllocScratchBytes);  // zeroes the array
    if (rc != HEAT3D_OK) {
      heat3d_destroy(s.ctx);
      s.ctx = nullptr;
      return fail(rc, "binding the scratch array failed");
    }
    s.N = N;
    s.order = order;
    s.precision = precision;
  }
  // The solve itself: the same steps as mg_vcycle, without its timing events
  // (creating an event is a resource allocation this entry point avoids).
  heat3d_ctx* ctx = s.ctx;
  heat3d_set_stream(ctx, stream);
  h3d::SdcLevel& L = ctx->lv[0];
  heat3d_stats loc{};
  ctx->bytes = 0;
  int rc = h3d_load_dense(ctx, 0, rhs, L.abi_p1);
  if (rc == HEAT3D_OK) rc = h3d_load_dense(ctx, 0, u, L.abi_p0);
  const int slot = L.nslots - 1;
  if (rc == HEAT3D_OK) rc = h3d_set_coefs(ctx, 0, slot, 0, 1, &c);
  if (rc == HEAT3D_OK && max_cycles > 0)
    rc = h3d_mg_solve(ctx, 0, slot, 0, 1, L.abi_p0, 0, L.abi_p1, 0, max_cycles, tol, &loc);
  if (rc < 0 && rc != HEAT3D_ENOTCONV) return fail(rc, heat3d_last_error(ctx));
  int rc2 = h3d_store_dense(ctx, 0, L.abi_p0, u);
  if (rc2 < 0) return fail(rc2, heat3d_last_error(ctx));
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess) return fail(HEAT3D_ECUDA, "stream error");
  loc.bytes = ctx->bytes;
  if (stats) *stats = loc;
  return rc;
}

const char* mg_vcycle_noalloc_last_error(void) { return g_err; }

}  // extern "C"
