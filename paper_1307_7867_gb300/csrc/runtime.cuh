// runtime.cuh -- the context structure and the host drivers shared by the
// runtime (runtime.cu), the CUDA-graph layer and the serving loop.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/heat3d.h"
#include "common.cuh"
#include "kernels.cuh"

namespace h3d {

struct MgBufs {
  void* b = nullptr;  // right-hand side of the level's error equation (level 0: the residual)
  void* e = nullptr;  // correction
  void* t = nullptr;  // ping-pong partner of e
};

// One SDC level of the hierarchy with its multigrid levels and its items
// (PFASST slices or independent problems), all of the same grid.
struct SdcLevel {
  heat3d_level L{};
  int B = 0;  // item capacity
  Grid g{};
  int nmg = 0;
  Grid mg[kMaxLevels]{};
  double h[kMaxLevels]{};
  double tau[kMaxNodes]{}, Q[kMaxNodes][kMaxNodes]{}, S[kMaxNodes - 1][kMaxNodes]{};
  // device buffers (workspace); node fields are [item][node] at stride g.fs
  double *U = nullptr, *F = nullptr, *I = nullptr;
  double *tauS = nullptr, *UGr = nullptr, *qF = nullptr, *D = nullptr;  // coarse level only
  // compact stencil only: W U at every node (layout of U), and per item the
  // weighted residual that the FAS restriction's W-solve takes as rhs
  double *WU = nullptr, *Wr = nullptr;
  double *abi_u = nullptr, *abi_b = nullptr, *abi_p0 = nullptr, *abi_p1 = nullptr;
  MgBufs mgb[kMaxLevels];
  double* phi = nullptr;  // sin(pi x_i), i = 1..N
  double* alpha_items = nullptr;
  double* alpha_nodes = nullptr;
  ItemSDC* items_d = nullptr;
  int nslots = 0;   // M - 1 substeps, mg_vcycle calls (slot M - 1), W-solve (slot M)
  void* coefT = nullptr;  // Coef<T>[slot][mg level][item]
  Coef<double>* coef64 = nullptr;  // Coef<double>[slot][item], finest multigrid level
  unsigned long long* norms = nullptr;
  int* active = nullptr;
  // device-side stop rule of the multigrid solves (chunked cycles): per-item
  // tolerance, cycles done and last residual norm; a NaN flag
  double* mg_tol_d = nullptr;
  int* mg_ncyc = nullptr;
  double* mg_last = nullptr;
  int* mg_flag = nullptr;
  // host mirrors
  std::vector<ItemSDC> items_h;
  std::vector<double> t0, nu, dt;
  bool has_tau = false;
  // launch shapes: multigrid kernels of level k in the solve precision, and
  // the FP64 kernels (operator, refinement residual) on the level's grid
  Shape shapeT[kMaxLevels];
  Shape shape64;
  // multigrid levels with N <= fuse_max run as one fused kernel per V-cycle
  // (when fuse_coarse is on); chosen by the autotuner among 15, 7, 3 and 0
  int fuse_max = 15;
  // every solve of this level runs as one persistent kernel (small grids):
  // its norm slots and barrier state
  bool persist = false;
  unsigned long long* pnorm = nullptr;
  int* pctl = nullptr;
};

// A captured chunk of solve cycles (each: V-cycle(s), norm reset, refinement
// residual, device-side stop rule) for one solve key.
struct CycleGraph {
  int lev = 0, slot = 0, b0 = 0, B = 0;
  int inner = 1;  // V-cycles per refinement step in this graph
  const double* u = nullptr;
  const double* rhs = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;  // kernels per replay
  double bytes = 0.0;      // algorithmic bytes per replay
  // profiling of the captured kernel class: event pairs owned by this graph
  int prof_class = 0;
  std::vector<cudaEvent_t> ev;
  double prof_bytes = 0.0, prof_dpops = 0.0, prof_flops = 0.0;
  long long prof_launches = 0;
};

}  // namespace h3d

struct heat3d_ctx {
  heat3d_config cfg{};
  h3d::SdcLevel lv[2];
  h3d::FasMap map{};
  h3d::FasMap* map_d = nullptr;
  cudaStream_t st = nullptr;
  char err[512] = {0};
  void* ws = nullptr;
  size_t ws_bytes = 0, ws_need = 0;
  bool bound = false;
  h3d::Shape shape{};
  double bytes = 0.0;  // algorithmic-bytes counter of the current call
  double t_start = 0.0, T_run = 0.0;  // interval of pfasst_run
  // per-launch CUDA-event timing of one kernel class (heat3d_profile)
  int prof_class = 0;
  std::vector<cudaEvent_t> prof_ev;  // pairs
  size_t prof_used = 0;              // pairs recorded and not yet harvested
  double prof_ms = 0.0, prof_bytes = 0.0, prof_dpops = 0.0, prof_flops = 0.0;
  // fraction of a multigrid launch's items that are still iterating (items
  // that have converged return at once): scales the profiled work
  double work_scale = 1.0;
  long long prof_launches = 0;
  // CUDA graphs of V-cycles (cfg.use_graphs); `capturing` routes profiling
  // events into the graph being captured
  std::vector<h3d::CycleGraph*> graphs;
  h3d::CycleGraph* capturing = nullptr;
};

// Event bracketing for the profiled kernel class: returns a pair index or -1.
int h3d_prof_begin(heat3d_ctx* c, int cls);
void h3d_prof_end(heat3d_ctx* c, int pair, double bytes, double dpops, double flops);

int h3d_fail(heat3d_ctx* c, int code, const char* fmt, ...);
// heat3d_workspace_size that also copies a validation failure's message to msg.
int h3d_workspace_size_msg(const heat3d_config* cfg, size_t* bytes, char* msg, size_t msg_len);
size_t h3d_tsize(const heat3d_ctx* c);
void h3d_fill_item(heat3d_ctx* c, int lev, int item, double t0);
int h3d_upload_items(heat3d_ctx* c, int lev, int b0, int B);
int h3d_set_coefs(heat3d_ctx* c, int lev, int slot, int b0, int B, const double* cvals);
int h3d_set_item_operators(heat3d_ctx* c, int lev, int b0, int B);
// tolv (optional): per-item tolerances for items [b0, b0+B), replacing tol.
int h3d_mg_solve(heat3d_ctx* c, int lev, int slot, int b0, int B, double* u, long long us,
                 const double* rhs, long long bs, int max_cycles, double tol, heat3d_stats* s,
                 const double* tolv = nullptr);
int h3d_eval_F(heat3d_ctx* c, int lev, int b0, int B);
int h3d_residual(heat3d_ctx* c, int lev, int b0, int B, double* res, std::vector<double>* per_item);
int h3d_sweep(heat3d_ctx* c, int lev, int b0, int B, double check_tol, heat3d_stats* s);
int h3d_fas_restrict(heat3d_ctx* c, int b0, int B, heat3d_stats* s = nullptr);
int h3d_fas_interpolate(heat3d_ctx* c, int b0, int B);
int h3d_spread(heat3d_ctx* c, int lev, int b0, int B, const double* u);
int h3d_run(heat3d_ctx* c, double* ucur, heat3d_stats* s);
int h3d_load_dense(heat3d_ctx* c, int lev, const double* src, double* dst_pitched);
int h3d_store_dense(heat3d_ctx* c, int lev, const double* src_pitched, double* dst);
void h3d_destroy_extras(heat3d_ctx* c);
int h3d_autotune(heat3d_ctx* c);
namespace h3d {
long long launches_total();
void launches_adjust(long long delta);
}
