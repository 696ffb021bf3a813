// runtime.cu -- host runtime and C ABI of libheat3d.so.
//
// The context owns the level hierarchy (SDC levels, multigrid levels), the
// collocation tables, per-item step data and the layout of the caller's
// workspace.  The drivers below enqueue the kernels of mg_kernels.cu and
// sdc_kernels.cu on the context's stream:
//   mg_solve   -- residual refinement with V(nu1, nu2) cycles (Sec. 1.2),
//   sweep      -- one IMEX-Euler SDC sweep (Sec. 1.1),
//   fas_*      -- restriction / tau / interpolation between the two levels,
//   run        -- SDC, MLSDC and PFASST over [0, T] (Sec. 1.1).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "../../include/heat3d.h"
#include "kernels.cuh"
#include "runtime.cuh"

using namespace h3d;

// ---------------------------------------------------------------------------
// small utilities
// ---------------------------------------------------------------------------

int h3d_fail(heat3d_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return h3d_fail(c, HEAT3D_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,       \
                      cudaGetErrorString(e_));                                          \
  } while (0)

#define RET(call)                          \
  do {                                     \
    int r_ = (call);                       \
    if (r_ < 0) return r_;                 \
  } while (0)

// Two timing events destroyed on every exit path of the call that made them.
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  EventPair() = default;
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

namespace h3d {
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

long long launches_total() { return g_launches.load(); }
void launches_adjust(long long delta) { g_launches.fetch_add(delta); }
}  // namespace h3d

// Event pair around one launch of the profiled kernel class.  While a
// V-cycle graph is being captured the pair belongs to that graph (and is read
// after each replay); otherwise it comes from the context's pool.
int h3d_prof_begin(heat3d_ctx* c, int cls) {
  if (c->prof_class == 0 || c->prof_class != cls) return -1;
  std::vector<cudaEvent_t>& pool = c->capturing ? c->capturing->ev : c->prof_ev;
  size_t used = c->capturing ? pool.size() / 2 : c->prof_used;
  if (used * 2 + 2 > pool.size()) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      pool.push_back(e);
    }
  }
  int pair = (int)used;
  if (!c->capturing) c->prof_used++;
  // inside a capture only an external record becomes an event-record node
  if (c->capturing) cudaEventRecordWithFlags(pool[2 * pair], c->st, cudaEventRecordExternal);
  else cudaEventRecord(pool[2 * pair], c->st);
  return pair;
}

void h3d_prof_end(heat3d_ctx* c, int pair, double bytes, double dpops, double flops) {
  if (pair < 0) return;
  if (c->capturing) {
    h3d::CycleGraph* g = c->capturing;
    cudaEventRecordWithFlags(g->ev[2 * pair + 1], c->st, cudaEventRecordExternal);
    g->prof_bytes += bytes;
    g->prof_dpops += dpops;
    g->prof_flops += flops;
    g->prof_launches += 1;
    return;
  }
  cudaEventRecord(c->prof_ev[2 * pair + 1], c->st);
  c->prof_bytes += bytes * c->work_scale;
  c->prof_dpops += dpops * c->work_scale;
  c->prof_flops += flops * c->work_scale;
  c->prof_launches += 1;
}

static void prof_harvest(heat3d_ctx* c) {
  cudaStreamSynchronize(c->st);
  for (size_t p = 0; p < c->prof_used; ++p) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[2 * p], c->prof_ev[2 * p + 1]) == cudaSuccess) c->prof_ms += ms;
    else cudaGetLastError();
  }
  c->prof_used = 0;
}

static bool is_pow2m1(int N) { return N >= 1 && ((N + 1) & N) == 0; }

// Gauss-Lobatto nodes on [0, 1] for M = 2..5: the ends and the roots of
// P'_{M-1}, found by Newton's method on P'_{n} from Chebyshev-Lobatto guesses.
static void lobatto_nodes(int M, double* tau) {
  const int n = M - 1;
  tau[0] = 0.0;
  tau[M - 1] = 1.0;
  for (int r = 1; r < n; ++r) {
    double x = -cos(M_PI * r / n);
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;  // P_0, P_1
      for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n, p0 = P_{n-1}
      double dp = n * (x * p1 - p0) / (x * x - 1.0);
      double d2p = (2.0 * x * dp - n * (n + 1) * p1) / (1.0 - x * x);
      double dx = dp / d2p;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    tau[r] = 0.5 * (x + 1.0);
  }
  std::sort(tau, tau + M);
}

// Q[m][j] = int_0^{tau_m} l_j: the weights q solve the moment equations
// sum_j q_j tau_j^p = tau_m^{p+1} / (p+1), p = 0..M-1 (Gaussian elimination).
static void integration_matrix(int M, const double* tau, double Q[kMaxNodes][kMaxNodes]) {
  for (int m = 0; m < M; ++m) {
    double A[kMaxNodes][kMaxNodes + 1];
    for (int p = 0; p < M; ++p) {
      for (int j = 0; j < M; ++j) A[p][j] = pow(tau[j], p);
      A[p][M] = pow(tau[m], p + 1) / (p + 1);
    }
    for (int col = 0; col < M; ++col) {
      int piv = col;
      for (int r = col + 1; r < M; ++r)
        if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
      for (int k = 0; k <= M; ++k) std::swap(A[col][k], A[piv][k]);
      for (int r = 0; r < M; ++r) {
        if (r == col) continue;
        double f = A[r][col] / A[col][col];
        for (int k = col; k <= M; ++k) A[r][k] -= f * A[col][k];
      }
    }
    for (int j = 0; j < M; ++j) Q[m][j] = (m == 0) ? 0.0 : A[j][M] / A[j][j];
  }
}

static double kappa_of(int forcing) {
  return forcing == HEAT3D_FORCING_EXACT ? 3.0 : 1.0;
}

// ---------------------------------------------------------------------------
// context set-up
// ---------------------------------------------------------------------------

static int validate(heat3d_ctx* c, const heat3d_config* cfg) {
  if (!cfg) return h3d_fail(c, HEAT3D_EINVAL, "null config");
  if (cfg->nlevels < 1 || cfg->nlevels > 2) return h3d_fail(c, HEAT3D_EINVAL, "nlevels must be 1 or 2");
  for (int l = 0; l < cfg->nlevels; ++l) {
    const heat3d_level& L = cfg->levels[l];
    if (!is_pow2m1(L.N) || L.N > (1 << 10) - 1)
      return h3d_fail(c, HEAT3D_EINVAL, "level %d: N=%d must be 2^k-1 (<= 1023)", l, L.N);
    if (L.order != 2 && L.order != 4 && L.order != kCompact)
      return h3d_fail(c, HEAT3D_EINVAL, "level %d: order must be 2, 4 or HEAT3D_COMPACT", l);
    if (l == 1 && L.order == kCompact)
      return h3d_fail(c, HEAT3D_EINVAL, "the compact stencil is for the fine level only");
    if (L.M < 2 || L.M > kMaxNodes) return h3d_fail(c, HEAT3D_EINVAL, "level %d: M must be 2..5", l);
  }
  if (cfg->nlevels == 2) {
    const heat3d_level &F = cfg->levels[0], &G = cfg->levels[1];
    if (!(F.N == G.N || F.N == 2 * G.N + 1))
      return h3d_fail(c, HEAT3D_EINVAL, "coarse N must equal fine N or (fine N - 1)/2");
  }
  if (!(cfg->nu > 0) || !(cfg->dt > 0)) return h3d_fail(c, HEAT3D_EINVAL, "nu and dt must be > 0");
  if (cfg->mg.nu1 < 1 || cfg->mg.nu2 < 0 || cfg->mg.max_cycles < 1)
    return h3d_fail(c, HEAT3D_EINVAL, "multigrid needs nu1 >= 1, nu2 >= 0, max_cycles >= 1");
  if (!(cfg->mg.rel >= 0 && cfg->mg.rel < 1))
    return h3d_fail(c, HEAT3D_EINVAL, "mg.rel must lie in [0, 1)");
  if (cfg->interp != 0 && cfg->interp != 2 && cfg->interp != 4 && cfg->interp != 6 &&
      cfg->interp != 8)
    return h3d_fail(c, HEAT3D_EINVAL, "interp must be 2 (trilinear), 4, 6 or 8 (midpoint rules)");
  if (cfg->persistent < -1 || cfg->persistent > 1)
    return h3d_fail(c, HEAT3D_EINVAL, "persistent must be -1 (automatic), 0 or 1");
  if (cfg->precision != HEAT3D_FP64 && cfg->precision != HEAT3D_MIXED)
    return h3d_fail(c, HEAT3D_EINVAL, "precision must be HEAT3D_FP64 or HEAT3D_MIXED");
  if (cfg->slices < 1 || cfg->sweeps_fine < 0 || cfg->sweeps_coarse < 0 || cfg->iters < 0)
    return h3d_fail(c, HEAT3D_EINVAL, "slices >= 1 and non-negative sweep/iteration counts required");
  return HEAT3D_OK;
}

static int setup_levels(heat3d_ctx* c) {
  const heat3d_config& cfg = c->cfg;
  int cap = std::max(std::max(cfg.batch, cfg.slices), 1);
  for (int l = 0; l < cfg.nlevels; ++l) {
    SdcLevel& L = c->lv[l];
    L.L = cfg.levels[l];
    L.B = cap;
    L.g = make_grid(L.L.N);
    L.nmg = 0;
    for (int n = L.L.N;; n = (n - 1) / 2) {
      L.mg[L.nmg] = make_grid(n);
      L.h[L.nmg] = 1.0 / (n + 1);
      L.nmg++;
      if (n == 1) break;
    }
    lobatto_nodes(L.L.M, L.tau);
    integration_matrix(L.L.M, L.tau, L.Q);
    for (int m = 0; m + 1 < L.L.M; ++m)
      for (int j = 0; j < L.L.M; ++j) L.S[m][j] = L.Q[m + 1][j] - L.Q[m][j];
    L.items_h.assign(cap, ItemSDC{});
    L.t0.assign(cap, 0.0);
    L.nu.assign(cap, cfg.nu);
    L.dt.assign(cap, cfg.dt);
  }
  if (cfg.nlevels == 2) {
    SdcLevel &F = c->lv[0], &G = c->lv[1];
    for (int m = 0; m < G.L.M; ++m) {
      int jm = -1;
      for (int j = 0; j < F.L.M; ++j)
        if (fabs(F.tau[j] - G.tau[m]) < 1e-13) jm = j;
      if (jm < 0) return h3d_fail(c, HEAT3D_EINVAL, "coarse nodes must be a subset of the fine nodes");
      c->map.jm[m] = jm;
    }
    for (int j = 0; j < F.L.M; ++j)
      for (int m = 0; m < G.L.M; ++m) {
        double v = 1.0;
        for (int i = 0; i < G.L.M; ++i)
          if (i != m) v *= (F.tau[j] - G.tau[i]) / (G.tau[m] - G.tau[i]);
        c->map.L[j][m] = v;
      }
  }
  return HEAT3D_OK;
}

size_t h3d_tsize(const heat3d_ctx* c) { return c->cfg.precision == HEAT3D_MIXED ? 4 : 8; }

// Lays out every device buffer in the workspace; with base == nullptr only
// measures.  Returns the byte count.
static size_t plan(heat3d_ctx* c, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    off = (off + 255) / 256 * 256;
    void* p = base ? (void*)(base + off) : nullptr;
    off += bytes;
    return p;
  };
  const size_t ts = h3d_tsize(c);
  for (int l = 0; l < c->cfg.nlevels; ++l) {
    SdcLevel& L = c->lv[l];
    const int M = L.L.M, B = L.B;
    const size_t fs = (size_t)L.g.fs * 8;
    L.U = (double*)take(fs * B * M);
    L.F = (double*)take(fs * B * M);
    L.I = (double*)take(fs * B * (M - 1));
    if (L.L.order == kCompact) {
      L.WU = (double*)take(fs * B * M);
      L.Wr = (double*)take(fs * B);
    }
    if (l == 1) {
      L.tauS = (double*)take(fs * B * (M - 1));
      L.UGr = (double*)take(fs * B * M);
      L.qF = (double*)take(fs * B * M);
      L.D = (double*)take(fs * B * c->lv[0].L.M);
    }
    L.abi_u = (double*)take(fs);
    L.abi_b = (double*)take(fs);
    L.abi_p0 = (double*)take(fs);
    L.abi_p1 = (double*)take(fs);
    for (int k = 0; k < L.nmg; ++k) {
      size_t f = (size_t)L.mg[k].fs * ts * B;
      L.mgb[k].b = take(f);
      L.mgb[k].e = take(f);
      L.mgb[k].t = take(f);
    }
    L.phi = (double*)take(sizeof(double) * L.L.N);
    L.alpha_items = (double*)take(sizeof(double) * B);
    L.alpha_nodes = (double*)take(sizeof(double) * B * M);
    L.items_d = (ItemSDC*)take(sizeof(ItemSDC) * B);
    L.nslots = M + 1;  // M-1 substeps, one slot for mg_vcycle calls, one for the W-solve
    L.coefT = take((ts == 8 ? sizeof(Coef<double>) : sizeof(Coef<float>)) * L.nslots * L.nmg * B);
    L.coef64 = (Coef<double>*)take(sizeof(Coef<double>) * L.nslots * B);
    L.norms = (unsigned long long*)take(sizeof(unsigned long long) * B);
    L.active = (int*)take(sizeof(int) * B);
    L.mg_tol_d = (double*)take(sizeof(double) * B);
    L.mg_ncyc = (int*)take(sizeof(int) * B);
    L.mg_last = (double*)take(sizeof(double) * B);
    L.mg_flag = (int*)take(sizeof(int) * 2);  // NaN flag, cycle cap
    L.pnorm = (unsigned long long*)take(sizeof(unsigned long long) * 2 * B);
    L.pctl = (int*)take(sizeof(int) * 4);
  }
  c->map_d = (FasMap*)take(sizeof(FasMap));
  off = (off + 255) / 256 * 256;
  return off;
}

// Per-item step data: dt S, dt Q, forcing integrals and the substep lengths.
void h3d_fill_item(heat3d_ctx* c, int lev, int item, double t0) {
  SdcLevel& L = c->lv[lev];
  const int M = L.L.M;
  const double dt = L.dt[item], nu = L.nu[item];
  const bool forced = c->cfg.forcing != HEAT3D_FORCING_NONE;
  const double kap = kappa_of(c->cfg.forcing);
  // compact stencil: the weighted system carries W f = g(t) W Phi, and Phi is
  // an eigenvector of W with eigenvalue (3 + 3 cos(pi h)) / 6
  const double wphi = L.L.order == kCompact ? (3.0 + 3.0 * cos(M_PI * L.h[0])) / 6.0 : 1.0;
  double g[kMaxNodes];
  for (int j = 0; j < M; ++j) {
    double t = t0 + dt * L.tau[j];
    g[j] = forced ? -(sin(t) - kap * nu * M_PI * M_PI * cos(t)) * wphi : 0.0;
  }
  ItemSDC& it = L.items_h[item];
  memset(&it, 0, sizeof(it));
  it.nu = nu;
  for (int m = 0; m + 1 < M; ++m) {
    it.dtm[m] = dt * (L.tau[m + 1] - L.tau[m]);
    double s = 0.0;
    for (int j = 0; j < M; ++j) {
      it.dtS[m][j] = dt * L.S[m][j];
      s += it.dtS[m][j] * g[j];
    }
    it.gS[m] = s;
  }
  for (int m = 0; m < M; ++m) {
    double s = 0.0;
    for (int j = 0; j < M; ++j) {
      it.dtQ[m][j] = dt * L.Q[m][j];
      s += it.dtQ[m][j] * g[j];
    }
    it.gQ[m] = s;
  }
  L.t0[item] = t0;
}

int h3d_upload_items(heat3d_ctx* c, int lev, int b0, int B) {
  SdcLevel& L = c->lv[lev];
  CK(cudaMemcpyAsync(L.items_d + b0, L.items_h.data() + b0, sizeof(ItemSDC) * B,
                     cudaMemcpyHostToDevice, c->st));
  return HEAT3D_OK;
}

// Multigrid coefficients of A = W - c Delta_h on every level (W = I but for
// the compact stencil), for slot `slot`
// of items [b0, b0 + B) with per-item c values.
int h3d_set_coefs(heat3d_ctx* c, int lev, int slot, int b0, int B, const double* cvals) {
  SdcLevel& L = c->lv[lev];
  const int order = L.L.order;
  const bool f32 = h3d_tsize(c) == 4;
  std::vector<Coef<double>> c64(B);
  std::vector<Coef<double>> cd((size_t)L.nmg * B);
  for (int k = 0; k < L.nmg; ++k) {
    const double h = L.h[k];
    for (int b = 0; b < B; ++b) {
      const Coef<double> q =
          mg_level_coef(order, cvals[b], h, k > 0 ? cd[(size_t)(k - 1) * B + b].wd : 0.0);
      cd[(size_t)k * B + b] = q;
      if (k == 0) c64[b] = q;
    }
  }
  CK(cudaMemcpyAsync(L.coef64 + (size_t)slot * L.B + b0, c64.data(), sizeof(Coef<double>) * B,
                     cudaMemcpyHostToDevice, c->st));
  for (int k = 0; k < L.nmg; ++k) {
    size_t base = ((size_t)slot * L.nmg + k) * L.B + b0;
    if (f32) {
      std::vector<Coef<float>> cf(B);
      for (int b = 0; b < B; ++b) {
        const Coef<double>& q = cd[(size_t)k * B + b];
        cf[b] = Coef<float>{(float)q.d,  (float)q.e,  (float)q.wd,  (float)q.a11,
                            (float)q.e2, (float)q.al, (float)q.om,  (float)q.be,
                            (float)q.be2, (float)q.rs, (float)q.a11w};
      }
      CK(cudaMemcpyAsync((Coef<float>*)L.coefT + base, cf.data(), sizeof(Coef<float>) * B,
                         cudaMemcpyHostToDevice, c->st));
    } else {
      CK(cudaMemcpyAsync((Coef<double>*)L.coefT + base, cd.data() + (size_t)k * B,
                         sizeof(Coef<double>) * B, cudaMemcpyHostToDevice, c->st));
    }
  }
  return HEAT3D_OK;
}

// Substep coefficients c = dt_m nu of items [b0, b0+B) for every substep slot,
// plus alpha = nu / h^2 (or nu / (12 h^2)) for the operator kernels.
int h3d_set_item_operators(heat3d_ctx* c, int lev, int b0, int B) {
  SdcLevel& L = c->lv[lev];
  const int M = L.L.M;
  std::vector<double> cv(B);
  for (int m = 0; m + 1 < M; ++m) {
    for (int b = 0; b < B; ++b) cv[b] = L.dt[b0 + b] * (L.tau[m + 1] - L.tau[m]) * L.nu[b0 + b];
    RET(h3d_set_coefs(c, lev, m, b0, B, cv.data()));
  }
  if (L.L.order == kCompact) {  // the weighting matrix W = A at c = 0
    for (int b = 0; b < B; ++b) cv[b] = 0.0;
    RET(h3d_set_coefs(c, lev, M, b0, B, cv.data()));
  }
  const double h = L.h[0];
  std::vector<double> ai(B), an((size_t)B * M);
  for (int b = 0; b < B; ++b) {
    double nu = L.nu[b0 + b];
    ai[b] = L.L.order == 2 ? nu / (h * h) : L.L.order == 4 ? nu / (12.0 * h * h) : nu / (6.0 * h * h);
    for (int m = 0; m < M; ++m) an[(size_t)b * M + m] = ai[b];
  }
  CK(cudaMemcpyAsync(L.alpha_items + b0, ai.data(), sizeof(double) * B, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(L.alpha_nodes + (size_t)b0 * M, an.data(), sizeof(double) * B * M,
                     cudaMemcpyHostToDevice, c->st));
  return HEAT3D_OK;
}

// ---------------------------------------------------------------------------
// multigrid (Sec. 1.2): residual refinement with V-cycles on the error
// ---------------------------------------------------------------------------

template <typename T>
static T* mgbuf(SdcLevel& L, int k, int which, int b0) {
  void* p = which == 0 ? L.mgb[k].b : which == 1 ? L.mgb[k].e : L.mgb[k].t;
  return (T*)p + (size_t)b0 * L.mg[k].fs;
}

template <typename T>
static const Coef<T>* coefT(SdcLevel& L, int slot, int k, int b0) {
  return (const Coef<T>*)L.coefT + ((size_t)slot * L.nmg + k) * L.B + b0;
}

// One V(nu1, nu2) cycle on level k for the error equation A e = b_k, every
// level holding its scaled right-hand side b' = wd b (slot 0; see Coef): on
// the finest level the FP64 residual kernel wrote it, on the others the
// restriction.  b' is also the first Jacobi iterate (the sweep from zero) and
// is never written during the cycle; the iterates alternate between slots 1
// and 2.  On level 0 the last post-smoothing sweep adds its result to u64.
// Returns the buffer holding the level's correction (nullptr on level 0).
// Algorithmic cost per point of one damped-Jacobi sweep (bytes, FP64 pipe
// operations, flops); `upd` adds the result to the FP64 solution; `same`: the
// iterate is b' itself (the sweep after the one from zero), read once.
template <typename T>
static void jacobi_cost(int order, bool upd, bool same, double* bytes, double* dp, double* fl) {
  const double ts = sizeof(T);
  // neighbour sums + fused multiply-adds (an FMA counts 2 flops)
  const double ops = order == 2 ? 7.0 : order == 4 ? 13.0 : 19.0;
  const double flops = order == 2 ? 9.0 : order == 4 ? 16.0 : 22.0;
  *bytes = (upd ? ts + 16.0 : 2.0 * ts) + (same ? 0.0 : ts);
  *dp = (sizeof(T) == 8 ? ops : 0.0) + (upd ? 1.0 : 0.0);
  *fl = flops + (upd ? 1.0 : 0.0);
}

template <typename T>
static int vcycle_level(heat3d_ctx* c, SdcLevel& L, int slot, int k, int b0, int B,
                        const int* act, double* u64, long long us, T** result, bool warm = false,
                        bool final = true) {
  // Level 0 options: `warm` starts from the correction in *result (else from
  // b' itself); `final` adds the correction to u64 in the last post-smoothing
  // sweep (else *result returns its buffer).
  const bool prof_here = k == 0 && &L == &c->lv[0];
  const Grid& g = L.mg[k];
  const int order = L.L.order;
  const int nu1 = c->cfg.mg.nu1, nu2 = c->cfg.mg.nu2;
  cudaStream_t st = c->st;
  T* bp = mgbuf<T>(L, k, 0, b0);
  T* e = mgbuf<T>(L, k, 1, b0);
  T* t = mgbuf<T>(L, k, 2, b0);
  const Coef<T>* cf = coefT<T>(L, slot, k, b0);
  const size_t ts = sizeof(T), pts = (size_t)g.N * g.N * g.N * B;
  if (k > 0 && c->cfg.fuse_coarse && g.N <= std::min(L.fuse_max, kFusedMaxN) &&
      L.L.order != kCompact) {
    // this level and every coarser one in a single kernel (same arithmetic)
    int Ns[kMaxLevels];
    const Coef<T>* cfs[kMaxLevels];
    const int nl = L.nmg - k;
    for (int l = 0; l < nl; ++l) {
      Ns[l] = L.mg[k + l].N;
      cfs[l] = coefT<T>(L, slot, k + l, b0);
    }
    CK(launch_vcycle_small<T>(order, nl, Ns, cfs, B, bp, e, g, nu1, nu2, act, st));
    c->bytes += 2.0 * ts * pts;
    *result = e;
    return HEAT3D_OK;
  }
  if (g.N == 1) {
    CK(launch_solve_one<T>(g, B, bp, e, cf, act, st));
    if (k == 0 && final) {
      CK(launch_update<T>(g, B, e, u64, us, act, st));
      *result = nullptr;
    } else {
      *result = e;
    }
    return HEAT3D_OK;
  }
  T* cur = bp;
  T* oth = e;
  int first = 1;
  if (k == 0 && warm) {
    cur = *result;
    oth = cur == e ? t : e;
    first = 0;
  }
  // after a sweep cur -> oth: the iterates then alternate between e and t
  auto advance = [&]() {
    if (cur == bp) {
      cur = oth;
      oth = oth == e ? t : e;
    } else {
      std::swap(cur, oth);
    }
  };
  // profiled fine-level Jacobi launches: all of them, or those that store the
  // error without the FP64 update
  auto prof_jacobi = [&](bool upd) {
    if (!prof_here) return -1;
    const int pr = h3d_prof_begin(c, HEAT3D_PROF_JACOBI_FINE);
    return pr >= 0 || upd ? pr : h3d_prof_begin(c, HEAT3D_PROF_JACOBI_FINE_STORE);
  };
  for (int s = first; s < nu1; ++s) {
    int pr = prof_jacobi(false);
    CK(launch_jacobi<T>(order, g, B, cur, bp, oth, nullptr, 0, cf, act, L.shapeT[k], st));
    double cb, cd, cfl;
    jacobi_cost<T>(order, false, cur == bp, &cb, &cd, &cfl);
    if (pr >= 0) h3d_prof_end(c, pr, cb * pts, cd * pts, cfl * pts);
    c->bytes += cb * pts;
    advance();
  }
  CK(launch_resid<T>(order, g, B, cur, bp, oth, cf, act, L.shapeT[k], st));
  CK(launch_restrict<T>(g, L.mg[k + 1], B, oth, mgbuf<T>(L, k + 1, 0, b0),
                        coefT<T>(L, slot, k + 1, b0), act, st));
  c->bytes += 3.0 * ts * pts + ts * pts * (1.0 + 1.0 / 8.0);
  T* ce = nullptr;
  RET(vcycle_level<T>(c, L, slot, k + 1, b0, B, act, u64, us, &ce));
  // prolongation into the iterate, or (no pre-smoothing sweep ran) from b'
  // into the free buffer that held the restricted residual
  T* dst = cur == bp ? oth : cur;
  CK(launch_prolong_add<T>(L.mg[k + 1], g, B, ce, L.mg[k + 1].fs, cur, dst, g.fs, act, st));
  c->bytes += ts * pts * (2.0 + 1.0 / 8.0);
  if (cur == bp) {
    cur = dst;
    oth = dst == e ? t : e;
  }
  for (int s = 0; s < nu2; ++s) {
    const bool upd = k == 0 && final && s == nu2 - 1;
    int pr = prof_jacobi(upd);
    if (upd) CK(launch_jacobi<T>(order, g, B, cur, bp, nullptr, u64, us, cf, act, L.shapeT[k], st));
    else CK(launch_jacobi<T>(order, g, B, cur, bp, oth, nullptr, 0, cf, act, L.shapeT[k], st));
    if (pr >= 0) {
      double cb, cd, cfl;
      jacobi_cost<T>(order, upd, false, &cb, &cd, &cfl);
      h3d_prof_end(c, pr, cb * pts, cd * pts, cfl * pts);
    }
    if (upd) {
      c->bytes += (2.0 * ts + 16.0) * pts;
      *result = nullptr;
      return HEAT3D_OK;
    }
    c->bytes += 3.0 * ts * pts;
    std::swap(cur, oth);
  }
  if (k == 0 && final) {
    CK(launch_update<T>(g, B, cur, u64, us, act, st));
    c->bytes += (ts + 16.0) * pts;
    *result = nullptr;
  } else {
    *result = cur;
  }
  return HEAT3D_OK;
}

static int read_norms(heat3d_ctx* c, SdcLevel& L, int b0, int B, std::vector<double>& out) {
  std::vector<unsigned long long> h(B);
  CK(cudaMemcpyAsync(h.data(), L.norms + b0, sizeof(unsigned long long) * B,
                     cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  out.resize(B);
  for (int b = 0; b < B; ++b) {
    unsigned long long v = h[b];
    double d;
    memcpy(&d, &v, 8);
    out[b] = d;  // NaN/Inf keep their bit patterns
  }
  return HEAT3D_OK;
}

// Solve (I - c_b Delta_h) u_b = rhs_b for items [b0, b0 + B) of level lev, u
// warm-started and updated in place (item strides us, bs).  Coefficients of
// slot `slot` must be set.  Returns ENOTCONV / ENAN per the tolerance rule.
// ---- CUDA graphs of one V-cycle + refinement residual ----

static bool graphs_usable(heat3d_ctx* c) {
  return c->cfg.use_graphs && c->st != nullptr && c->st != cudaStreamLegacy &&
         c->st != cudaStreamPerThread;
}

static CycleGraph* find_graph(heat3d_ctx* c, int lev, int slot, int b0, int B, const double* u,
                              const double* rhs, int inner) {
  for (CycleGraph* g : c->graphs)
    if (g->lev == lev && g->slot == slot && g->b0 == b0 && g->B == B && g->u == u && g->rhs == rhs &&
        g->inner == inner)
      return g;
  return nullptr;
}

static void free_graph(CycleGraph* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  delete g;
}

static void drop_graph(heat3d_ctx* c, CycleGraph* g) {
  c->graphs.erase(std::find(c->graphs.begin(), c->graphs.end(), g));
  free_graph(g);
}

// Adds the profiled launches of one completed replay.
static void graph_harvest(heat3d_ctx* c, CycleGraph* g) {
  for (size_t p = 0; p + 1 < g->ev.size(); p += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g->ev[p], g->ev[p + 1]) == cudaSuccess) c->prof_ms += ms;
    else cudaGetLastError();  // a failed timing read must not fail the next launch
  }
  c->prof_bytes += g->prof_bytes * c->work_scale;
  c->prof_dpops += g->prof_dpops * c->work_scale;
  c->prof_flops += g->prof_flops * c->work_scale;
  // launches that did work: a chunk's cycles after convergence skip every item
  c->prof_launches += llround(g->prof_launches * c->work_scale);
}

// Captures fn() (the kernels of one chunk of cycles) into a new graph for this key.  The
// launches and bytes it enqueues are recorded per replay instead of now.
template <typename Fn>
static int capture_graph(heat3d_ctx* c, int lev, int slot, int b0, int B, const double* u,
                         const double* rhs, int inner, Fn& fn, CycleGraph** out) {
  CycleGraph* g = new CycleGraph();
  g->lev = lev; g->slot = slot; g->b0 = b0; g->B = B; g->u = u; g->rhs = rhs; g->inner = inner;
  g->prof_class = c->prof_class;
  const long long l0 = h3d::launches_total();
  const double by0 = c->bytes;
  cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    delete g;
    return h3d_fail(c, HEAT3D_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  }
  c->capturing = g;
  int rc = fn();
  c->capturing = nullptr;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(c->st, &graph);
  g->launches = h3d::launches_total() - l0;
  h3d::launches_adjust(-g->launches);
  g->bytes = c->bytes - by0;
  c->bytes = by0;
  if (rc < 0 || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    free_graph(g);
    return rc < 0 ? rc : h3d_fail(c, HEAT3D_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    free_graph(g);
    return h3d_fail(c, HEAT3D_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  c->graphs.push_back(g);
  *out = g;
  return HEAT3D_OK;
}

// Stats and return code of a solve whose stop rule ran on the device: per
// item the cycles done, the last residual norm and its tolerance.
// vcycles >= 0: the V-cycles done when the refinement steps did not all
// take `inner` of them.
static int solve_outcome(heat3d_ctx* c, int lev, int B, int inner, bool fixed, double tol,
                         int max_cycles, const std::vector<double>& tl,
                         const std::vector<int>& hcyc, const std::vector<double>& last, int nan,
                         heat3d_stats* s, long long vcycles = -1) {
  if (nan) return h3d_fail(c, HEAT3D_ENAN, "NaN/Inf residual in a multigrid solve");
  long long total = 0;
  double mx = 0;
  int notconv = 0;
  for (int b = 0; b < B; ++b) {
    total += hcyc[b];
    mx = std::max(mx, last[b]);
    if (!fixed && !(last[b] <= tl[b])) ++notconv;
  }
  if (vcycles < 0) vcycles = total * inner;
  if (s) {
    s->vcycles += vcycles;
    s->vcycles_level[lev] += vcycles;
    s->solves += B;
    s->mg_residual = mx;
  }
  if (notconv > 0) {
    if (s) s->notconv += notconv;
    return h3d_fail(c, HEAT3D_ENOTCONV, "multigrid: %d item(s) above tol %.3g after %d cycles",
                    notconv, tol, max_cycles);
  }
  return HEAT3D_OK;
}

// Algorithmic bytes of one item's refinement step (inner V-cycles and the
// FP64 residual) in the persistent kernel: the launch sequence's operations,
// with the levels from N <= 7 down in shared memory.
template <typename T>
static double persist_step_bytes(const SdcLevel& L, int inner, int nu1, int nu2) {
  const double ts = sizeof(T);
  int kb = 1;
  while (kb < L.nmg && L.mg[kb].N > 7) ++kb;
  double by = 0.0;
  for (int q = 0; q < inner; ++q) {
    const bool warm = q > 0, final = q == inner - 1;
    for (int k = 0; k < kb; ++k) {
      const double n = (double)L.mg[k].N * L.mg[k].N * L.mg[k].N;
      // warm: nu1 sweeps; cold: nu1 - 1 launched sweeps, the first reading b'
      // once as both iterate and right-hand side
      by += (k == 0 && warm) ? nu1 * 3.0 * ts * n
                             : (nu1 > 1 ? 2.0 * ts * n + (nu1 - 2) * 3.0 * ts * n : 0.0);
      by += 3.0 * ts * n + ts * n * (1.0 + 1.0 / 8.0);
      by += ts * n * (2.0 + 1.0 / 8.0);
      for (int s = 0; s < nu2; ++s) by += (k == 0 && final && s == nu2 - 1) ? (2.0 * ts + 16.0) * n : 3.0 * ts * n;
      if (k == 0 && final && nu2 == 0) by += (ts + 16.0) * n;
    }
    const double nb = (double)L.mg[kb].N * L.mg[kb].N * L.mg[kb].N;
    by += 2.0 * ts * nb;
  }
  const double n0 = (double)L.mg[0].N * L.mg[0].N * L.mg[0].N;
  return by + (16.0 + ts) * n0;
}

template <typename T>
static int mg_solve_T(heat3d_ctx* c, int lev, int slot, int b0, int B, double* u, long long us,
                      const double* rhs, long long bs, int max_cycles, double tol,
                      const double* tolv, heat3d_stats* s) {
  SdcLevel& L = c->lv[lev];
  const Grid& g = L.mg[0];
  const int order = L.L.order;
  cudaStream_t st = c->st;
  int* act = L.active + b0;
  std::vector<int> ha(B, 1);
  CK(cudaMemcpyAsync(act, ha.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
  T* bp = mgbuf<T>(L, 0, 0, b0);  // b' = wd r, written by the FP64 residual
  const Coef<T>* cf = coefT<T>(L, slot, 0, b0);
  const Coef<double>* c64 = L.coef64 + (size_t)slot * L.B + b0;
  const double pts = (double)g.N * g.N * g.N * B;
  const bool fixed = tol < 0;
  std::vector<double> nrm;
  auto residual = [&]() -> int {
    CK(cudaMemsetAsync(L.norms + b0, 0, sizeof(unsigned long long) * B, st));
    int pr = lev == 0 ? h3d_prof_begin(c, HEAT3D_PROF_RESID64_FINE) : -1;
    CK(launch_resid64<T>(order, g, B, u, us, rhs, bs, c64, bp, cf, L.norms + b0, act, L.shape64, st));
    if (pr >= 0) {
      // neighbour sums + 2 FMAs (+ the FP64 b' multiply when T is double)
      double dp = (order == 2 ? 7.0 : order == 4 ? 13.0 : 19.0) + (sizeof(T) == 8 ? 1.0 : 0.0);
      double fl = (order == 2 ? 9.0 : order == 4 ? 16.0 : 22.0) + 1.0;
      h3d_prof_end(c, pr, (16.0 + sizeof(T)) * pts, dp * pts, fl * pts);
    }
    c->bytes += (16.0 + sizeof(T)) * pts;
    return HEAT3D_OK;
  };
  // inner = 0 (mixed precision, tolerance solves): the number of FP32
  // V-cycles per FP64 residual is chosen per refinement step on the host from
  // the residuals seen so far (graph path, one step per replay); the other
  // paths and fixed-count solves take 3.
  const bool adaptive = c->cfg.mg.inner == 0 && sizeof(T) == 4 && tol >= 0;
  const int inner = adaptive ? 3 : std::max(1, c->cfg.mg.inner);
  if (L.persist) {
    // the whole solve in one persistent kernel (same cycles and results)
    std::vector<double> tl(B);
    for (int b = 0; b < B; ++b) tl[b] = fixed ? -1.0 : (tolv ? tolv[b] : tol);
    CK(cudaMemcpyAsync(L.mg_tol_d + b0, tl.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(L.mg_ncyc + b0, 0, sizeof(int) * B, st));
    CK(cudaMemsetAsync(L.mg_flag, 0, sizeof(int), st));
    MgPersist<T> p{};
    p.nlev = L.nmg;
    for (int k = 0; k < L.nmg; ++k) {
      p.g[k] = L.mg[k];
      p.b[k] = mgbuf<T>(L, k, 0, b0);
      p.e[k] = mgbuf<T>(L, k, 1, b0);
      p.t[k] = mgbuf<T>(L, k, 2, b0);
      p.cf[k] = coefT<T>(L, slot, k, b0);
    }
    p.c64 = c64;
    p.u = u;
    p.us = us;
    p.rhs = rhs;
    p.bs = bs;
    p.B = B;
    p.nu1 = c->cfg.mg.nu1;
    p.nu2 = c->cfg.mg.nu2;
    p.inner = inner;
    p.max_cycles = max_cycles;
    p.norm2 = L.pnorm;
    p.active = act;
    p.ncyc = L.mg_ncyc + b0;
    p.last = L.mg_last + b0;
    p.tol = L.mg_tol_d + b0;
    p.nan_flag = L.mg_flag;
    p.ctl = L.pctl;
    CK(launch_mg_persist<T>(order, p, st));
    std::vector<int> hcyc(B);
    std::vector<double> last(B);
    int hnan = 0, hctl[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(hcyc.data(), L.mg_ncyc + b0, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(last.data(), L.mg_last + b0, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hnan, L.mg_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hctl, L.pctl, sizeof(hctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hctl[1])  // the barrier's error word
      return h3d_fail(c, HEAT3D_ETIMEOUT, "persistent multigrid solve: a grid barrier gave up waiting");
    long long done = 0;
    for (int b = 0; b < B; ++b) done += hcyc[b];
    c->bytes += (double)done * persist_step_bytes<T>(L, inner, c->cfg.mg.nu1, c->cfg.mg.nu2) +
                (16.0 + sizeof(T)) * pts;
    return solve_outcome(c, lev, B, inner, fixed, tol, max_cycles, tl, hcyc, last, hnan, s);
  }
  int nin = inner;  // V-cycles of the next refinement step
  auto one_cycle = [&]() -> int {
    T* cur = nullptr;
    for (int q = 0; q < nin; ++q)
      RET(vcycle_level<T>(c, L, slot, 0, b0, B, act, u, us, &cur, q > 0, q == nin - 1));
    return residual();
  };
  if (graphs_usable(c)) {
    // Chunked cycles: the stop rule runs on the device after every residual
    // (launch_mg_check turns converged items off, so the kernels of later
    // cycles skip them), and the host synchronises once per chunk of cycles:
    // the same cycles as checking after each one.  Small grids take chunks
    // of 4 (their cycles are short against a host round trip), large grids 1.
    const int chunk = g.N >= 127 || adaptive ? 1 : 4;
    std::vector<double> tl(B);
    for (int b = 0; b < B; ++b) tl[b] = fixed ? -1.0 : (tolv ? tolv[b] : tol);
    const int hdr[2] = {0, max_cycles};
    CK(cudaMemcpyAsync(L.mg_tol_d + b0, tl.data(), sizeof(double) * B, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(L.mg_flag, hdr, sizeof(hdr), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(L.mg_ncyc + b0, 0, sizeof(int) * B, st));
    RET(residual());
    CK(launch_mg_check(B, L.norms + b0, act, L.mg_tol_d + b0, L.mg_ncyc + b0, L.mg_last + b0,
                       L.mg_flag + 1, L.mg_flag, true, st));
    auto chunk_fn = [&]() -> int {
      for (int q = 0; q < chunk; ++q) {
        RET(one_cycle());
        CK(launch_mg_check(B, L.norms + b0, act, L.mg_tol_d + b0, L.mg_ncyc + b0, L.mg_last + b0,
                           L.mg_flag + 1, L.mg_flag, false, st));
      }
      return HEAT3D_OK;
    };
    std::vector<int> hact(B), hcyc(B, 0), prev(B, 0);
    std::vector<double> lastv(B), lastp(B);
    // adaptive: the worst active item's residual over its tolerance, and the
    // contraction per FP32 V-cycle seen in the previous step (start 0.2)
    double rho = 0.2;
    if (adaptive) {
      CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(lastv.data(), L.mg_last + b0, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    int launched = 0;
    long long vdone = 0;
    for (;;) {
      if (adaptive) {
        double q = 1.0;
        for (int b = 0; b < B; ++b)
          if (hact[b] && tl[b] > 0) q = std::max(q, lastv[b] / tl[b]);
        // cycles to reach the tolerance at the observed contraction, 1 to 4
        // (an FP32 error equation gains about 6 digits per refinement step)
        const double need = std::log(std::min(q, 1e6)) / -std::log(rho);
        nin = std::max(1, std::min(4, (int)std::ceil(need - 1e-9)));
        lastp = lastv;
      }
      CycleGraph* gph = find_graph(c, lev, slot, b0, B, u, rhs, nin);
      if (gph && gph->prof_class != c->prof_class) {
        drop_graph(c, gph);
        gph = nullptr;
      }
      if (!gph) RET(capture_graph(c, lev, slot, b0, B, u, rhs, nin, chunk_fn, &gph));
      CK(cudaGraphLaunch(gph->exec, st));
      h3d::launches_adjust(gph->launches);
      launched += chunk;
      CK(cudaMemcpyAsync(hact.data(), act, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(hcyc.data(), L.mg_ncyc + b0, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
      if (adaptive)
        CK(cudaMemcpyAsync(lastv.data(), L.mg_last + b0, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      long long done = 0;
      for (int b = 0; b < B; ++b) done += hcyc[b] - prev[b];
      vdone += done * nin;
      if (adaptive) {  // worst contraction per V-cycle of the items that took this step
        double worst = 0.0;
        for (int b = 0; b < B; ++b)
          if (hcyc[b] > prev[b] && lastp[b] > 0 && lastv[b] <= 1e300)
            worst = std::max(worst, std::pow(lastv[b] / lastp[b], 1.0 / nin));
        if (worst > 0) rho = std::min(0.7, std::max(0.02, worst));
      }
      prev = hcyc;
      // work of this replay: item-cycles done out of chunk * B launched
      c->work_scale = (double)done / ((double)chunk * B);
      c->bytes += gph->bytes * c->work_scale;
      if (!gph->ev.empty()) graph_harvest(c, gph);
      c->work_scale = 1.0;
      bool any = false;
      for (int b = 0; b < B; ++b) any = any || hact[b];
      if (!any || launched >= max_cycles) break;
    }
    std::vector<double> last(B);
    int hflag[2];
    CK(cudaMemcpyAsync(last.data(), L.mg_last + b0, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hflag, L.mg_flag, sizeof(hflag), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return solve_outcome(c, lev, B, inner, fixed, tol, max_cycles, tl, hcyc, last, hflag[0], s, vdone);
  }
  RET(residual());
  int cycles = 0, live = B;
  if (!fixed) {
    RET(read_norms(c, L, b0, B, nrm));
    for (int b = 0; b < B; ++b) {
      if (!(nrm[b] <= 1e300)) return h3d_fail(c, HEAT3D_ENAN, "NaN/Inf residual in a multigrid solve");
      if (nrm[b] <= (tolv ? tolv[b] : tol)) { ha[b] = 0; --live; }
    }
    if (live < B) CK(cudaMemcpyAsync(act, ha.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
  }
  while (cycles < max_cycles && live > 0) {
    c->work_scale = (double)live / B;  // converged items skip their blocks
    int rc = one_cycle();
    c->work_scale = 1.0;
    RET(rc);
    ++cycles;
    if (s) {
      s->vcycles += (long long)live * inner;
      s->vcycles_level[lev] += (long long)live * inner;
    }
    if (!fixed) {
      RET(read_norms(c, L, b0, B, nrm));
      bool changed = false;
      for (int b = 0; b < B; ++b) {
        if (!ha[b]) continue;
        if (!(nrm[b] <= 1e300)) return h3d_fail(c, HEAT3D_ENAN, "NaN/Inf residual in a multigrid solve");
        if (nrm[b] <= (tolv ? tolv[b] : tol)) { ha[b] = 0; --live; changed = true; }
      }
      if (changed && live > 0)
        CK(cudaMemcpyAsync(act, ha.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st));
    }
  }
  if (s) s->solves += B;
  if (fixed) {
    if (s) {
      RET(read_norms(c, L, b0, B, nrm));
      double mx = 0;
      for (double v : nrm) mx = std::max(mx, v);
      s->mg_residual = mx;
    }
    return HEAT3D_OK;
  }
  double mx = 0;
  for (int b = 0; b < B; ++b) mx = std::max(mx, nrm[b]);
  if (s) s->mg_residual = mx;
  if (live > 0) {
    if (s) s->notconv += live;
    return h3d_fail(c, HEAT3D_ENOTCONV, "multigrid: %d item(s) above tol %.3g after %d cycles", live,
                    tol, max_cycles);
  }
  return HEAT3D_OK;
}

int h3d_mg_solve(heat3d_ctx* c, int lev, int slot, int b0, int B, double* u, long long us,
                 const double* rhs, long long bs, int max_cycles, double tol, heat3d_stats* s,
                 const double* tolv) {
  if (h3d_tsize(c) == 4)
    return mg_solve_T<float>(c, lev, slot, b0, B, u, us, rhs, bs, max_cycles, tol, tolv, s);
  return mg_solve_T<double>(c, lev, slot, b0, B, u, us, rhs, bs, max_cycles, tol, tolv, s);
}

// ---------------------------------------------------------------------------
// SDC (Sec. 1.1)
// ---------------------------------------------------------------------------

// W U at the node fields of U (compact stencil only, else nullptr): WU has
// the layout of U.
static double* wu_of(SdcLevel& L, const double* u) {
  return L.WU ? L.WU + (u - L.U) : nullptr;
}

// The fields the quadrature kernel takes as "U": W U for the compact stencil
// (weighted collocation form), else U.
static double* ubase_of(SdcLevel& L, double* u) { return L.WU ? L.WU + (u - L.U) : u; }

// F at every node of items [b0, b0+B) from U.
int h3d_eval_F(heat3d_ctx* c, int lev, int b0, int B) {
  SdcLevel& L = c->lv[lev];
  const int M = L.L.M;
  const long long fs = L.g.fs;
  CK(launch_lap(L.L.order, L.g, B * M, L.U + (size_t)b0 * M * fs, fs, L.F + (size_t)b0 * M * fs, fs,
                L.alpha_nodes + (size_t)b0 * M, nullptr, nullptr, 0, nullptr, c->lv[lev].shape64, c->st,
                wu_of(L, L.U + (size_t)b0 * M * fs)));
  c->bytes += 16.0 * L.L.N * L.L.N * (double)L.L.N * B * M;
  return HEAT3D_OK;
}

// Collocation residual of items [b0, b0+B): max over items into *res (and per
// item into per_item when given).  Synchronises.
int h3d_residual(heat3d_ctx* c, int lev, int b0, int B, double* res, std::vector<double>* per_item) {
  SdcLevel& L = c->lv[lev];
  const int M = L.L.M;
  const long long fs = L.g.fs;
  CK(cudaMemsetAsync(L.norms + b0, 0, sizeof(unsigned long long) * B, c->st));
  CK(launch_integrals(M, L.g, B, ubase_of(L, L.U + (size_t)b0 * M * fs), L.F + (size_t)b0 * M * fs,
                      (lev == 1 && L.has_tau) ? L.tauS + (size_t)b0 * (M - 1) * fs : nullptr,
                      nullptr, L.items_d + b0, L.phi, L.norms + b0, nullptr, c->st));
  std::vector<double> n;
  RET(read_norms(c, L, b0, B, n));
  double mx = 0;
  for (double v : n) {
    if (!(v <= 1e300)) return h3d_fail(c, HEAT3D_ENAN, "NaN/Inf in the collocation residual");
    mx = std::max(mx, v);
  }
  if (res) *res = mx;
  if (per_item) *per_item = n;
  return HEAT3D_OK;
}

// One sweep over items [b0, b0+B).  When check_tol >= 0 the residual of the
// incoming iterate is computed by the quadrature kernel first; if it is
// <= check_tol for every item the sweep is skipped and 1 is returned.  With
// mg.rel > 0 (and mg.tol >= 0) the same residual r_b sets item b's solver
// tolerance for this sweep to max(mg.tol, mg.rel * r_b).
int h3d_sweep(heat3d_ctx* c, int lev, int b0, int B, double check_tol, heat3d_stats* s) {
  SdcLevel& L = c->lv[lev];
  const int M = L.L.M;
  const long long fs = L.g.fs;
  const double pts = (double)L.L.N * L.L.N * L.L.N * B;
  cudaStream_t st = c->st;
  double* U = L.U + (size_t)b0 * M * fs;
  double* F = L.F + (size_t)b0 * M * fs;
  double* I = L.I + (size_t)b0 * (M - 1) * fs;
  const heat3d_mg& mg = c->cfg.mg;
  const bool adapt = mg.rel > 0 && mg.tol >= 0;
  const bool want = check_tol >= 0 || adapt;
  if (want) CK(cudaMemsetAsync(L.norms + b0, 0, sizeof(unsigned long long) * B, st));
  CK(launch_integrals(M, L.g, B, ubase_of(L, U), F,
                      (lev == 1 && L.has_tau) ? L.tauS + (size_t)b0 * (M - 1) * fs : nullptr,
                      I, L.items_d + b0, L.phi, want ? L.norms + b0 : nullptr, nullptr, st));
  c->bytes += 8.0 * pts * (2 * M + (M - 1) + ((lev == 1 && L.has_tau) ? (M - 1) : 0));
  std::vector<double> tolv;
  if (want) {
    std::vector<double> n;
    RET(read_norms(c, L, b0, B, n));
    double mx = 0;
    for (double v : n) {
      if (!(v <= 1e300)) return h3d_fail(c, HEAT3D_ENAN, "NaN/Inf in the collocation residual");
      mx = std::max(mx, v);
    }
    if (s) s->residual = mx;
    if (check_tol >= 0 && mx <= check_tol) return 1;
    if (adapt) {
      tolv.resize(B);
      for (int b = 0; b < B; ++b) tolv[b] = std::max(mg.tol, mg.rel * n[b]);
    }
  }
  int status = HEAT3D_OK;
  for (int m = 0; m + 1 < M; ++m) {
    int rc = h3d_mg_solve(c, lev, m, b0, B, U + (size_t)(m + 1) * fs, (long long)M * fs,
                          I + (size_t)m * fs, (long long)(M - 1) * fs, mg.max_cycles, mg.tol, s,
                          adapt ? tolv.data() : nullptr);
    if (rc == HEAT3D_ENOTCONV) status = rc;
    else if (rc < 0) return rc;
    const bool add = m + 1 <= M - 2;
    CK(launch_lap(L.L.order, L.g, B, U + (size_t)(m + 1) * fs, (long long)M * fs,
                  F + (size_t)(m + 1) * fs, (long long)M * fs, L.alpha_items + b0,
                  add ? I + (size_t)(m + 1) * fs : nullptr, add ? I + (size_t)(m + 1) * fs : nullptr,
                  (long long)(M - 1) * fs, nullptr, L.shape64, st, wu_of(L, U + (size_t)(m + 1) * fs)));
    c->bytes += pts * (16.0 + (add ? 16.0 : 0.0));
  }
  if (s) s->sweeps += 1;
  return status;
}

// ---------------------------------------------------------------------------
// FAS between level 0 (fine) and level 1 (coarse)
// ---------------------------------------------------------------------------

// Compact fine level: the fine integrals of the weighted system are mapped
// back by W^{-1} (Sec. 1.2) in the form U_jm - U_0 + W^{-1} r, r the weighted
// residual at node jm; the W-solve (multigrid slot M, c = 0) writes its
// result into the fine integral fields I (free between sweeps) and stops at
// max(mg.tol, 0.01 max|r_b|) per item.
static int compact_wsolves(heat3d_ctx* c, int b0, int B, heat3d_stats* s) {
  SdcLevel& F = c->lv[0];
  const int MF = F.L.M, MG = c->lv[1].L.M;
  const long long ff = F.g.fs;
  const long long xs = (long long)(MF - 1) * ff;
  const heat3d_mg& mg = c->cfg.mg;
  int status = HEAT3D_OK;
  std::vector<double> n, tolv(B);
  for (int m = 1; m < MG; ++m) {
    const int jm = c->map.jm[m];
    double* X = F.I + (size_t)b0 * (MF - 1) * ff + (size_t)(m - 1) * ff;
    double* R = F.Wr + (size_t)b0 * ff;
    CK(cudaMemsetAsync(F.norms + b0, 0, sizeof(unsigned long long) * B, c->st));
    CK(launch_fas_wresid(MF, F.g, B, jm, F.WU + (size_t)b0 * MF * ff, F.F + (size_t)b0 * MF * ff,
                         F.items_d + b0, F.phi, R, X, xs, F.norms + b0, c->st));
    c->bytes += 8.0 * F.L.N * F.L.N * (double)F.L.N * B * (MF + 4);
    RET(read_norms(c, F, b0, B, n));
    for (int b = 0; b < B; ++b) tolv[b] = std::max(mg.tol, 0.01 * n[b]);
    int rc = h3d_mg_solve(c, 0, MF, b0, B, X, xs, R, ff, mg.max_cycles, mg.tol, s,
                          mg.tol >= 0 ? tolv.data() : nullptr);
    if (rc == HEAT3D_ENOTCONV) status = rc;
    else if (rc < 0) return rc;
  }
  return status;
}

int h3d_fas_restrict(heat3d_ctx* c, int b0, int B, heat3d_stats* s) {
  SdcLevel &F = c->lv[0], &G = c->lv[1];
  const int MF = F.L.M, MG = G.L.M;
  const long long ff = F.g.fs, gf = G.g.fs;
  cudaStream_t st = c->st;
  int status = HEAT3D_OK;
  const double* X = nullptr;
  if (F.L.order == kCompact) {
    status = compact_wsolves(c, b0, B, s);
    if (status < 0 && status != HEAT3D_ENOTCONV) return status;
    X = F.I + (size_t)b0 * (MF - 1) * ff;
  }
  CK(launch_fas_inject(MF, MG, F.g, G.g, B, F.U + (size_t)b0 * MF * ff, F.F + (size_t)b0 * MF * ff,
                       G.U + (size_t)b0 * MG * gf, G.UGr + (size_t)b0 * MG * gf,
                       G.qF + (size_t)b0 * MG * gf, F.items_d + b0, c->map_d, F.phi, st, X,
                       (long long)(MF - 1) * ff));
  CK(launch_lap(G.L.order, G.g, B * MG, G.U + (size_t)b0 * MG * gf, gf, G.F + (size_t)b0 * MG * gf, gf,
                G.alpha_nodes + (size_t)b0 * MG, nullptr, nullptr, 0, nullptr, G.shape64, st));
  CK(launch_fas_tau(MG, G.g, B, G.qF + (size_t)b0 * MG * gf, G.F + (size_t)b0 * MG * gf,
                    G.tauS + (size_t)b0 * (MG - 1) * gf, G.items_d + b0, G.phi, st));
  G.has_tau = true;
  const double pg = (double)G.L.N * G.L.N * G.L.N * B;
  c->bytes += pg * 8.0 * (2 * MF + 3 * MG) + pg * 16.0 * MG + pg * 8.0 * (2 * MG + MG - 1);
  return status;
}

int h3d_fas_interpolate(heat3d_ctx* c, int b0, int B) {
  SdcLevel &F = c->lv[0], &G = c->lv[1];
  const int MF = F.L.M, MG = G.L.M;
  const long long ff = F.g.fs, gf = G.g.fs;
  cudaStream_t st = c->st;
  double* D = G.D + (size_t)b0 * MF * gf;
  CK(launch_fas_delta(MF, MG, G.g, B, G.U + (size_t)b0 * MG * gf, G.UGr + (size_t)b0 * MG * gf, D,
                      c->map_d, st));
  if (F.L.N == G.L.N) {
    CK(launch_update<double>(F.g, B * MF, D, F.U + (size_t)b0 * MF * ff, ff, nullptr, st));
  } else if (c->cfg.interp >= 4) {
    const int npts = c->cfg.interp;
    if (MF >= 3) {
      // separable passes node by node, temporaries in the fine integral
      // fields I (free between sweeps): fields 0 and 1 of each item
      const long long is = (long long)(MF - 1) * ff;
      double* I0 = F.I + (size_t)b0 * (MF - 1) * ff;
      for (int j = 0; j < MF; ++j)
        CK(launch_prolong_add_mid(npts, G.g, F.g, B, D + (size_t)j * gf, (long long)MF * gf,
                                  F.U + (size_t)b0 * MF * ff + (size_t)j * ff, (long long)MF * ff,
                                  st, I0, I0 + ff, is));
    } else {
      CK(launch_prolong_add_mid(npts, G.g, F.g, B * MF, D, gf, F.U + (size_t)b0 * MF * ff, ff, st));
    }
  } else {
    CK(launch_prolong_add<double>(G.g, F.g, B * MF, D, gf, F.U + (size_t)b0 * MF * ff,
                                  F.U + (size_t)b0 * MF * ff, ff, nullptr, st));
  }
  RET(h3d_eval_F(c, 0, b0, B));
  const double pf = (double)F.L.N * F.L.N * F.L.N * B;
  c->bytes += pf * MF * 16.0 + pf / 8.0 * 8.0 * (2 * MG + MF);
  return HEAT3D_OK;
}

// ---------------------------------------------------------------------------
// drivers over [0, T]
// ---------------------------------------------------------------------------

// Spread the pitched field u (one item) to every node of items [b0, b0+B).
int h3d_spread(heat3d_ctx* c, int lev, int b0, int B, const double* u) {
  SdcLevel& L = c->lv[lev];
  const int M = L.L.M;
  const long long fs = L.g.fs;
  CK(launch_copy(L.g, B * M, u, 0, L.U + (size_t)b0 * M * fs, fs, c->st));
  RET(h3d_eval_F(c, lev, b0, B));
  c->bytes += 8.0 * L.L.N * L.L.N * (double)L.L.N * B * M;
  return HEAT3D_OK;
}

// Serial coarse pass over slices 0..P-1: slice p > 0 starts from the coarse
// end value of slice p-1.
static int coarse_pass(heat3d_ctx* c, int P, heat3d_stats* s) {
  SdcLevel& G = c->lv[1];
  const int MG = G.L.M;
  const long long gf = G.g.fs;
  int status = HEAT3D_OK;
  for (int p = 0; p < P; ++p) {
    if (p > 0) {
      CK(launch_copy(G.g, 1, G.U + ((size_t)(p - 1) * MG + MG - 1) * gf, 0, G.U + (size_t)p * MG * gf, 0, c->st));
      CK(launch_lap(G.L.order, G.g, 1, G.U + (size_t)p * MG * gf, 0, G.F + (size_t)p * MG * gf, 0,
                    G.alpha_items + p, nullptr, nullptr, 0, nullptr, G.shape64, c->st));
    }
    for (int k = 0; k < c->cfg.sweeps_coarse; ++k) {
      int rc = h3d_sweep(c, 1, p, 1, -1.0, s);
      if (rc == HEAT3D_ENOTCONV) status = rc;
      else if (rc < 0) return rc;
    }
  }
  return status;
}

// Fine end value of slice p-1 becomes node 0 of slice p (p = 1..P-1).
static int forward_fine(heat3d_ctx* c, int P) {
  if (P < 2) return HEAT3D_OK;
  SdcLevel& F = c->lv[0];
  const int MF = F.L.M;
  const long long ff = F.g.fs;
  CK(launch_copy(F.g, P - 1, F.U + (size_t)(MF - 1) * ff, (long long)MF * ff, F.U + (size_t)MF * ff,
                 (long long)MF * ff, c->st));
  CK(launch_lap(F.L.order, F.g, P - 1, F.U + (size_t)MF * ff, (long long)MF * ff, F.F + (size_t)MF * ff,
                (long long)MF * ff, F.alpha_items + 1, nullptr, nullptr, 0, nullptr, F.shape64, c->st,
                wu_of(F, F.U + (size_t)MF * ff)));
  return HEAT3D_OK;
}

int h3d_run(heat3d_ctx* c, double* ucur, heat3d_stats* s) {
  const heat3d_config& cfg = c->cfg;
  SdcLevel& F = c->lv[0];
  const int P = cfg.nlevels == 2 ? cfg.slices : 1;
  const int nsteps = (int)llround(c->T_run / cfg.dt);
  if (nsteps < 1 || fabs(nsteps * cfg.dt - c->T_run) > 1e-9 * std::max(1.0, c->T_run))
    return h3d_fail(c, HEAT3D_EINVAL, "T must be a multiple of dt");
  if (nsteps % P != 0) return h3d_fail(c, HEAT3D_EINVAL, "number of steps must be a multiple of slices");
  if (P > F.B) return h3d_fail(c, HEAT3D_EINVAL, "slices exceed the batch capacity");
  const int MF = F.L.M;
  const long long ff = F.g.fs;
  int status = HEAT3D_OK;
  for (int l = 0; l < cfg.nlevels; ++l) {
    for (int p = 0; p < P; ++p) {
      c->lv[l].nu[p] = cfg.nu;
      c->lv[l].dt[p] = cfg.dt;
    }
    RET(h3d_set_item_operators(c, l, 0, P));
  }
  for (int blk = 0; blk < nsteps / P; ++blk) {
    const double tb = c->t_start + (double)blk * P * cfg.dt;
    for (int l = 0; l < cfg.nlevels; ++l) {
      for (int p = 0; p < P; ++p) h3d_fill_item(c, l, p, tb + p * cfg.dt);
      RET(h3d_upload_items(c, l, 0, P));
    }
    RET(h3d_spread(c, 0, 0, P, ucur));
    if (cfg.nlevels == 1) {
      for (int k = 0; k < cfg.sweeps_fine; ++k) {
        int rc = h3d_sweep(c, 0, 0, 1, cfg.tol_sdc >= 0 ? cfg.tol_sdc : -1.0, s);
        if (rc == 1) break;
        if (rc == HEAT3D_ENOTCONV) status = rc;
        else if (rc < 0) return rc;
      }
    } else {
      c->lv[1].has_tau = false;
      if (cfg.predictor) {
        int rr = h3d_fas_restrict(c, 0, P, s);
        if (rr == HEAT3D_ENOTCONV) status = rr;
        else if (rr < 0) return rr;
        int rc = coarse_pass(c, P, s);
        if (rc == HEAT3D_ENOTCONV) status = rc;
        else if (rc < 0) return rc;
        RET(h3d_fas_interpolate(c, 0, P));
        RET(forward_fine(c, P));
      }
      for (int it = 0; it < cfg.iters; ++it) {
        bool done = false;
        for (int k = 0; k < cfg.sweeps_fine; ++k) {
          double chk = (k == 0 && it > 0 && cfg.tol_sdc >= 0) ? cfg.tol_sdc : -1.0;
          int rc = h3d_sweep(c, 0, 0, P, chk, s);
          if (rc == 1) { done = true; break; }
          if (rc == HEAT3D_ENOTCONV) status = rc;
          else if (rc < 0) return rc;
        }
        if (done) break;
        int rr = h3d_fas_restrict(c, 0, P, s);
        if (rr == HEAT3D_ENOTCONV) status = rr;
        else if (rr < 0) return rr;
        int rc = coarse_pass(c, P, s);
        if (rc == HEAT3D_ENOTCONV) status = rc;
        else if (rc < 0) return rc;
        RET(h3d_fas_interpolate(c, 0, P));
        RET(forward_fine(c, P));
        if (s) s->iters += 1;
      }
    }
    if (s) {
      double r = 0;
      RET(h3d_residual(c, 0, 0, P, &r, nullptr));
      s->residual = r;
      s->steps += P;
    }
    CK(launch_copy(F.g, 1, F.U + ((size_t)(P - 1) * MF + MF - 1) * ff, 0, ucur, 0, c->st));
  }
  return status;
}

// ---------------------------------------------------------------------------
// autotuner: launch shape per multigrid level (all shapes give identical results)
// ---------------------------------------------------------------------------

template <typename Launch>
static float time_shape(heat3d_ctx* c, cudaEvent_t e0, cudaEvent_t e1, Launch&& launch) {
  if (launch() != cudaSuccess) return 1e30f;  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, c->st);
    cudaError_t e = launch();
    cudaEventRecord(e1, c->st);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  return best;
}

static bool tune_log() {
  const char* v = getenv("HEAT3D_TUNE_LOG");
  return v && v[0] == '1';
}

// vec4: the operator has the four-points-per-thread FP32 tiles (kinds 7-14,
// and 15-26 with the z neighbours in registers, 19-26 loading planes by
// TMA, 23-26 with a producer warp and no block barriers); the latter also
// try a chunk of 12 planes and the chunks that fill one or two whole waves
// of the GPU.
static std::vector<Shape> shape_candidates(int N, bool vec4) {
  std::vector<Shape> v;
  for (int zc : {1, 2, 4, 8, 16, 32, 64})
    if (zc <= N) v.push_back(Shape{1, zc});
  if (N >= 16) {
    for (int kind = 2; kind <= (vec4 ? 14 : 6); ++kind)
      for (int zc : {2, 4, 8, 16, 32, 64})
        if (zc <= N) v.push_back(Shape{kind, zc});
    if (vec4)  // zc -1, -2: the chunk length that fills one or two whole waves
      for (int kind = 15; kind <= 26; ++kind)
        for (int zc : {8, 12, 16, 32, -1, -2})
          if (zc <= N) v.push_back(Shape{kind, zc});
  }
  return v;
}

template <typename T>
static int autotune_T(heat3d_ctx* c, cudaEvent_t e0, cudaEvent_t e1) {
  for (int lev = 0; lev < c->cfg.nlevels; ++lev) {
    SdcLevel& L = c->lv[lev];
    for (int k = 0; k < L.nmg; ++k) {
      const Grid& g = L.mg[k];
      const Coef<T>* cf = coefT<T>(L, 0, k, 0);
      T* b = mgbuf<T>(L, k, 0, 0);
      T* e = mgbuf<T>(L, k, 1, 0);
      T* t = mgbuf<T>(L, k, 2, 0);
      float best = 1e30f;
      Shape pick{1, std::min(16, g.N)};
      for (Shape sh : shape_candidates(g.N, sizeof(T) == 4)) {
        float ms = time_shape(c, e0, e1, [&] {
          return launch_jacobi<T>(L.L.order, g, L.B, e, b, t, nullptr, 0, cf, nullptr, sh, c->st);
        });
        if (tune_log())
          fprintf(stderr, "tune jacobi T%zu order %d N %d B %d kind %d zc %d: %.4f ms\n", sizeof(T),
                  L.L.order, g.N, L.B, sh.kind, sh.zc, ms);
        if (ms < best) { best = ms; pick = sh; }
      }
      L.shapeT[k] = pick;
    }
    float best = 1e30f;
    Shape pick{1, std::min(16, L.g.N)};
    const long long fs = L.g.fs;
    for (Shape sh : shape_candidates(L.g.N, false)) {
      float ms = time_shape(c, e0, e1, [&] {
        return launch_lap(L.L.order, L.g, L.B, L.U, (long long)L.L.M * fs, L.F, (long long)L.L.M * fs,
                          L.alpha_items, nullptr, nullptr, 0, nullptr, sh, c->st);
      });
      if (ms < best) { best = ms; pick = sh; }
    }
    L.shape64 = pick;
    // How far down to fuse the coarse levels: the fused kernel runs on one SM
    // per item, so deep fusion saves launches but can cost FP64 throughput.
    // Time the V-cycle below the first level with N <= 15 for each choice.
    int k15 = -1;
    for (int k = 1; k < L.nmg; ++k)
      if (L.mg[k].N <= kFusedMaxN) { k15 = k; break; }
    if (c->cfg.fuse_coarse && L.L.order != kCompact && k15 > 0) {
      float bestf = 1e30f;
      int pickf = kFusedMaxN;
      for (int fm : {15, 7, 3, 0}) {
        L.fuse_max = fm;
        float ms = time_shape(c, e0, e1, [&] {
          T* cur = nullptr;
          return vcycle_level<T>(c, L, 0, k15, 0, L.B, nullptr, nullptr, 0, &cur) == HEAT3D_OK
                     ? cudaSuccess
                     : cudaErrorUnknown;
        });
        if (tune_log())
          fprintf(stderr, "tune fuse T%zu order %d below N %d: fuse_max %d: %.4f ms\n", sizeof(T),
                  L.L.order, L.mg[k15].N, fm, ms);
        if (ms < bestf) { bestf = ms; pickf = fm; }
      }
      L.fuse_max = pickf;
    }
  }
  return HEAT3D_OK;
}

// Tuning file (environment variable HEAT3D_TUNE_FILE): one line per SDC level,
// "tsize order N B fuse_max kind64 zc64 n kind_0 zc_0 ... kind_{n-1} zc_{n-1}".
// A context whose level is listed takes those shapes instead of timing them
// (so that a profiler's run uses the shapes of the measured run); levels that
// are not listed are timed and appended.
static bool tune_file_lookup(heat3d_ctx* c, SdcLevel& L, const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  bool found = false;
  int ts, order, N, B, fm, k64, z64, n;
  while (!found && fscanf(f, "%d %d %d %d %d %d %d %d", &ts, &order, &N, &B, &fm, &k64, &z64, &n) == 8) {
    std::vector<Shape> sh(n > 0 && n <= kMaxLevels ? n : 0);
    bool ok = n > 0 && n <= kMaxLevels;
    for (int k = 0; k < n; ++k) {
      int kd = 0, zc = 0;
      if (fscanf(f, "%d %d", &kd, &zc) != 2) { ok = false; break; }
      if (ok) sh[k] = Shape{kd, zc};
    }
    if (ok && ts == (int)h3d_tsize(c) && order == L.L.order && N == L.L.N && B == L.B && n == L.nmg) {
      for (int k = 0; k < n; ++k) L.shapeT[k] = sh[k];
      L.shape64 = Shape{k64, z64};
      L.fuse_max = fm;
      found = true;
    }
  }
  fclose(f);
  return found;
}

static void tune_file_append(heat3d_ctx* c, const SdcLevel& L, const char* path) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%d %d %d %d %d %d %d %d", (int)h3d_tsize(c), L.L.order, L.L.N, L.B, L.fuse_max,
          L.shape64.kind, L.shape64.zc, L.nmg);
  for (int k = 0; k < L.nmg; ++k) fprintf(f, " %d %d", L.shapeT[k].kind, L.shapeT[k].zc);
  fprintf(f, "\n");
  fclose(f);
}

int h3d_autotune(heat3d_ctx* c) {
  const char* tf = getenv("HEAT3D_TUNE_FILE");
  bool all_listed = tf && tf[0];
  if (all_listed)
    for (int l = 0; l < c->cfg.nlevels; ++l) all_listed = tune_file_lookup(c, c->lv[l], tf) && all_listed;
  if (all_listed) return HEAT3D_OK;
  EventPair ev;
  CK(cudaEventCreate(&ev.e0));
  CK(cudaEventCreate(&ev.e1));
  const long long l0 = h3d::launches_total();
  int rc = h3d_tsize(c) == 4 ? autotune_T<float>(c, ev.e0, ev.e1)
                             : autotune_T<double>(c, ev.e0, ev.e1);
  h3d::launches_adjust(-(h3d::launches_total() - l0));  // tuning launches are not work
  CK(cudaStreamSynchronize(c->st));
  if (rc == HEAT3D_OK && tf && tf[0])
    for (int l = 0; l < c->cfg.nlevels; ++l) tune_file_append(c, c->lv[l], tf);
  return rc;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// dense host-or-device N^3 array -> pitched field (one item) via abi_b staging.
int h3d_load_dense(heat3d_ctx* c, int lev, const double* src, double* dst_pitched) {
  SdcLevel& L = c->lv[lev];
  const size_t n = (size_t)L.L.N * L.L.N * L.L.N;
  const double* dsrc = src;
  if (!is_device_ptr(src)) {
    CK(cudaMemcpyAsync(L.abi_b, src, n * 8, cudaMemcpyHostToDevice, c->st));
    dsrc = L.abi_b;
  }
  CK(launch_dense_to_pitched(L.g, 1, dsrc, dst_pitched, 0, c->st));
  return HEAT3D_OK;
}

int h3d_store_dense(heat3d_ctx* c, int lev, const double* src_pitched, double* dst) {
  SdcLevel& L = c->lv[lev];
  const size_t n = (size_t)L.L.N * L.L.N * L.L.N;
  if (is_device_ptr(dst)) {
    CK(launch_pitched_to_dense(L.g, 1, src_pitched, 0, dst, c->st));
    return HEAT3D_OK;
  }
  CK(launch_pitched_to_dense(L.g, 1, src_pitched, 0, L.abi_b, c->st));
  CK(cudaMemcpyAsync(dst, L.abi_b, n * 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return HEAT3D_OK;
}

// A lost TMA plane copy in an FP32 stencil (bounded wait gave up): the
// affected tile was not computed, so the call fails with HEAT3D_ETIMEOUT.
static int check_loader(heat3d_ctx* c) {
  if (h3d_tsize(c) != 4) return HEAT3D_OK;
  int flag = 0;
  CK(loader_timeouts_take(c->st, &flag));
  if (flag) return h3d_fail(c, HEAT3D_ETIMEOUT, "an FP32 stencil's TMA plane copy did not complete");
  return HEAT3D_OK;
}

#define NEED_BOUND(c)                                                                  \
  do {                                                                                 \
    if (!(c)) return HEAT3D_EINVAL;                                                    \
    if (!(c)->bound) return h3d_fail((c), HEAT3D_ESTATE, "no workspace bound");        \
  } while (0)

int h3d_workspace_size_msg(const heat3d_config* cfg, size_t* bytes, char* msg, size_t msg_len) {
  if (!cfg || !bytes) return HEAT3D_EINVAL;
  heat3d_ctx tmp;
  int rc = validate(&tmp, cfg);
  if (rc >= 0) {
    tmp.cfg = *cfg;
    rc = setup_levels(&tmp);
  }
  if (rc < 0) {
    if (msg && msg_len) snprintf(msg, msg_len, "%s", tmp.err);
    return rc;
  }
  *bytes = plan(&tmp, nullptr);
  return HEAT3D_OK;
}

extern "C" {

void heat3d_config_default(heat3d_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->nu = 0.1;
  cfg->T = 1.0;
  cfg->dt = 1.0 / 64;
  cfg->nlevels = 2;
  cfg->levels[0] = heat3d_level{31, 4, 5};
  cfg->levels[1] = heat3d_level{15, 2, 3};
  cfg->sweeps_fine = 2;
  cfg->sweeps_coarse = 1;
  cfg->slices = 1;
  cfg->iters = 20;
  cfg->tol_sdc = 1e-10;
  cfg->predictor = 1;
  cfg->mg = heat3d_mg{2, 1, 50, 1e-10, 1, 0.0};
  cfg->precision = HEAT3D_FP64;
  cfg->forcing = HEAT3D_FORCING_PAPER_LITERAL;
  cfg->batch = 1;
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->use_graphs = 0;
  cfg->autotune = 1;
  cfg->fuse_coarse = 1;
  cfg->interp = 2;
  cfg->persistent = -1;
}

int heat3d_workspace_size(const heat3d_config* cfg, size_t* bytes) {
  if (!cfg || !bytes) return HEAT3D_EINVAL;
  heat3d_ctx tmp;
  int rc = validate(&tmp, cfg);
  if (rc < 0) return rc;
  tmp.cfg = *cfg;
  rc = setup_levels(&tmp);
  if (rc < 0) return rc;
  *bytes = plan(&tmp, nullptr);
  return HEAT3D_OK;
}

int heat3d_init(const heat3d_config* cfg, heat3d_ctx** out) {
  if (!out) return HEAT3D_EINVAL;
  *out = nullptr;
  heat3d_ctx* c = new heat3d_ctx();
  int rc = validate(c, cfg);
  if (rc < 0) { delete c; return rc; }
  c->cfg = *cfg;
  c->st = (cudaStream_t)cfg->stream;
  rc = setup_levels(c);
  if (rc < 0) { delete c; return rc; }
  c->ws_need = plan(c, nullptr);
  c->t_start = 0.0;
  c->T_run = cfg->T;
  *out = c;
  return HEAT3D_OK;
}

int heat3d_bind_workspace(heat3d_ctx* c, void* dptr, size_t bytes) {
  if (!c || !dptr) return HEAT3D_EINVAL;
  if (bytes < c->ws_need) return h3d_fail(c, HEAT3D_ENOMEM, "workspace %zu < %zu bytes", bytes, c->ws_need);
  if (((uintptr_t)dptr) % 256) return h3d_fail(c, HEAT3D_EINVAL, "workspace must be 256-byte aligned");
  CK(cudaSetDevice(c->cfg.device));
  plan(c, (char*)dptr);
  c->ws = dptr;
  c->ws_bytes = bytes;
  CK(cudaMemsetAsync(dptr, 0, c->ws_need, c->st));
  CK(cudaMemcpyAsync(c->map_d, &c->map, sizeof(FasMap), cudaMemcpyHostToDevice, c->st));
  for (int l = 0; l < c->cfg.nlevels; ++l) {
    SdcLevel& L = c->lv[l];
    std::vector<double> phi(L.L.N);
    for (int i = 0; i < L.L.N; ++i) phi[i] = sin(M_PI * (i + 1) * L.h[0]);
    CK(cudaMemcpyAsync(L.phi, phi.data(), sizeof(double) * L.L.N, cudaMemcpyHostToDevice, c->st));
    RET(h3d_set_item_operators(c, l, 0, L.B));
    for (int b = 0; b < L.B; ++b) h3d_fill_item(c, l, b, 0.0);
    RET(h3d_upload_items(c, l, 0, L.B));
  }
  CK(cudaStreamSynchronize(c->st));
  c->bound = true;
  // persistent solve kernel: grids with N <= 31 by default, up to
  // kPersistMaxN when forced (orders 2 and 4, cooperative launch needed)
  int coop = 0;
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->cfg.device));
  for (int l = 0; l < c->cfg.nlevels; ++l) {
    SdcLevel& L = c->lv[l];
    const int lim = c->cfg.persistent > 0 ? kPersistMaxN : 31;
    L.persist = c->cfg.persistent != 0 && coop && mg_persist_supported(L.L.order, L.L.N) &&
                L.L.N <= lim;
  }
  if (c->cfg.autotune) RET(h3d_autotune(c));
  // HEAT3D_FUSE_MAX=n forces the coarse-level fusion depth (testing)
  if (const char* f = getenv("HEAT3D_FUSE_MAX")) {
    int fm = -1;
    if (sscanf(f, "%d", &fm) == 1 && fm >= 0)
      for (int l = 0; l < c->cfg.nlevels; ++l) c->lv[l].fuse_max = fm;
  }
  // HEAT3D_SHAPE=kind,zc forces one launch shape on every stencil (testing:
  // every shape must give bitwise the same results)
  if (const char* f = getenv("HEAT3D_SHAPE")) {
    int kind = 0, zc = 0;
    if (sscanf(f, "%d,%d", &kind, &zc) == 2 && kind >= 1 && kind <= 26 && zc >= -2 && zc != 0) {
      for (int l = 0; l < c->cfg.nlevels; ++l) {
        SdcLevel& L = c->lv[l];
        for (int k = 0; k < L.nmg; ++k)
          if (kind == 1 || L.mg[k].N >= 16) L.shapeT[k] = Shape{kind, zc};
        if (kind == 1 || L.g.N >= 16) L.shape64 = Shape{kind, zc};
      }
    }
  }
  return HEAT3D_OK;
}

int heat3d_set_interval(heat3d_ctx* c, double t0, double T) {
  if (!c || !(T > 0)) return HEAT3D_EINVAL;
  c->t_start = t0;
  c->T_run = T;
  return HEAT3D_OK;
}

long long heat3d_kernel_launches(void) { return h3d::g_launches.load(); }

int heat3d_profile(heat3d_ctx* c, int kernel_class) {
  if (!c || kernel_class < 0 || kernel_class > HEAT3D_PROF_JACOBI_FINE_STORE) return HEAT3D_EINVAL;
  cudaStreamSynchronize(c->st);
  c->prof_used = 0;
  c->prof_ms = c->prof_bytes = c->prof_dpops = c->prof_flops = 0.0;
  c->prof_launches = 0;
  c->prof_class = kernel_class;
  return HEAT3D_OK;
}

int heat3d_profile_read(heat3d_ctx* c, double* ms, long long* launches, double* bytes,
                        double* dp_ops, double* flops) {
  if (!c) return HEAT3D_EINVAL;
  prof_harvest(c);
  if (ms) *ms = c->prof_ms;
  if (launches) *launches = c->prof_launches;
  if (bytes) *bytes = c->prof_bytes;
  if (dp_ops) *dp_ops = c->prof_dpops;
  if (flops) *flops = c->prof_flops;
  return HEAT3D_OK;
}

int heat3d_destroy(heat3d_ctx* c) {
  if (!c) return HEAT3D_EINVAL;
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  for (CycleGraph* g : c->graphs) free_graph(g);
  c->graphs.clear();
  h3d_destroy_extras(c);
  delete c;
  return HEAT3D_OK;
}

const char* heat3d_last_error(const heat3d_ctx* c) { return c ? c->err : "null context"; }

int heat3d_set_stream(heat3d_ctx* c, void* stream) {
  if (!c) return HEAT3D_EINVAL;
  c->st = (cudaStream_t)stream;
  return HEAT3D_OK;
}

int heat3d_apply_laplacian(heat3d_ctx* c, int level, const double* u, double* out) {
  NEED_BOUND(c);
  if (level < 0 || level >= c->cfg.nlevels || !u || !out) return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  SdcLevel& L = c->lv[level];
  RET(h3d_load_dense(c, level, u, L.abi_u));
  CK(launch_lap(L.L.order, L.g, 1, L.abi_u, 0, L.abi_p0, 0, L.alpha_items, nullptr, nullptr, 0,
                nullptr, L.shape64, c->st));
  RET(h3d_store_dense(c, level, L.abi_p0, out));
  return HEAT3D_OK;
}

int mg_vcycle(heat3d_ctx* c, int level, double cc, const double* rhs, double* u, int max_cycles,
              double tol, heat3d_stats* stats) {
  NEED_BOUND(c);
  if (level < 0 || level >= c->cfg.nlevels || !rhs || !u || max_cycles < 0 || !(cc >= 0))
    return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  SdcLevel& L = c->lv[level];
  EventPair ev;
  CK(cudaEventCreate(&ev.e0));
  CK(cudaEventCreate(&ev.e1));
  CK(cudaEventRecord(ev.e0, c->st));
  double* ub = L.abi_p0;  // pitched solution
  double* bb = L.abi_p1;  // pitched right-hand side
  RET(h3d_load_dense(c, level, rhs, bb));
  RET(h3d_load_dense(c, level, u, ub));
  const int slot = L.nslots - 1;
  RET(h3d_set_coefs(c, level, slot, 0, 1, &cc));
  heat3d_stats loc{};
  c->bytes = 0;
  int rc = max_cycles > 0 ? h3d_mg_solve(c, level, slot, 0, 1, ub, 0, bb, 0, max_cycles, tol, &loc)
                          : HEAT3D_OK;
  if (rc < 0 && rc != HEAT3D_ENOTCONV) return rc;
  RET(check_loader(c));
  RET(h3d_store_dense(c, level, ub, u));
  CK(cudaEventRecord(ev.e1, c->st));
  CK(cudaEventSynchronize(ev.e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, ev.e0, ev.e1);
  loc.seconds = ms * 1e-3;
  loc.bytes = c->bytes;
  if (stats) *stats = loc;
  return rc;
}

int heat3d_set_state(heat3d_ctx* c, int level, int item, double t0, const double* u0) {
  NEED_BOUND(c);
  if (level < 0 || level >= c->cfg.nlevels || item < 0 || item >= c->lv[level].B || !u0)
    return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  SdcLevel& L = c->lv[level];
  RET(h3d_load_dense(c, level, u0, L.abi_u));
  RET(h3d_spread(c, level, item, 1, L.abi_u));
  h3d_fill_item(c, level, item, t0);
  RET(h3d_upload_items(c, level, item, 1));
  CK(cudaStreamSynchronize(c->st));
  return HEAT3D_OK;
}

int heat3d_get_node(heat3d_ctx* c, int level, int item, int node, double* out) {
  NEED_BOUND(c);
  if (level < 0 || level >= c->cfg.nlevels || item < 0 || item >= c->lv[level].B || node < 0 ||
      node >= c->lv[level].L.M || !out)
    return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  SdcLevel& L = c->lv[level];
  RET(h3d_store_dense(c, level, L.U + ((size_t)item * L.L.M + node) * L.g.fs, out));
  CK(cudaStreamSynchronize(c->st));
  return HEAT3D_OK;
}

int heat3d_set_node(heat3d_ctx* c, int level, int item, int node, const double* in) {
  NEED_BOUND(c);
  if (level < 0 || level >= c->cfg.nlevels || item < 0 || item >= c->lv[level].B || node < 0 ||
      node >= c->lv[level].L.M || !in)
    return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  SdcLevel& L = c->lv[level];
  double* dst = L.U + ((size_t)item * L.L.M + node) * L.g.fs;
  RET(h3d_load_dense(c, level, in, dst));
  CK(launch_lap(L.L.order, L.g, 1, dst, 0, L.F + ((size_t)item * L.L.M + node) * L.g.fs, 0,
                L.alpha_items + item, nullptr, nullptr, 0, nullptr, L.shape64, c->st, wu_of(L, dst)));
  CK(cudaStreamSynchronize(c->st));
  return HEAT3D_OK;
}

int sdc_sweep(heat3d_ctx* c, int level, int batch_begin, int batch_count, heat3d_stats* stats) {
  NEED_BOUND(c);
  if (level < 0 || level >= c->cfg.nlevels || batch_begin < 0 || batch_count < 1 ||
      batch_begin + batch_count > c->lv[level].B)
    return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  heat3d_stats loc{};
  c->bytes = 0;
  int rc = h3d_sweep(c, level, batch_begin, batch_count, -1.0, &loc);
  CK(cudaStreamSynchronize(c->st));
  RET(check_loader(c));
  loc.bytes = c->bytes;
  if (stats) *stats = loc;
  return rc;
}

int heat3d_sdc_residual(heat3d_ctx* c, int level, int item, double* residual) {
  NEED_BOUND(c);
  if (level < 0 || level >= c->cfg.nlevels || item < 0 || item >= c->lv[level].B || !residual)
    return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  return h3d_residual(c, level, item, 1, residual, nullptr);
}

int heat3d_fas_restrict(heat3d_ctx* c, int begin, int count) {
  NEED_BOUND(c);
  if (c->cfg.nlevels != 2 || begin < 0 || count < 1 || begin + count > c->lv[0].B)
    return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  int rc = h3d_fas_restrict(c, begin, count, nullptr);
  if (rc < 0 && rc != HEAT3D_ENOTCONV) return rc;
  CK(cudaStreamSynchronize(c->st));
  return rc;
}

int heat3d_fas_interpolate(heat3d_ctx* c, int begin, int count) {
  NEED_BOUND(c);
  if (c->cfg.nlevels != 2 || begin < 0 || count < 1 || begin + count > c->lv[0].B)
    return h3d_fail(c, HEAT3D_EINVAL, "bad arguments");
  RET(h3d_fas_interpolate(c, begin, count));
  CK(cudaStreamSynchronize(c->st));
  return HEAT3D_OK;
}

int pfasst_run(heat3d_ctx* c, const double* u0, double* uT, heat3d_stats* stats) {
  NEED_BOUND(c);
  if (!u0 || !uT) return h3d_fail(c, HEAT3D_EINVAL, "null u0/uT");
  SdcLevel& F = c->lv[0];
  EventPair ev;
  CK(cudaEventCreate(&ev.e0));
  CK(cudaEventCreate(&ev.e1));
  CK(cudaEventRecord(ev.e0, c->st));
  heat3d_stats loc{};
  c->bytes = 0;
  RET(h3d_load_dense(c, 0, u0, F.abi_u));
  int rc = h3d_run(c, F.abi_u, &loc);
  if (rc < 0 && rc != HEAT3D_ENOTCONV) return rc;
  RET(check_loader(c));
  RET(h3d_store_dense(c, 0, F.abi_u, uT));
  CK(cudaEventRecord(ev.e1, c->st));
  CK(cudaEventSynchronize(ev.e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, ev.e0, ev.e1);
  loc.seconds = ms * 1e-3;
  loc.bytes = c->bytes;
  if (stats) *stats = loc;
  return rc;
}

}  // extern "C"
