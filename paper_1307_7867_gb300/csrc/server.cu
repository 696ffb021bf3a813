// server.cu -- continuous-batching serving loop for independent heat-equation
// solves (zero forcing, 3-node SDC, 7-point Laplacian, fixed sweeps per step).
//
// Requests are grouped by grid size N.  A group owns one heat3d context whose
// item slots hold the requests resident on the device; its workspace, plus
// one pitched "current value" field per slot and the initial-value tables,
// come from the caller's device pool through a first-fit sub-allocator.  A
// request is admitted when its group has a free slot and (for a new group)
// the pool has room; otherwise it waits in arrival order.  One scheduler
// thread advances every group by one time step per round: the group's
// resident requests are packed into items 0..A-1, swept together (per-item
// nu, dt, forcing data, multigrid masks), and unpacked.  A request whose last
// step is done is copied to host memory, its slot freed at once, and new
// requests join the next round.  Each item's arithmetic depends only on its
// own data, so a result is the same alone or in any mix.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "runtime.cuh"

using namespace h3d;

namespace {

constexpr int kModes = 8;

// u(x) = sum_m amp_m sx_m[i] sy_m[j] sz_m[k], tables of sin(k pi x).
__global__ void k_modes_ic(Grid g, int nm, const double* __restrict__ tab,
                           const double* __restrict__ amp, double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.N || j >= g.N) return;
  const int N = g.N;
  double s = 0.0;
  for (int m = 0; m < nm; ++m) {
    const double* t = tab + (size_t)m * 3 * N;
    s = fma(amp[m] * t[i], t[N + j] * t[2 * N + k], s);
  }
  u[(long long)k * g.plane + (long long)j * g.px + i] = s;
}

struct Pool {
  char* base = nullptr;
  size_t bytes = 0;
  std::map<size_t, size_t> used;  // offset -> size
  char* alloc(size_t n) {
    n = (n + 255) / 256 * 256;
    size_t off = 0;
    for (auto& kv : used) {
      if (kv.first - off >= n) break;
      off = kv.first + kv.second;
    }
    if (off + n > bytes) return nullptr;
    used[off] = n;
    return base + off;
  }
  void release(char* p) {
    if (p) used.erase((size_t)(p - base));
  }
  size_t free_bytes() const {
    size_t u = 0;
    for (auto& kv : used) u += kv.second;
    return bytes - u;
  }
};

struct Req {
  uint64_t ticket = 0;
  heat3d_request in{};
  int nsteps = 0, step = 0, slot = -1;
  double t_submit = 0, t_done = 0;
  heat3d_stats st{};
  std::vector<double> result;  // dense N^3 at completion
  int status = HEAT3D_OK;
  bool done = false;
};

struct Group {
  int N = 0;
  heat3d_ctx* ctx = nullptr;
  char* chunk = nullptr;
  double* ucur = nullptr;  // [slot] pitched fields
  double* tab = nullptr;   // 3 * N * kModes doubles
  double* amp = nullptr;   // kModes doubles
  std::vector<std::shared_ptr<Req>> slots;
  int active() const {
    int a = 0;
    for (auto& s : slots) a += s != nullptr;
    return a;
  }
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct heat3d_server {
  heat3d_server_config cfg{};
  cudaStream_t st = nullptr;
  Pool pool;
  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<std::shared_ptr<Req>> pending;
  std::map<uint64_t, std::shared_ptr<Req>> all;
  std::map<int, std::unique_ptr<Group>> groups;
  std::vector<double> latencies;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  char err[512] = {0};
};

static int srv_fail(heat3d_server* s, int code, const char* msg) {
  if (s) snprintf(s->err, sizeof(s->err), "%s", msg);
  return code;
}

static heat3d_config group_config(const heat3d_server* s, int N) {
  heat3d_config c;
  heat3d_config_default(&c);
  c.nlevels = 1;
  c.levels[0] = heat3d_level{N, 2, 3};
  c.sweeps_fine = s->cfg.sweeps;
  c.tol_sdc = -1.0;
  c.mg = s->cfg.mg;
  c.precision = s->cfg.precision;
  c.forcing = HEAT3D_FORCING_NONE;
  c.batch = s->cfg.max_active;
  c.slices = 1;
  c.device = s->cfg.device;
  c.stream = s->st;
  return c;
}

static size_t group_bytes(const heat3d_server* s, int N, size_t* ws_out) {
  heat3d_config c = group_config(s, N);
  size_t ws = 0;
  if (heat3d_workspace_size(&c, &ws) != HEAT3D_OK) return 0;
  Grid g = make_grid(N);
  size_t extra = (size_t)g.fs * 8 * s->cfg.max_active + 256 + sizeof(double) * (3 * N * kModes + kModes) + 512;
  if (ws_out) *ws_out = ws;
  return ws + extra;
}

static Group* get_group(heat3d_server* s, int N) {
  auto it = s->groups.find(N);
  if (it != s->groups.end()) return it->second.get();
  size_t ws = 0;
  size_t need = group_bytes(s, N, &ws);
  char* chunk = s->pool.alloc(need);
  if (!chunk) return nullptr;
  auto g = std::make_unique<Group>();
  g->N = N;
  g->chunk = chunk;
  heat3d_config c = group_config(s, N);
  if (heat3d_init(&c, &g->ctx) != HEAT3D_OK || heat3d_bind_workspace(g->ctx, chunk, ws) != HEAT3D_OK) {
    if (g->ctx) heat3d_destroy(g->ctx);
    s->pool.release(chunk);
    return nullptr;
  }
  char* p = chunk + (ws + 255) / 256 * 256;
  Grid gr = make_grid(N);
  g->ucur = (double*)p;
  p += (size_t)gr.fs * 8 * s->cfg.max_active;
  p = (char*)(((uintptr_t)p + 255) / 256 * 256);
  g->tab = (double*)p;
  p += sizeof(double) * 3 * N * kModes;
  g->amp = (double*)p;
  g->slots.assign(s->cfg.max_active, nullptr);
  Group* raw = g.get();
  s->groups[N] = std::move(g);
  return raw;
}

static void release_group(heat3d_server* s, int N) {
  auto it = s->groups.find(N);
  if (it == s->groups.end()) return;
  heat3d_destroy(it->second->ctx);
  s->pool.release(it->second->chunk);
  s->groups.erase(it);
}

// Initial value of a newly admitted request into its slot's current field.
static int admit(heat3d_server* s, Group* g, int slot, Req& r) {
  const int N = g->N;
  std::vector<double> tab((size_t)3 * N * kModes, 0.0), amp(kModes, 0.0);
  const double h = 1.0 / (N + 1);
  int nm = std::min(r.in.nmodes, kModes);
  for (int m = 0; m < nm; ++m) {
    amp[m] = r.in.amp[m];
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < N; ++i) tab[((size_t)m * 3 + a) * N + i] = sin(M_PI * r.in.k[m][a] * (i + 1) * h);
  }
  if (cudaMemcpyAsync(g->tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
      cudaMemcpyAsync(g->amp, amp.data(), sizeof(double) * kModes, cudaMemcpyHostToDevice, s->st) != cudaSuccess)
    return HEAT3D_ECUDA;
  Grid gr = make_grid(N);
  k_modes_ic<<<dim3((N + 31) / 32, (N + 7) / 8, N), dim3(32, 8), 0, s->st>>>(
      gr, nm, g->tab, g->amp, g->ucur + (size_t)slot * gr.fs);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return HEAT3D_ECUDA;
  g->slots[slot] = nullptr;  // assigned by the caller
  r.slot = slot;
  r.step = 0;
  return HEAT3D_OK;
}

// One time step for every resident request of the group.
static int step_group(heat3d_server* s, Group* g, std::vector<std::shared_ptr<Req>>& finished) {
  heat3d_ctx* c = g->ctx;
  SdcLevel& L = c->lv[0];
  std::vector<std::shared_ptr<Req>> act;
  for (auto& r : g->slots)
    if (r) act.push_back(r);
  const int A = (int)act.size();
  if (A == 0) return HEAT3D_OK;
  const Grid& gr = L.g;
  const int M = L.L.M;
  for (int i = 0; i < A; ++i) {
    L.nu[i] = act[i]->in.nu;
    L.dt[i] = act[i]->in.dt;
    h3d_fill_item(c, 0, i, act[i]->step * act[i]->in.dt);
  }
  int rc = h3d_set_item_operators(c, 0, 0, A);
  if (rc < 0) return rc;
  rc = h3d_upload_items(c, 0, 0, A);
  if (rc < 0) return rc;
  for (int i = 0; i < A; ++i) {
    if (launch_copy(gr, M, g->ucur + (size_t)act[i]->slot * gr.fs, 0, L.U + (size_t)i * M * gr.fs, gr.fs,
                    s->st) != cudaSuccess)
      return HEAT3D_ECUDA;
  }
  rc = h3d_eval_F(c, 0, 0, A);
  if (rc < 0) return rc;
  heat3d_stats st{};
  int status = HEAT3D_OK;
  for (int k = 0; k < s->cfg.sweeps; ++k) {
    rc = h3d_sweep(c, 0, 0, A, -1.0, &st);
    if (rc == HEAT3D_ENOTCONV) status = rc;
    else if (rc < 0) return rc;
  }
  for (int i = 0; i < A; ++i) {
    if (launch_copy(gr, 1, L.U + ((size_t)i * M + M - 1) * gr.fs, 0, g->ucur + (size_t)act[i]->slot * gr.fs, 0,
                    s->st) != cudaSuccess)
      return HEAT3D_ECUDA;
    Req& r = *act[i];
    r.step += 1;
    r.st.sweeps += s->cfg.sweeps;
    r.st.steps += 1;
    r.st.vcycles += st.vcycles / std::max(A, 1);
    if (status == HEAT3D_ENOTCONV) r.status = status;
    if (r.step >= r.nsteps) finished.push_back(act[i]);
  }
  for (auto& fr : finished) {
    if (fr->slot < 0 || g->slots[fr->slot] != fr) continue;
    const size_t n = (size_t)gr.N * gr.N * gr.N;
    fr->result.resize(n);
    rc = h3d_store_dense(c, 0, g->ucur + (size_t)fr->slot * gr.fs, fr->result.data());
    if (rc < 0) return rc;
    g->slots[fr->slot] = nullptr;
    fr->slot = -1;
  }
  return HEAT3D_OK;
}

static void worker_loop(heat3d_server* s) {
  cudaSetDevice(s->cfg.device);
  std::vector<std::shared_ptr<Req>> waiting;  // admitted order (FIFO)
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool idle = waiting.empty();
      for (auto& kv : s->groups) idle = idle && kv.second->active() == 0;
      if (idle && s->pending.empty()) {
        s->cv_submit.wait(lk, [&] { return s->stop || !s->pending.empty(); });
      }
      if (s->stop) return;
      while (!s->pending.empty()) {
        waiting.push_back(s->pending.front());
        s->pending.pop_front();
      }
    }
    // admission in arrival order; a request that cannot be placed keeps its place
    for (size_t q = 0; q < waiting.size();) {
      auto r = waiting[q];
      Group* g = get_group(s, r->in.N);
      if (!g) {
        // free empty groups of other sizes to make room, then retry once
        std::vector<int> empty;
        for (auto& kv : s->groups)
          if (kv.second->active() == 0 && kv.first != r->in.N) empty.push_back(kv.first);
        for (int N : empty) release_group(s, N);
        g = get_group(s, r->in.N);
      }
      int slot = -1;
      if (g)
        for (int i = 0; i < (int)g->slots.size(); ++i)
          if (!g->slots[i]) { slot = i; break; }
      if (!g || slot < 0) { ++q; continue; }
      int rc = admit(s, g, slot, *r);
      if (rc < 0) {
        std::lock_guard<std::mutex> lk(s->mu);
        r->status = rc;
        r->done = true;
        r->t_done = now_s();
        waiting.erase(waiting.begin() + q);
        s->cv_done.notify_all();
        continue;
      }
      g->slots[slot] = r;
      waiting.erase(waiting.begin() + q);
    }
    std::vector<std::shared_ptr<Req>> finished;
    for (auto& kv : s->groups) {
      std::vector<std::shared_ptr<Req>> fin;
      int rc = step_group(s, kv.second.get(), fin);
      if (rc < 0) {
        for (auto& r : kv.second->slots)
          if (r) { r->status = rc; fin.push_back(r); r->slot = -1; }
        std::fill(kv.second->slots.begin(), kv.second->slots.end(), nullptr);
      }
      finished.insert(finished.end(), fin.begin(), fin.end());
    }
    if (!finished.empty()) {
      double t = now_s();
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& r : finished) {
        r->t_done = t;
        r->st.seconds = t - r->t_submit;
        r->done = true;
        if (r->status == HEAT3D_OK) s->latencies.push_back(r->st.seconds);
      }
      s->cv_done.notify_all();
    }
  }
}

extern "C" {

int heat3d_server_create(const heat3d_server_config* cfg, heat3d_server** out) {
  if (!cfg || !out || !cfg->pool || cfg->pool_bytes == 0 || cfg->max_active < 1 || cfg->sweeps < 1)
    return HEAT3D_EINVAL;
  if (cfg->precision != HEAT3D_FP64 && cfg->precision != HEAT3D_MIXED) return HEAT3D_EINVAL;
  if (cfg->mg.nu1 < 1 || cfg->mg.max_cycles < 1 || !(cfg->mg.rel >= 0 && cfg->mg.rel < 1))
    return HEAT3D_EINVAL;
  auto* s = new heat3d_server();
  s->cfg = *cfg;
  if (cudaSetDevice(cfg->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return HEAT3D_ECUDA;
  }
  char* base = (char*)(((uintptr_t)cfg->pool + 255) / 256 * 256);
  s->pool.base = base;
  s->pool.bytes = cfg->pool_bytes - (size_t)(base - (char*)cfg->pool);
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return HEAT3D_OK;
}

int heat3d_submit(heat3d_server* s, const heat3d_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return HEAT3D_EINVAL;
  if (!(req->N >= 3 && ((req->N + 1) & req->N) == 0) || !(req->nu > 0) || !(req->dt > 0) ||
      !(req->T > 0) || req->nmodes < 0 || req->nmodes > kModes)
    return srv_fail(s, HEAT3D_EINVAL, "bad request");
  double ns = req->T / req->dt;
  int nsteps = (int)llround(ns);
  if (nsteps < 1 || fabs(ns - nsteps) > 1e-9 * ns) return srv_fail(s, HEAT3D_EINVAL, "T must be a multiple of dt");
  if (group_bytes(s, req->N, nullptr) > s->pool.bytes)
    return srv_fail(s, HEAT3D_ENOMEM, "request can never fit in the pool");
  auto r = std::make_shared<Req>();
  r->in = *req;
  r->nsteps = nsteps;
  r->t_submit = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  r->ticket = s->next_ticket++;
  s->all[r->ticket] = r;
  s->pending.push_back(r);
  *ticket = r->ticket;
  s->cv_submit.notify_all();
  return HEAT3D_OK;
}

int heat3d_poll(heat3d_server* s, uint64_t ticket, int* done) {
  if (!s || !done) return HEAT3D_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return srv_fail(s, HEAT3D_EINVAL, "unknown ticket");
  *done = it->second->done ? 1 : 0;
  return HEAT3D_OK;
}

int heat3d_wait(heat3d_server* s, uint64_t ticket, double* u_out, heat3d_stats* stats) {
  if (!s) return HEAT3D_EINVAL;
  std::shared_ptr<Req> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return srv_fail(s, HEAT3D_EINVAL, "unknown ticket");
    r = it->second;
    s->cv_done.wait(lk, [&] { return r->done; });
    s->all.erase(it);
  }
  if (stats) *stats = r->st;
  if (r->status < 0 && r->status != HEAT3D_ENOTCONV) return r->status;
  if (u_out && !r->result.empty()) {
    cudaPointerAttributes a;
    bool dev = cudaPointerGetAttributes(&a, u_out) == cudaSuccess && a.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    if (dev) {
      if (cudaMemcpy(u_out, r->result.data(), r->result.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return HEAT3D_ECUDA;
    } else {
      memcpy(u_out, r->result.data(), r->result.size() * 8);
    }
  }
  return r->status;
}

int heat3d_server_latency(heat3d_server* s, double* p50, double* p99, long long* completed) {
  if (!s) return HEAT3D_EINVAL;
  std::vector<double> v;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    v = s->latencies;
  }
  if (completed) *completed = (long long)v.size();
  if (v.empty()) {
    if (p50) *p50 = 0;
    if (p99) *p99 = 0;
    return HEAT3D_OK;
  }
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) {
    size_t i = (size_t)ceil(q * v.size()) - 1;
    return v[std::min(i, v.size() - 1)];
  };
  if (p50) *p50 = pct(0.50);
  if (p99) *p99 = pct(0.99);
  return HEAT3D_OK;
}

int heat3d_server_destroy(heat3d_server* s) {
  if (!s) return HEAT3D_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_submit.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaStreamSynchronize(s->st);
  std::vector<int> Ns;
  for (auto& kv : s->groups) Ns.push_back(kv.first);
  for (int N : Ns) release_group(s, N);
  cudaStreamDestroy(s->st);
  delete s;
  return HEAT3D_OK;
}

const char* heat3d_server_last_error(const heat3d_server* s) { return s ? s->err : "null server"; }

}  // extern "C"

void h3d_destroy_extras(heat3d_ctx*) {}
