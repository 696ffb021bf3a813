// server.cu -- continuous-batching serving loop for independent heat-equation
// solves (zero forcing, 3-node SDC, 7-point Laplacian, fixed sweeps per step).
//
// Requests are grouped by grid size N.  A group owns one heat3d context whose
// item slots hold the requests resident on the device, its own CUDA stream
// and its own stepping thread; its workspace, plus one pitched "current
// value" field per slot and the initial-value tables, come from the caller's
// device pool through a first-fit sub-allocator.  The admission thread hands
// a request to its group when the group has a free slot and (for a new group)
// the pool has room; otherwise the request waits in arrival order.  Each
// group thread advances its group by one time step per round: requests handed
// over since the last round get their initial values, the resident requests
// are packed into items 0..A-1, swept together (per-item nu, dt, forcing
// data, multigrid masks) and unpacked.  A request whose last step is done is
// copied to host memory and its slot freed at once; a waiting request takes
// it in the next round.  Groups of different sizes run on their own streams
// from their own threads, so their kernels overlap on the device and a small
// request does not wait behind a large one's step.  Each item's arithmetic
// depends only on its own data, so a result is the same alone or in any mix.
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
  cudaStream_t st = nullptr;
  char* chunk = nullptr;
  double* ucur = nullptr;  // [slot] pitched fields
  double* tab = nullptr;   // 3 * N * kModes doubles
  double* amp = nullptr;   // kModes doubles
  std::vector<std::shared_ptr<Req>> slots;  // the group thread's own
  // guarded by the server mutex:
  std::deque<std::shared_ptr<Req>> incoming;  // handed over, not yet started
  int reserved = 0;                           // residents + incoming
  bool stop = false;
  std::condition_variable cv;  // wakes the group thread
  std::thread th;
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
  Pool pool;  // the admission thread's own
  std::mutex mu;
  std::condition_variable cv_submit, cv_done;
  std::deque<std::shared_ptr<Req>> pending;
  std::map<uint64_t, std::shared_ptr<Req>> all;
  std::map<int, std::unique_ptr<Group>> groups;  // created and released by the admission thread
  std::vector<double> latencies;
  uint64_t next_ticket = 1;
  uint64_t freed = 0;  // counts slot releases, so that waiting requests are retried
  bool stop = false;
  std::thread worker;
  char err[512] = {0};
};

static int srv_fail(heat3d_server* s, int code, const char* msg) {
  if (s) snprintf(s->err, sizeof(s->err), "%s", msg);
  return code;
}

static heat3d_config group_config(const heat3d_server* s, int N, cudaStream_t st) {
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
  c.stream = st;
  // V-cycles replayed from CUDA graphs with the stop rule on the device (one
  // graph per substep and number of resident requests, captured on first use)
  c.use_graphs = 1;
  return c;
}

static size_t group_bytes(const heat3d_server* s, int N, size_t* ws_out) {
  heat3d_config c = group_config(s, N, nullptr);
  size_t ws = 0;
  if (heat3d_workspace_size(&c, &ws) != HEAT3D_OK) return 0;
  Grid g = make_grid(N);
  size_t extra = (size_t)g.fs * 8 * s->cfg.max_active + 256 + sizeof(double) * (3 * N * kModes + kModes) + 512;
  if (ws_out) *ws_out = ws;
  return ws + extra;
}

static void group_loop(heat3d_server* s, Group* g);

// The group of size N, created (context, stream, pool chunk, thread) when
// there is none; nullptr when the pool has no room for it.
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
  if (cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking) != cudaSuccess) {
    s->pool.release(chunk);
    return nullptr;
  }
  heat3d_config c = group_config(s, N, g->st);
  if (heat3d_init(&c, &g->ctx) != HEAT3D_OK || heat3d_bind_workspace(g->ctx, chunk, ws) != HEAT3D_OK) {
    if (g->ctx) heat3d_destroy(g->ctx);
    cudaStreamDestroy(g->st);
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
  raw->th = std::thread(group_loop, s, raw);
  return raw;
}

// Stops the group's thread (the group holds no request) and returns its memory.
static void release_group(heat3d_server* s, int N) {
  auto it = s->groups.find(N);
  if (it == s->groups.end()) return;
  Group* g = it->second.get();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    g->stop = true;
    g->cv.notify_all();
  }
  if (g->th.joinable()) g->th.join();
  cudaStreamSynchronize(g->st);
  heat3d_destroy(g->ctx);
  cudaStreamDestroy(g->st);
  s->pool.release(g->chunk);
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
  // the next admission of this group reuses the tables: stream order keeps
  // them intact until this request's kernel has read them, and a copy from
  // pageable memory has taken the host data when the call returns
  if (cudaMemcpyAsync(g->tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, g->st) != cudaSuccess ||
      cudaMemcpyAsync(g->amp, amp.data(), sizeof(double) * kModes, cudaMemcpyHostToDevice, g->st) != cudaSuccess)
    return HEAT3D_ECUDA;
  Grid gr = make_grid(N);
  k_modes_ic<<<dim3((N + 31) / 32, (N + 7) / 8, N), dim3(32, 8), 0, g->st>>>(
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
                    g->st) != cudaSuccess)
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
  if (s->cfg.precision == HEAT3D_MIXED) {  // a lost TMA plane copy fails the step
    int lost = 0;
    if (loader_timeouts_take(g->st, &lost) != cudaSuccess) return HEAT3D_ECUDA;
    if (lost) return HEAT3D_ETIMEOUT;
  }
  for (int i = 0; i < A; ++i) {
    if (launch_copy(gr, 1, L.U + ((size_t)i * M + M - 1) * gr.fs, 0, g->ucur + (size_t)act[i]->slot * gr.fs, 0,
                    g->st) != cudaSuccess)
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

// Marks finished requests done and frees their slots for waiting requests.
static void complete(heat3d_server* s, Group* g, std::vector<std::shared_ptr<Req>>& fin) {
  if (fin.empty()) return;
  double t = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& r : fin) {
    r->t_done = t;
    r->st.seconds = t - r->t_submit;
    r->done = true;
    if (r->status == HEAT3D_OK) s->latencies.push_back(r->st.seconds);
  }
  g->reserved -= (int)fin.size();
  s->freed += 1;
  s->cv_done.notify_all();
  s->cv_submit.notify_all();
}

// A group's thread: starts the requests handed over to it, then advances its
// residents by one time step per round on the group's stream.
static void group_loop(heat3d_server* s, Group* g) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    std::deque<std::shared_ptr<Req>> inc;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      g->cv.wait(lk, [&] { return s->stop || g->stop || !g->incoming.empty() || g->active() > 0; });
      if (s->stop) return;
      if (g->stop && g->incoming.empty() && g->active() == 0) return;
      inc.swap(g->incoming);
    }
    std::vector<std::shared_ptr<Req>> fin;
    for (auto& r : inc) {
      int slot = -1;
      for (int i = 0; i < (int)g->slots.size(); ++i)
        if (!g->slots[i]) { slot = i; break; }
      int rc = slot < 0 ? HEAT3D_EINVAL : admit(s, g, slot, *r);
      if (rc < 0) {
        r->status = rc;
        fin.push_back(r);
        continue;
      }
      g->slots[slot] = r;
    }
    int rc = step_group(s, g, fin);
    if (rc < 0) {
      for (auto& r : g->slots)
        if (r) { r->status = rc; fin.push_back(r); r->slot = -1; }
      std::fill(g->slots.begin(), g->slots.end(), nullptr);
    }
    complete(s, g, fin);
  }
}

// The admission thread: hands requests, in arrival order, to their group when
// it has a free slot (creating the group, or releasing idle groups of other
// sizes to make room for it); a request that cannot be placed keeps its place.
static void worker_loop(heat3d_server* s) {
  cudaSetDevice(s->cfg.device);
  std::vector<std::shared_ptr<Req>> waiting;  // arrival order (FIFO)
  uint64_t seen = 0;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_submit.wait(lk, [&] {
        return s->stop || !s->pending.empty() || (!waiting.empty() && s->freed != seen);
      });
      if (s->stop) return;
      seen = s->freed;
      while (!s->pending.empty()) {
        waiting.push_back(s->pending.front());
        s->pending.pop_front();
      }
    }
    for (size_t q = 0; q < waiting.size();) {
      auto r = waiting[q];
      Group* g = get_group(s, r->in.N);
      if (!g) {
        std::vector<int> idle;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          for (auto& kv : s->groups)
            if (kv.second->reserved == 0 && kv.first != r->in.N) idle.push_back(kv.first);
        }
        for (int N : idle) release_group(s, N);
        g = get_group(s, r->in.N);
      }
      bool placed = false;
      if (g) {
        std::lock_guard<std::mutex> lk(s->mu);
        if (g->reserved < s->cfg.max_active) {
          g->incoming.push_back(r);
          g->reserved += 1;
          g->cv.notify_all();
          placed = true;
        }
      }
      if (placed) waiting.erase(waiting.begin() + q);
      else ++q;
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
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
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
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->groups) kv.second->cv.notify_all();
  }
  std::vector<int> Ns;
  for (auto& kv : s->groups) Ns.push_back(kv.first);
  for (int N : Ns) release_group(s, N);
  delete s;
  return HEAT3D_OK;
}

const char* heat3d_server_last_error(const heat3d_server* s) { return s ? s->err : "null server"; }

}  // extern "C"

void h3d_destroy_extras(heat3d_ctx*) {}
