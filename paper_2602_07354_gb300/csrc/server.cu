// Solve server: continuous batching of elasticity solves under a device-memory budget.
//
// Requests (one RVE, one applied strain, a tolerance) arrive at any time.  Each step the server
//   1. admits queued requests in arrival order while the next one fits the budget (first-fit in a
//      device arena carved from the caller's workspace) and a slot is free: uploads its ids and
//      per-phase tables, builds its Jacobi inverse and marks it for initialisation;
//   2. advances every active request by K PCG iterations in the shared persistent launches of a
//      recorded CUDA graph (the launch shape is fixed, so the graph serves any mix of requests);
//   3. forms the final FP64 fluctuation and true residual of requests that stopped, reads the
//      states once, and moves stopped requests to the finished list.
// A request keeps its CG state resident on the device from admission to retirement, and its
// iterates depend only on its own grid, tiling and load, so its result is the same alone and in
// any mix.  Retired memory returns to the arena when the client collects the result.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "engine.h"

using namespace elas;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
thread_local std::string g_server_err;
double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing on free.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Request {
  long long id = 0;
  GridHost grid;
  std::vector<int32_t> phase;  // host copy until admission
  double strain[6] = {0, 0, 0, 0, 0, 0};
  double tol = 1e-8;
  int max_iter = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  // device block
  size_t off = 0, bytes = 0;
  Prob prob{};
  Tiling tl{};
  int slot = -1;      // index in the engine's problem table while active
  DevState final_state{};
  bool finished = false;
};

struct Layout {
  size_t phase, coef64, coef32, cfull, sig, minv, w, w_hi, w_lo, g, h, Ah, z, parts, total;
  long long stride;
};

Layout request_layout(const Geo& geo, int n_phases, bool mixed, const Tiling& tl) {
  const long long N = geo.N;
  const size_t vb = mixed ? sizeof(float) : sizeof(double);
  const size_t P = (size_t)std::max(n_phases, 1);
  Layout L{};
  L.stride = std::max<long long>(tl.n_tiles, chunks_of(N));
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = align_up(o + b);
    return at;
  };
  L.phase = take(sizeof(int32_t) * N);
  L.coef64 = take(sizeof(double) * kCoefStride * P);
  L.coef32 = take(sizeof(float) * kCoef32Stride * P);
  L.cfull = take(sizeof(double) * kSymStride * P);
  L.sig = take(sizeof(double) * 6 * P);
  L.minv = take(vb * 6 * N);
  L.w = take(sizeof(double) * 3 * N);
  L.w_hi = mixed ? take(sizeof(float) * 3 * N) : 0;
  L.w_lo = mixed ? take(sizeof(float) * 3 * N) : 0;
  L.g = take(vb * 3 * N);
  L.h = take(vb * 3 * N);
  L.Ah = take(vb * 3 * N);
  L.z = take(vb * 3 * N);
  L.parts = take(sizeof(double) * kPartsSlots * L.stride);
  L.total = o;
  return L;
}

// the largest operator tile any grid may get: the fixed launch shape of the server's graph
// (eb 4: FP32, 8: native FP64, 0: double-float)
size_t max_tile_smem(int eb) {
  size_t m = 0;
  const int threads = apply_max_threads(eb == 0 ? 8 : eb);
  for (int tx = 4; tx <= 40; ++tx)
    for (int ty = 2; ty <= 24; ++ty)
      if ((tx + 1) * (ty + 1) <= threads)
        m = std::max(m, eb == 0 ? apply_smem_bytes_ff(tx, ty) : apply_smem_bytes(tx, ty, eb));
  return m;
}

}  // namespace

struct elas_server {
  int precision = ELAS_PREC_MIXED;
  int max_active = 0, K = 50, replace_every = 50;
  double drop2 = 0.0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  char* arena_base = nullptr;
  size_t budget = 0;
  Arena arena;
  Engine eng;
  std::deque<Request*> queue;
  std::vector<Request*> slots;  // slot i = problem i of the engine (nullptr: free, no work items)
  std::map<long long, Request*> finished;
  long long next_id = 1;
  long long n_done = 0;
  bool graph_ok = false;
  std::string err;
};

namespace {

int sfail(elas_server* s, int code, const std::string& m) {
  if (s)
    s->err = m;
  else
    g_server_err = m;
  return code;
}

size_t table_bytes_for(size_t budget, int max_active) {
  const long long vox = (long long)(budget / 96) + 1;
  const long long cap_apply = vox / 48 + 4096LL * max_active;
  const long long cap_vec = vox / kVecChunk + 2LL * max_active;
  return engine_table_bytes(max_active, cap_apply, cap_vec);
}

int n_active(const elas_server* s) {
  int n = 0;
  for (const Request* r : s->slots) n += r != nullptr;
  return n;
}

// Rebuild the engine's problem table from the slots.  A request keeps its slot (and with it its
// solver state in the engine's state table) from admission to retirement; a free slot is a
// problem without work items.
int rebuild(elas_server* s) {
  int hi = 0;
  for (int i = 0; i < (int)s->slots.size(); ++i)
    if (s->slots[i]) hi = i + 1;
  std::vector<Prob> ps(hi);
  for (int i = 0; i < hi; ++i) {
    if (s->slots[i]) {
      ps[i] = s->slots[i]->prob;
    } else {
      ps[i] = Prob{};
      ps[i].nx = ps[i].ny = ps[i].nz = 2;
      ps[i].N = 8;
      ps[i].tx = ps[i].ty = 1;
      ps[i].kc = 1;
      ps[i].tiles_x = ps[i].tiles_y = 1;
      ps[i].n_tiles = 0;
      ps[i].n_chunks = 0;
    }
  }
  std::string m;
  int r = engine_set_problems(s->eng, ps, &m);
  if (r != ELAS_OK) return sfail(s, r, "server: " + m);
  return ELAS_OK;
}

}  // namespace

extern "C" {

const char* elas_server_last_error(const elas_server* s) { return s ? s->err.c_str() : g_server_err.c_str(); }

int elas_server_workspace_bytes(size_t budget_bytes, int max_active, size_t* bytes) {
  if (!bytes || max_active <= 0 || budget_bytes < (1u << 20))
    return sfail(nullptr, ELAS_ERR_INVALID_ARG, "elas_server_workspace_bytes: bad arguments");
  *bytes = align_up(budget_bytes) + table_bytes_for(budget_bytes, max_active);
  return ELAS_OK;
}

int elas_server_create(elas_server** out, size_t budget_bytes, int max_active, int precision, int iters_per_step,
                       void* workspace, size_t ws_bytes, void* cuda_stream) {
  if (!out) return sfail(nullptr, ELAS_ERR_INVALID_ARG, "elas_server_create: out is NULL");
  *out = nullptr;
  if (max_active <= 0 || budget_bytes < (1u << 20) || (precision != ELAS_PREC_FP64 && precision != ELAS_PREC_MIXED))
    return sfail(nullptr, ELAS_ERR_INVALID_ARG, "elas_server_create: bad arguments");
  const size_t need = align_up(budget_bytes) + table_bytes_for(budget_bytes, max_active);
  if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || ws_bytes < need)
    return sfail(nullptr, ELAS_ERR_WORKSPACE, "elas_server_create: workspace too small or misaligned");
  elas_server* s = new elas_server();
  s->precision = precision;
  s->max_active = max_active;
  s->stream = (cudaStream_t)cuda_stream;
  const bool mixed = precision == ELAS_PREC_MIXED;
  s->replace_every = mixed ? 50 : 0;
  s->K = iters_per_step > 0 ? iters_per_step : (mixed ? 50 : 32);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete s;
    return sfail(nullptr, ELAS_ERR_CUDA, "elas_server_create: device query");
  }
  s->slots.assign(max_active, nullptr);
  s->arena_base = (char*)workspace;
  s->budget = align_up(budget_bytes);
  s->arena.reset(s->budget);
  const long long vox = (long long)(budget_bytes / 96) + 1;
  s->eng.fixed_smem32 = max_tile_smem(4);
  s->eng.fixed_smem64 = max_tile_smem(8);
  s->eng.fixed_smemff = max_tile_smem(0);
  std::string m;
  int r = engine_init(s->eng, mixed, s->sm_count, apply_max_threads(mixed ? 4 : 8), max_active,
                      vox / 48 + 4096LL * max_active, vox / kVecChunk + 2LL * max_active, s->arena_base + s->budget,
                      s->stream, &m);
  if (r != ELAS_OK) {
    engine_destroy(s->eng);
    delete s;
    return sfail(nullptr, r, "elas_server_create: " + m);
  }
  *out = s;
  return ELAS_OK;
}

void elas_server_destroy(elas_server* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (Request* q : s->queue) delete q;
  for (Request* q : s->slots) delete q;
  for (auto& kv : s->finished) delete kv.second;
  engine_destroy(s->eng);
  delete s;
}

int elas_server_submit(elas_server* s, const elas_rve* rve, const double* strain, double tol, int max_iter,
                       long long* id) {
  if (!s || !rve || !strain || !id || !(tol >= 0.0) || max_iter < 0)
    return sfail(s, ELAS_ERR_INVALID_ARG, "elas_server_submit: bad arguments");
  for (int q = 0; q < 6; ++q)
    if (!std::isfinite(strain[q])) return sfail(s, ELAS_ERR_INVALID_ARG, "elas_server_submit: non-finite strain");
  Request* r = new Request();
  std::string m;
  int rc = grid_prepare(r->grid, rve->nx, rve->ny, rve->nz, rve->phase_id, rve->n_phases, rve->C_local,
                        rve->rodrigues, &m);
  if (rc != ELAS_OK) {
    delete r;
    return sfail(s, rc, "elas_server_submit: " + m);
  }
  const bool mixed = s->precision == ELAS_PREC_MIXED;
  const Geo geo{rve->nx, rve->ny, rve->nz, r->grid.N};
  r->tl = choose_tiling(geo, mixed ? 4 : 8, s->sm_count);
  const Layout L = request_layout(geo, rve->n_phases, mixed, r->tl);
  if (L.total > s->budget) {
    delete r;
    return sfail(s, ELAS_ERR_ADMISSION, "elas_server_submit: the request alone exceeds the memory budget");
  }
  r->bytes = L.total;
  r->phase.assign(rve->phase_id, rve->phase_id + r->grid.N);
  std::copy(strain, strain + 6, r->strain);
  r->tol = tol;
  r->max_iter = max_iter;
  r->id = s->next_id++;
  r->t_submit = now_s();
  s->queue.push_back(r);
  *id = r->id;
  return ELAS_OK;
}

int elas_server_step(elas_server* s, int* n_active_out, int* n_queued, int* n_finished) {
  if (!s) return ELAS_ERR_INVALID_ARG;
  const bool mixed = s->precision == ELAS_PREC_MIXED;
  cudaStream_t st = s->stream;
  std::string m;
  // 1. admission, in arrival order, while the head of the queue fits
  std::vector<Request*> fresh;
  while (!s->queue.empty() && n_active(s) < s->max_active) {
    Request* r = s->queue.front();
    size_t off = 0;
    if (!s->arena.alloc(r->bytes, &off)) break;
    s->queue.pop_front();
    int slot = 0;
    while (s->slots[slot]) ++slot;
    s->slots[slot] = r;
    r->slot = slot;
    r->off = off;
    r->t_admit = now_s();
    const Geo geo{r->grid.nx, r->grid.ny, r->grid.nz, r->grid.N};
    const Layout L = request_layout(geo, r->grid.n_phases, mixed, r->tl);
    char* base = s->arena_base + off;
    Prob& p = r->prob;
    p = Prob{};
    p.nx = geo.nx; p.ny = geo.ny; p.nz = geo.nz; p.N = geo.N;
    p.tx = r->tl.tx; p.ty = r->tl.ty; p.kc = r->tl.kc; p.tiles_x = r->tl.tiles_x; p.tiles_y = r->tl.tiles_y;
    p.n_tiles = (int)r->tl.n_tiles;
    p.n_chunks = (int)chunks_of(geo.N);
    p.parts_stride = (int)L.stride;
    p.phase = (int32_t*)(base + L.phase);
    p.coef64 = (double*)(base + L.coef64);
    p.coef32 = (float*)(base + L.coef32);
    p.sig = (double*)(base + L.sig);
    p.minv = base + L.minv;
    p.w = (double*)(base + L.w);
    p.w_hi = mixed ? (float*)(base + L.w_hi) : nullptr;
    p.w_lo = mixed ? (float*)(base + L.w_lo) : nullptr;
    p.g = base + L.g; p.h = base + L.h; p.Ah = base + L.Ah; p.z = base + L.z;
    p.parts = (double*)(base + L.parts);
    const GridHost& G = r->grid;
    std::vector<double> sig;
    grid_sigma(G, r->strain, sig);
    cudaError_t e = cudaMemcpyAsync((void*)p.phase, r->phase.data(), sizeof(int32_t) * G.N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void*)p.coef64, G.coef64.data(), sizeof(double) * G.coef64.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void*)p.coef32, G.coef32.data(), sizeof(float) * G.coef32.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + L.cfull, G.cfull.data(), sizeof(double) * G.cfull.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((void*)p.sig, sig.data(), sizeof(double) * sig.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)  // Algorithm 2 part 1
      e = launch_jacobi(geo, p.phase, p.coef64, mixed ? nullptr : (double*)p.minv,
                        mixed ? (float*)p.minv : nullptr, s->sm_count, st);
    if (e != cudaSuccess) return sfail(s, ELAS_ERR_CUDA, std::string("server admission: ") + cudaGetErrorString(e));
    r->phase.clear();
    r->phase.shrink_to_fit();
    fresh.push_back(r);
  }
  if (!fresh.empty()) {
    int rc = rebuild(s);
    if (rc != ELAS_OK) return rc;
    std::vector<SolveSetup> su(fresh.size());
    std::vector<int> idx(fresh.size());
    for (size_t k = 0; k < fresh.size(); ++k) {
      Request* r = fresh[k];
      std::vector<double> sig;
      su[k].bscale2 = grid_sigma(r->grid, r->strain, sig);
      su[k].tol = r->tol;
      su[k].tol2_true = r->tol * r->tol;
      strain_tensor(r->strain, su[k].E);
      su[k].max_iter = r->max_iter;
      su[k].stop_rule = mixed ? ELAS_STOP_TRUE : ELAS_STOP_PRECOND;
      su[k].replace_every = s->replace_every;
      su[k].drop2 = s->drop2;
      idx[k] = r->slot;
    }
    cudaError_t e = cudaMemcpyAsync(s->eng.d_setups, su.data(), sizeof(SolveSetup) * su.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->eng.d_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_state_init(s->eng.bd, s->eng.d_setups, s->eng.d_idx, (int)fresh.size(), st);
    if (e == cudaSuccess) e = launch_pcg_init(s->eng.bd, mixed, st);
    if (e != cudaSuccess) return sfail(s, ELAS_ERR_CUDA, std::string("server init: ") + cudaGetErrorString(e));
  }
  // 2. K iterations of every active request
  const int n_slots = (int)s->eng.probs.size();
  if (n_active(s) > 0) {
    int rc = record_batch(s->eng, s->K, &m);
    if (rc != ELAS_OK) return sfail(s, rc, "server: " + m);
    cudaError_t e = cudaGraphLaunch(s->eng.exec, st);
    // 3. final FP64 w and true residual of the requests that stopped
    if (e == cudaSuccess && mixed) e = launch_w_combine(s->eng.bd, GATE_FINALIZE, st);
    if (e == cudaSuccess) e = launch_apply(s->eng.bd, AK_F64_NORM, POST_TRUE_NORM, GATE_FINALIZE, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->eng.h_states, s->eng.d_states, sizeof(DevState) * n_slots, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return sfail(s, ELAS_ERR_CUDA, std::string("server step: ") + cudaGetErrorString(e));
    const double t = now_s();
    int retired = 0;
    for (int i = 0; i < n_slots; ++i) {
      Request* r = s->slots[i];
      if (!r) continue;
      const DevState& hs = s->eng.h_states[i];
      if (hs.done && hs.finalized) {
        r->final_state = hs;
        r->finished = true;
        r->t_done = t;
        s->finished[r->id] = r;
        s->slots[i] = nullptr;
        ++retired;
        ++s->n_done;
      }
    }
    if (retired) {
      int rc2 = rebuild(s);
      if (rc2 != ELAS_OK) return rc2;
    }
    if (n_finished) *n_finished = retired;
  } else if (n_finished) {
    *n_finished = 0;
  }
  if (n_active_out) *n_active_out = n_active(s);
  if (n_queued) *n_queued = (int)s->queue.size();
  return ELAS_OK;
}

int elas_server_poll(elas_server* s, long long id, elas_solve_info* info, double* w_out, double* latency_s,
                     int* done) {
  if (!s || !done) return sfail(s, ELAS_ERR_INVALID_ARG, "elas_server_poll: bad arguments");
  auto it = s->finished.find(id);
  if (it == s->finished.end()) {
    *done = 0;
    return ELAS_OK;
  }
  Request* r = it->second;
  const DevState& hs = r->final_state;
  *done = 1;
  if (info) {
    int status = hs.status == ST_RUNNING ? ELAS_MAX_ITER : hs.status;
    info->iters = hs.iter;
    info->status = status;
    info->relres_precond = hs.gg0 > 0 ? std::sqrt(std::max(hs.gg, 0.0) / hs.gg0) : 0.0;
    info->relres_true = hs.bb > 0 ? std::sqrt(hs.rr_true / hs.bb) : std::sqrt(hs.rr_true);
    info->n_replacements = hs.n_repl;
    info->launches = 0;
    info->seconds = r->t_done - r->t_admit;
  }
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  const bool admitted = r->bytes > 0;  // a request cancelled while queued has no device block
  if (w_out && admitted) {
    if (cudaMemcpyAsync(w_out, r->prob.w, sizeof(double) * 3 * r->grid.N, cudaMemcpyDeviceToDevice, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
      return sfail(s, ELAS_ERR_CUDA, "elas_server_poll: copy");
  }
  if (admitted) s->arena.release(r->off, r->bytes);
  s->finished.erase(it);
  delete r;
  return ELAS_OK;
}

int elas_server_cancel(elas_server* s, long long id) {
  if (!s) return ELAS_ERR_INVALID_ARG;
  if (s->finished.count(id)) return ELAS_OK;
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    Request* r = *it;
    if (r->id != id) continue;
    s->queue.erase(it);
    r->final_state = DevState{};
    r->final_state.status = ELAS_CANCELLED;
    r->final_state.done = 1;
    r->finished = true;
    r->t_done = now_s();
    r->bytes = 0;  // never admitted: no device block, no fluctuation
    s->finished[id] = r;
    ++s->n_done;
    return ELAS_OK;
  }
  for (Request* r : s->slots) {
    if (!r || r->id != id) continue;
    // between steps the stream is idle: mark the solver state stopped; the next step skips its
    // iterations, forms its final w and true residual and retires it
    const int sd[2] = {ELAS_CANCELLED, 1};  // DevState::status, DevState::done
    DevState* st = s->eng.d_states + r->slot;
    static_assert(offsetof(DevState, done) == offsetof(DevState, status) + sizeof(int), "status, done adjacent");
    cudaError_t e = cudaMemcpyAsync(&st->status, sd, sizeof sd, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return sfail(s, ELAS_ERR_CUDA, std::string("elas_server_cancel: ") + cudaGetErrorString(e));
    return ELAS_OK;
  }
  return sfail(s, ELAS_ERR_INVALID_ARG, "elas_server_cancel: unknown request id");
}

int elas_server_set_replacement(elas_server* s, int replace_every, int replace_drop) {
  if (!s) return ELAS_ERR_INVALID_ARG;
  if (replace_every < 0 || replace_drop < 0)
    return sfail(s, ELAS_ERR_INVALID_ARG, "elas_server_set_replacement: negative argument");
  if (s->replace_every == 0) return ELAS_OK;  // FP64 server: no replacements
  if (replace_every > 0) s->replace_every = replace_every;
  s->drop2 = replace_drop > 0 ? std::pow(10.0, -2.0 * replace_drop) : 0.0;
  return ELAS_OK;
}

int elas_server_stats(elas_server* s, size_t* bytes_in_use, int* n_active_out, int* n_queued, long long* n_done) {
  if (!s) return ELAS_ERR_INVALID_ARG;
  if (bytes_in_use) *bytes_in_use = s->arena.used();
  if (n_active_out) *n_active_out = n_active(s);
  if (n_queued) *n_queued = (int)s->queue.size();
  if (n_done) *n_done = s->n_done;
  return ELAS_OK;
}

}  // extern "C"
