// Batched solves: many RVEs of uneven size, each with several load cases, advanced together.
//
// Every (RVE, load case) pair is one problem of a shared Engine: one persistent operator launch,
// one update and one direction launch per iteration serve all of them, recorded once as a CUDA
// graph of K iterations and replayed.  The operator tiling of each grid size comes from the
// autotuner's record (elas_batch_autotune) or the cost model.  A problem's iterates depend only on
// its own grid, tiling and load, so its result is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"

using namespace elas;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
thread_local std::string g_batch_err;

struct RveDev {
  GridHost grid;
  Geo geo{};
  Tiling tl{};
  int32_t* phase = nullptr;
  double* coef64 = nullptr;
  float* coef32 = nullptr;
  double* cfull = nullptr;
  void* minv = nullptr;
};

struct ProbDev {
  int rve = 0, rhs = 0;
  double* sig = nullptr;
  double* w = nullptr;
  float *w_hi = nullptr, *w_lo = nullptr;
  void *g = nullptr, *h = nullptr, *Ah = nullptr, *z = nullptr;
  double* parts = nullptr;
  long long stride = 0;
};

struct Carve {
  char* base;
  size_t off = 0;
  char* take(size_t bytes) {
    char* p = base ? base + off : nullptr;
    off = align_up(off + bytes);
    return p;
  }
};

}  // namespace

struct elas_batch {
  int n_rve = 0, n_rhs = 0, precision = ELAS_PREC_MIXED;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  std::vector<RveDev> rves;
  std::vector<ProbDev> probs;
  Engine main, aux;
  double* parts_stress = nullptr;
  DevState* stress_state = nullptr;
  char* main_tables = nullptr;
  char* aux_tables = nullptr;
  long long max_stride = 0, cap_apply = 0, cap_vec = 0;
  std::string err;
};

namespace {

int bfail(elas_batch* b, int code, const std::string& m) {
  if (b)
    b->err = m;
  else
    g_batch_err = m;
  return code;
}

// Workspace layout (sizing when base == nullptr).  Per RVE: ids, tables, Jacobi inverse; per
// problem: load-case sigma, w (FP64 and the mixed pair), g, h, Ah, z and per-item partials.
size_t batch_carve(elas_batch* b, char* base, int n_rve, const elas_rve* rv, int n_rhs, int precision,
                   const std::vector<Tiling>& tls) {
  const bool mixed = precision == ELAS_PREC_MIXED;
  const size_t vb = mixed ? sizeof(float) : sizeof(double);
  (void)tls;
  long long cap_apply = 0, cap_vec = 0, max_bound = 0;
  for (int i = 0; i < n_rve; ++i) {
    const long long N = (long long)rv[i].nx * rv[i].ny * rv[i].nz;
    cap_apply += (long long)n_rhs * max_tiles_bound(N);  // room for any tiling the autotuner picks
    cap_vec += (long long)n_rhs * chunks_of(N);
    max_bound = std::max(max_bound, std::max(max_tiles_bound(N), chunks_of(N)));
  }
  Carve cv{base};
  char* t_main = cv.take(engine_table_bytes(n_rve * n_rhs, cap_apply, cap_vec));
  char* t_aux = cv.take(engine_table_bytes(1, max_bound, max_bound));
  double* parts_stress = (double*)cv.take(sizeof(double) * 6 * kMaxParts);
  if (b) {
    b->main_tables = t_main;
    b->aux_tables = t_aux;
    b->parts_stress = parts_stress;
    b->max_stride = max_bound;
    b->cap_apply = cap_apply;
    b->cap_vec = cap_vec;
  }
  for (int i = 0; i < n_rve; ++i) {
    const long long N = (long long)rv[i].nx * rv[i].ny * rv[i].nz;
    const size_t P = (size_t)std::max(rv[i].n_phases, 1);
    int32_t* phase = (int32_t*)cv.take(sizeof(int32_t) * N);
    double* coef64 = (double*)cv.take(sizeof(double) * kCoefStride * P);
    float* coef32 = (float*)cv.take(sizeof(float) * kCoef32Stride * P);
    double* cfull = (double*)cv.take(sizeof(double) * kSymStride * P);
    void* minv = cv.take(vb * 6 * N);
    if (b) {
      RveDev& R = b->rves[i];
      R.phase = phase; R.coef64 = coef64; R.coef32 = coef32; R.cfull = cfull; R.minv = minv;
    }
    const long long stride = std::max(max_tiles_bound(N), chunks_of(N));
    for (int r = 0; r < n_rhs; ++r) {
      ProbDev pd;
      pd.rve = i;
      pd.rhs = r;
      pd.sig = (double*)cv.take(sizeof(double) * 6 * P);
      pd.w = (double*)cv.take(sizeof(double) * 3 * N);
      pd.w_hi = mixed ? (float*)cv.take(sizeof(float) * 3 * N) : nullptr;
      pd.w_lo = mixed ? (float*)cv.take(sizeof(float) * 3 * N) : nullptr;
      pd.g = cv.take(vb * 3 * N);
      pd.h = cv.take(vb * 3 * N);
      pd.Ah = cv.take(vb * 3 * N);
      pd.z = cv.take(vb * 3 * N);
      pd.parts = (double*)cv.take(sizeof(double) * kPartsSlots * stride);
      pd.stride = stride;
      if (b) b->probs.push_back(pd);
    }
  }
  return cv.off;
}

std::vector<Tiling> batch_tilings(int n_rve, const elas_rve* rv, int precision, int sm_count) {
  std::vector<Tiling> tls;
  for (int i = 0; i < n_rve; ++i)
    tls.push_back(choose_tiling(Geo{rv[i].nx, rv[i].ny, rv[i].nz, (long long)rv[i].nx * rv[i].ny * rv[i].nz},
                                precision == ELAS_PREC_MIXED ? 4 : 8, sm_count));
  return tls;
}

Prob prob_of(elas_batch* b, const ProbDev& pd) {
  const RveDev& R = b->rves[pd.rve];
  Prob p{};
  p.nx = R.geo.nx; p.ny = R.geo.ny; p.nz = R.geo.nz; p.N = R.geo.N;
  p.tx = R.tl.tx; p.ty = R.tl.ty; p.kc = R.tl.kc; p.tiles_x = R.tl.tiles_x; p.tiles_y = R.tl.tiles_y;
  p.n_tiles = (int)R.tl.n_tiles;
  p.n_chunks = (int)chunks_of(R.geo.N);
  p.parts_stride = (int)pd.stride;
  p.phase = R.phase;
  p.coef64 = R.coef64;
  p.coef32 = R.coef32;
  p.sig = pd.sig;
  p.minv = R.minv;
  p.w = pd.w; p.w_hi = pd.w_hi; p.w_lo = pd.w_lo;
  p.g = pd.g; p.h = pd.h; p.Ah = pd.Ah; p.z = pd.z;
  p.z_bytes = (long long)(b->precision == ELAS_PREC_MIXED ? sizeof(float) : sizeof(double)) * 3 * R.geo.N;
  p.parts = pd.parts;
  return p;
}

int sm_count_now(int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ELAS_ERR_CUDA;
  if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ELAS_ERR_CUDA;
  return ELAS_OK;
}

}  // namespace

extern "C" {

const char* elas_batch_last_error(const elas_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

int elas_batch_workspace_bytes(int n_rve, const elas_rve* rves, int n_rhs, int precision, size_t* bytes) {
  if (!bytes || n_rve <= 0 || !rves || n_rhs <= 0 || (precision != ELAS_PREC_FP64 && precision != ELAS_PREC_MIXED))
    return bfail(nullptr, ELAS_ERR_INVALID_ARG, "elas_batch_workspace_bytes: bad arguments");
  for (int i = 0; i < n_rve; ++i)
    if (rves[i].nx < 2 || rves[i].ny < 2 || rves[i].nz < 2 || rves[i].n_phases < 0)
      return bfail(nullptr, ELAS_ERR_INVALID_ARG, "elas_batch_workspace_bytes: grid dimensions must be >= 2");
  *bytes = batch_carve(nullptr, nullptr, n_rve, rves, n_rhs, precision, {});
  return ELAS_OK;
}

int elas_batch_create(elas_batch** out, int n_rve, const elas_rve* rves, int n_rhs, int precision, void* workspace,
                      size_t ws_bytes, void* cuda_stream) {
  if (!out) return bfail(nullptr, ELAS_ERR_INVALID_ARG, "elas_batch_create: out is NULL");
  *out = nullptr;
  if (n_rve <= 0 || !rves || n_rhs <= 0 || (precision != ELAS_PREC_FP64 && precision != ELAS_PREC_MIXED))
    return bfail(nullptr, ELAS_ERR_INVALID_ARG, "elas_batch_create: bad arguments");
  int sms = 0;
  if (sm_count_now(&sms) != ELAS_OK) return bfail(nullptr, ELAS_ERR_CUDA, "elas_batch_create: device query");
  elas_batch* b = new elas_batch();
  b->n_rve = n_rve;
  b->n_rhs = n_rhs;
  b->precision = precision;
  b->stream = (cudaStream_t)cuda_stream;
  b->sm_count = sms;
  b->rves.resize(n_rve);
  auto bail = [&](int code) {
    g_batch_err = b->err;
    engine_destroy(b->main);
    engine_destroy(b->aux);
    delete b;
    return code;
  };
  for (int i = 0; i < n_rve; ++i) {
    std::string m;
    int r = grid_prepare(b->rves[i].grid, rves[i].nx, rves[i].ny, rves[i].nz, rves[i].phase_id, rves[i].n_phases,
                         rves[i].C_local, rves[i].rodrigues, &m);
    if (r != ELAS_OK) {
      char buf[48];
      std::snprintf(buf, sizeof buf, "elas_batch_create: RVE %d: ", i);
      return bail(bfail(b, r, buf + m));
    }
    b->rves[i].geo = Geo{rves[i].nx, rves[i].ny, rves[i].nz, b->rves[i].grid.N};
  }
  const std::vector<Tiling> tls = batch_tilings(n_rve, rves, precision, sms);
  const size_t need = batch_carve(nullptr, nullptr, n_rve, rves, n_rhs, precision, tls);
  if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || ws_bytes < need) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "elas_batch_create: workspace needs %zu bytes, 256-byte aligned (got %zu)", need,
                  ws_bytes);
    return bail(bfail(b, ELAS_ERR_WORKSPACE, buf));
  }
  batch_carve(b, (char*)workspace, n_rve, rves, n_rhs, precision, tls);
  for (int i = 0; i < n_rve; ++i) b->rves[i].tl = tls[i];
  const bool mixed = precision == ELAS_PREC_MIXED;
  std::string m;
  int r = engine_init(b->main, mixed, sms, apply_max_threads(mixed ? 4 : 8), n_rve * n_rhs, b->cap_apply, b->cap_vec,
                      b->main_tables, b->stream, &m);
  if (r == ELAS_OK)
    r = engine_init(b->aux, mixed, sms, apply_max_threads(mixed ? 4 : 8), 1, b->max_stride, b->max_stride,
                    b->aux_tables, b->stream, &m);
  if (r != ELAS_OK) return bail(bfail(b, r, "elas_batch_create: " + m));
  b->stress_state = b->aux.d_states;
  // uploads
  cudaStream_t s = b->stream;
  for (int i = 0; i < n_rve; ++i) {
    RveDev& R = b->rves[i];
    cudaError_t e = cudaMemcpyAsync(R.phase, rves[i].phase_id, sizeof(int32_t) * R.geo.N, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(R.coef64, R.grid.coef64.data(), sizeof(double) * R.grid.coef64.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(R.coef32, R.grid.coef32.data(), sizeof(float) * R.grid.coef32.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(R.cfull, R.grid.cfull.data(), sizeof(double) * R.grid.cfull.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(bfail(b, ELAS_ERR_CUDA, std::string("elas_batch_create: upload: ") + cudaGetErrorString(e)));
  }
  std::vector<Prob> ps;
  for (const ProbDev& pd : b->probs) ps.push_back(prob_of(b, pd));
  r = engine_set_problems(b->main, ps, &m);
  if (r != ELAS_OK) return bail(bfail(b, r, "elas_batch_create: " + m));
  *out = b;
  return ELAS_OK;
}

void elas_batch_destroy(elas_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  engine_destroy(b->main);
  engine_destroy(b->aux);
  delete b;
}

int elas_batch_set_fp64_operator(elas_batch* b, int form) {
  if (!b) return ELAS_ERR_INVALID_ARG;
  if (form != ELAS_FP64_OP_PAIRED && form != ELAS_FP64_OP_NATIVE) {
    b->err = "elas_batch_set_fp64_operator: form must be ELAS_FP64_OP_PAIRED or _NATIVE";
    return ELAS_ERR_INVALID_ARG;
  }
  engine_set_ff64(b->main, form == ELAS_FP64_OP_PAIRED);
  engine_set_ff64(b->aux, form == ELAS_FP64_OP_PAIRED);
  return ELAS_OK;
}

int elas_batch_autotune(elas_batch* b, int max_candidates) {
  if (!b) return ELAS_ERR_INVALID_ARG;
  const bool mixed = b->precision == ELAS_PREC_MIXED;
  const int eb = mixed ? 4 : 8;
  const size_t vb = mixed ? sizeof(float) : sizeof(double);
  std::map<std::tuple<int, int, int>, Tiling> done;
  std::string m;
  for (size_t k = 0; k < b->probs.size(); ++k) {
    ProbDev& pd = b->probs[k];
    RveDev& R = b->rves[pd.rve];
    const auto key = std::make_tuple(R.geo.nx, R.geo.ny, R.geo.nz);
    auto it = done.find(key);
    if (it == done.end()) {
      if (cudaMemsetAsync(pd.h, 0, vb * 3 * R.geo.N, b->stream) != cudaSuccess)
        return bfail(b, ELAS_ERR_CUDA, "elas_batch_autotune: memset");
      Prob proto = prob_of(b, pd);
      proto.parts = pd.parts;
      proto.parts_stride = (int)pd.stride;
      Tiling best{};
      // candidates must fit the problem's partial-sum buffer
      int r = tune_tiling(b->aux, proto, eb, b->sm_count, pd.stride, max_candidates, &best, nullptr, &m);
      if (r != ELAS_OK) return bfail(b, r, "elas_batch_autotune: " + m);
      it = done.emplace(key, best).first;
    }
    R.tl = it->second;
  }
  std::vector<Prob> ps;
  for (const ProbDev& pd : b->probs) ps.push_back(prob_of(b, pd));
  int r = engine_set_problems(b->main, ps, &m);
  if (r != ELAS_OK) return bfail(b, r, "elas_batch_autotune: " + m);
  return ELAS_OK;
}

int elas_batch_solve(elas_batch* b, const double* strains, double tol, int max_iter, const elas_solve_opts* opts,
                     elas_solve_info* infos) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!b) return ELAS_ERR_INVALID_ARG;
  const int n = (int)b->probs.size();
  if (!strains || !(tol >= 0.0) || max_iter < 0) return bfail(b, ELAS_ERR_INVALID_ARG, "elas_batch_solve: bad arguments");
  for (int i = 0; i < 6 * n; ++i)
    if (!std::isfinite(strains[i])) return bfail(b, ELAS_ERR_INVALID_ARG, "elas_batch_solve: non-finite strain");
  const bool mixed = b->precision == ELAS_PREC_MIXED;
  int stop_rule = mixed ? ELAS_STOP_TRUE : ELAS_STOP_PRECOND;
  int replace_every = mixed ? 50 : 0;
  double drop2 = 0.0;
  int K = 0;
  if (opts) {
    if (opts->precond != ELAS_PRECOND_BLOCK)
      return bfail(b, ELAS_ERR_INVALID_ARG, "elas_batch_solve: batches use the point-block Jacobi preconditioner");
    if (opts->stop_rule == ELAS_STOP_PRECOND || opts->stop_rule == ELAS_STOP_TRUE) stop_rule = opts->stop_rule;
    if (opts->replace_every > 0) replace_every = opts->replace_every;
    if (opts->replace_drop > 0) drop2 = std::pow(10.0, -2.0 * opts->replace_drop);
    if (opts->check_every > 0) K = opts->check_every;
  }
  if (K <= 0) K = mixed ? std::min(replace_every, 50) : 32;
  cudaStream_t s = b->stream;
  // Algorithm 2 part 1 per RVE, then per-problem loads
  for (RveDev& R : b->rves) {
    cudaError_t e = launch_jacobi(R.geo, R.phase, R.coef64, mixed ? nullptr : (double*)R.minv,
                                  mixed ? (float*)R.minv : nullptr, b->sm_count, s);
    if (e != cudaSuccess) return bfail(b, ELAS_ERR_CUDA, std::string("elas_batch_solve: Jacobi: ") + cudaGetErrorString(e));
  }
  std::vector<SolveSetup> su(n);
  for (int k = 0; k < n; ++k) {
    const ProbDev& pd = b->probs[k];
    const double* e6 = strains + 6 * k;
    std::vector<double> sig;
    su[k].bscale2 = grid_sigma(b->rves[pd.rve].grid, e6, sig);
    cudaError_t e = cudaMemcpyAsync(pd.sig, sig.data(), sizeof(double) * sig.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bfail(b, ELAS_ERR_CUDA, "elas_batch_solve: load upload");
    su[k].tol = tol;
    su[k].tol2_true = tol * tol;
    strain_tensor(e6, su[k].E);
    su[k].max_iter = max_iter;
    su[k].stop_rule = stop_rule;
    su[k].replace_every = mixed ? replace_every : 0;
    su[k].drop2 = mixed ? drop2 : 0.0;
  }
  int launches = 0;
  std::string m;
  int r = engine_solve(b->main, su, K, &launches, &m);
  if (r != ELAS_OK) return bfail(b, r, "elas_batch_solve: " + m);
  launches += (int)b->rves.size();
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bool nonfinite = false;
  for (int k = 0; k < n; ++k) {
    const DevState& hs = b->main.h_states[k];
    int status = hs.done ? hs.status : ELAS_MAX_ITER;
    if (status == ST_RUNNING) status = ELAS_MAX_ITER;
    nonfinite |= status == ELAS_NONFINITE;
    if (infos) {
      infos[k].iters = hs.iter;
      infos[k].status = status;
      infos[k].relres_precond = hs.gg0 > 0 ? std::sqrt(std::max(hs.gg, 0.0) / hs.gg0) : 0.0;
      infos[k].relres_true = hs.bb > 0 ? std::sqrt(hs.rr_true / hs.bb) : std::sqrt(hs.rr_true);
      infos[k].n_replacements = hs.n_repl;
      infos[k].launches = launches;
      infos[k].seconds = secs;
    }
  }
  if (nonfinite) return bfail(b, ELAS_ERR_NONFINITE, "elas_batch_solve: non-finite value in an iteration");
  return ELAS_OK;
}

int elas_batch_fluctuation(elas_batch* b, int rve, int rhs, double* w_out) {
  if (!b || rve < 0 || rve >= b->n_rve || rhs < 0 || rhs >= b->n_rhs || !w_out)
    return bfail(b, ELAS_ERR_INVALID_ARG, "elas_batch_fluctuation: bad arguments");
  const ProbDev& pd = b->probs[(size_t)rve * b->n_rhs + rhs];
  if (cudaMemcpyAsync(w_out, pd.w, sizeof(double) * 3 * b->rves[rve].geo.N, cudaMemcpyDeviceToDevice, b->stream) !=
      cudaSuccess)
    return bfail(b, ELAS_ERR_CUDA, "elas_batch_fluctuation: copy");
  return ELAS_OK;
}

int elas_batch_stress(elas_batch* b, int rve, int rhs, const double* strain, double* stress, double* von_mises,
                      double* macro_stress) {
  if (!b || rve < 0 || rve >= b->n_rve || rhs < 0 || rhs >= b->n_rhs || !strain)
    return bfail(b, ELAS_ERR_INVALID_ARG, "elas_batch_stress: bad arguments");
  const ProbDev& pd = b->probs[(size_t)rve * b->n_rhs + rhs];
  const RveDev& R = b->rves[rve];
  DevState* st = b->stress_state;
  cudaError_t e = launch_stress(R.geo, R.phase, R.cfull, strain, pd.w, stress, von_mises, b->parts_stress, &st->ctr[3],
                                st->macro, b->sm_count, b->stream);
  if (e != cudaSuccess) return bfail(b, ELAS_ERR_CUDA, "elas_batch_stress: launch");
  if (macro_stress) {
    if (cudaMemcpyAsync(b->aux.h_states, st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
      return bfail(b, ELAS_ERR_CUDA, "elas_batch_stress: read");
    for (int q = 0; q < 6; ++q) macro_stress[q] = b->aux.h_states[0].macro[q];
  }
  return ELAS_OK;
}

}  // extern "C"
