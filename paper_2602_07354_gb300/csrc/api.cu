// C ABI of libelas: context, workspace, host-side FP64 preparation and the PCG driver.
//
// The paper's workflow (ELAS3D-Xtal, arXiv 2602.07354, Sec. 2.1.3, Fig. 1) maps onto the calls:
//   stages 1-3 (parameters, microstructure, stiffness)  -> elas_create
//   stage 4 (affine start, energy gradient)              -> first kernel of elas_pcg_solve
//   stage 5 (dembx PCG, Algorithm 2)                     -> elas_pcg_solve
//   post-processing (stress_OpenMP, full-field vM)       -> elas_stress
// All device memory comes from the caller's workspace; this file allocates none.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"

using namespace elas;

namespace {

thread_local std::string g_create_err;
constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Rodrigues formula R = I + 2/(1 + rho.rho) ([rho]x + [rho]x^2) for rho = tan(theta/2) n.
void rodrigues_matrix(const double* r, double R[3][3]) {
  const double K[3][3] = {{0, -r[2], r[1]}, {r[2], 0, -r[0]}, {-r[1], r[0], 0}};
  const double f = 2.0 / (1.0 + r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double k2 = 0.0;
      for (int m = 0; m < 3; ++m) k2 += K[i][m] * K[m][j];
      R[i][j] = (i == j ? 1.0 : 0.0) + f * (K[i][j] + k2);
    }
}

}  // namespace

namespace elas {

// Eq. 4 / Algorithm 1: C' = Q C Q^T with Q the 6x6 Bond matrix of the stress rotation
// sigma' = R sigma R^T in Voigt order 11,22,33,23,13,12: for row (i,j) and column (k,l),
// Q = R_ik R_jl (+ R_il R_jk when k != l, since the shear pair (k,l)/(l,k) shares a slot).
void bond_rotate(const double* C6_local, const double* rho, double* C6_global) {
  double R[3][3];
  rodrigues_matrix(rho, R);
  const int vi[6] = {0, 1, 2, 1, 0, 0}, vj[6] = {0, 1, 2, 2, 2, 1};
  double Q[6][6];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      const int i = vi[I], j = vj[I], k = vi[J], l = vj[J];
      Q[I][J] = R[i][k] * R[j][l] + (k != l ? R[i][l] * R[j][k] : 0.0);
    }
  double T[6][6];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      double a = 0.0;
      for (int K = 0; K < 6; ++K) a += Q[I][K] * C6_local[K * 6 + J];
      T[I][J] = a;
    }
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      double a = 0.0;
      for (int K = 0; K < 6; ++K) a += T[I][K] * Q[J][K];
      C6_global[I * 6 + J] = a;
    }
}

}  // namespace elas

namespace elas {

void strain_tensor(const double* e6, double E[9]) {
  E[0] = e6[0]; E[4] = e6[1]; E[8] = e6[2];
  E[5] = E[7] = e6[3];
  E[2] = E[6] = e6[4];
  E[1] = E[3] = e6[5];
}

int grid_prepare(GridHost& g, int nx, int ny, int nz, const int32_t* phase_id, int n_phases, const double* C_local,
                 const double* rodrigues, std::string* err) {
  auto bad = [&](const std::string& m) {
    if (err) *err = m;
    return ELAS_ERR_INVALID_ARG;
  };
  if (nx < 2 || ny < 2 || nz < 2) return bad("every grid dimension must be >= 2");
  if (!phase_id || n_phases < 0 || (n_phases > 0 && !C_local)) return bad("phase_id / C_local missing");
  const long long N = (long long)nx * ny * nz;
  if (N > (1LL << 31) - 1) return bad("more than 2^31-1 voxels");
  g.nx = nx; g.ny = ny; g.nz = nz; g.N = N; g.n_phases = n_phases;
  g.count.assign(std::max(n_phases, 1), 0);
  for (long long e = 0; e < N; ++e) {
    const int p = phase_id[e];
    if (p < -1 || p >= n_phases) {
      char buf[128];
      std::snprintf(buf, sizeof buf, "phase_id[%lld] = %d outside [-1, %d)", e, p, n_phases);
      return bad(buf);
    }
    if (p >= 0) ++g.count[p];
  }
  if (n_phases > 0 && !finite_all(C_local, 36 * (size_t)n_phases)) return bad("C_local has a non-finite entry");
  if (rodrigues && !finite_all(rodrigues, 3 * (size_t)n_phases)) return bad("rodrigues has a non-finite entry");
  for (int p = 0; p < n_phases; ++p) {
    const double* C = C_local + 36 * p;
    double mx = 0.0;
    for (int i = 0; i < 36; ++i) mx = std::max(mx, std::fabs(C[i]));
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j)
        if (std::fabs(C[i * 6 + j] - C[j * 6 + i]) > 1e-12 * mx) {
          char buf[96];
          std::snprintf(buf, sizeof buf, "C_local of phase %d is not symmetric", p);
          return bad(buf);
        }
  }
  const size_t P = (size_t)std::max(n_phases, 1);
  g.cglob.assign(36 * P, 0.0);
  g.coef64.assign(kCoefStride * P, 0.0);
  g.coef32.assign(kCoef32Stride * P, 0.0f);
  g.cfull.assign(kSymStride * P, 0.0);
  const double zero_rho[3] = {0, 0, 0};
  for (int p = 0; p < n_phases; ++p) {
    double* Cg = &g.cglob[36 * p];
    bond_rotate(C_local + 36 * p, rodrigues ? rodrigues + 3 * p : zero_rho, Cg);
    for (int i = 0; i < 6; ++i)  // symmetrise the rotated matrix (round-off only)
      for (int j = i + 1; j < 6; ++j) Cg[i * 6 + j] = Cg[j * 6 + i] = 0.5 * (Cg[i * 6 + j] + Cg[j * 6 + i]);
    bool solid = false;
    for (int i = 0; i < 36; ++i) solid |= (C_local[36 * p + i] != 0.0);
    for (int i = 0; i < 6; ++i)
      for (int j = i; j < 6; ++j) {
        const double v = solid ? Cg[i * 6 + j] : 0.0;
        g.cfull[kSymStride * p + pk(i, j)] = v;
        g.coef64[kCoefStride * p + kCoefMode0 + pk(i, j)] = v / 16.0;
        g.coef64[kCoefStride * p + kCoefMode1 + pk(i, j)] = v / 48.0;
        g.coef64[kCoefStride * p + kCoefMode2 + pk(i, j)] = v / 144.0;
      }
    g.coef64[kCoefStride * p + kCoefFlag] = solid ? 1.0 : 0.0;
    g.coef64[kCoefStride * p + kCoefMode0 + kCoefSolid0] = solid ? 1.0 : 0.0;
    // diagonal blocks of K_e for the Jacobi preconditioner (Eq. 9):
    // (K_e)_aa,ij = C_ikjl M_kl with M = (I + 3 s s^T) / 36, s = (2ax-1, 2ay-1, 2az-1)
    static const int vs[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    static const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
    for (int a = 0; a < 4; ++a) {
      const double sv[3] = {2.0 * (a & 1) - 1.0, 2.0 * ((a >> 1) & 1) - 1.0, -1.0};
      for (int q = 0; q < 6; ++q) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l)
            acc += g.cfull[kSymStride * p + pk(vs[pi[q]][k], vs[pj[q]][l])] * ((k == l ? 1.0 : 0.0) + 3.0 * sv[k] * sv[l]);
        g.coef64[kCoefStride * p + kCoefJac + 6 * a + q] = solid ? acc / 36.0 : 0.0;
      }
    }
    if (!solid)
      for (int i = 0; i < 36; ++i) Cg[i] = 0.0;
  }
  for (size_t p = 0; p < P; ++p) {
    const double* src = &g.coef64[kCoefStride * p];
    float* dst = &g.coef32[kCoef32Stride * p];
    for (int i = 0; i < kCoefStride; ++i) dst[i] = (float)src[i];
    // float-pair copy of the three scaled blocks (entries 0..23 each, the solid flag included)
    const int blk[3] = {kCoefMode0, kCoefMode1, kCoefMode2};
    for (int b = 0; b < 3; ++b)
      for (int i = 0; i < 24; ++i) {
        const double v = src[blk[b] + i];
        const float hi = (float)v;
        dst[kCoefFF + kCoefFFBlock * b + 2 * i] = hi;
        dst[kCoefFF + kCoefFFBlock * b + 2 * i + 1] = (float)(v - (double)hi);
      }
  }
  return ELAS_OK;
}

// Per-phase sigma = C E (tensor components 11,22,33,23,13,12) for the closed-form right-hand side,
// and the no-cancellation scale of b: sum_e sum_a |sigma_e s_a / 4|^2 = 1/2 sum_e |sigma_e|_F^2.
double grid_sigma(const GridHost& g, const double* e6, std::vector<double>& sig) {
  const double ev[6] = {e6[0], e6[1], e6[2], 2 * e6[3], 2 * e6[4], 2 * e6[5]};
  sig.assign(6 * (size_t)std::max(g.n_phases, 1), 0.0);
  double s2 = 0.0;
  for (int p = 0; p < g.n_phases; ++p) {
    for (int r = 0; r < 6; ++r) {
      double a = 0.0;
      for (int q = 0; q < 6; ++q) a += g.cglob[36 * p + 6 * r + q] * ev[q];
      sig[6 * p + r] = a;
    }
    const double* S = &sig[6 * p];
    const double f2 = S[0] * S[0] + S[1] * S[1] + S[2] * S[2] + 2 * (S[3] * S[3] + S[4] * S[4] + S[5] * S[5]);
    s2 += 0.5 * f2 * (double)g.count[p];
  }
  return s2;
}

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, Tiling> g_tuned;
}  // namespace

Tiling choose_tiling(const Geo& geo, int elem_bytes, int sm_count) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_tuple(geo.nx, geo.ny, geo.nz, elem_bytes, sm_count));
    if (it != g_tuned.end()) return it->second;
  }
  return make_tiling(geo, elem_bytes, sm_count);
}

void record_tuned_tiling(const Geo& geo, int elem_bytes, int sm_count, const Tiling& t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[std::make_tuple(geo.nx, geo.ny, geo.nz, elem_bytes, sm_count)] = t;
}

long long max_tiles_bound(long long N) { return N / 48 + 4096; }

int tune_tiling(Engine& e, const Prob& proto, int eb, int sm_count, long long max_tiles, int max_candidates,
                Tiling* best_out, double* best_ms, std::string* err) {
  if (max_candidates <= 0) max_candidates = 12;
  const Geo geo{proto.nx, proto.ny, proto.nz, proto.N};
  const int threads = apply_max_threads(eb);
  // candidates: the cost model's choice plus the best alternatives over tile shapes and z-chunks,
  // ranked by the slots they waste (ragged edge tiles, the one-voxel halo, the z halo, idle SMs)
  std::vector<std::pair<double, Tiling>> cands;
  const Tiling base = make_tiling(geo, eb, sm_count);
  cands.push_back({0.0, base});
  const int kcs[] = {2, 4, 8, 12, 16, 24, 32, 48, 64};
  for (int tx = 4; tx <= 40; ++tx)
    for (int ty = 2; ty <= 24; ++ty) {
      const int nv = (tx + 1) * (ty + 1);
      if (nv > threads || nv < threads * 3 / 4) continue;
      for (int kc : kcs) {
        if (kc > geo.nz) continue;
        Tiling t = make_tiling(geo, eb, sm_count, tx, ty, kc);
        if (t.n_tiles <= 0 || t.n_tiles > max_tiles) continue;
        const double slots = (double)sm_count * apply_resident_blocks(eb, threads, t.smem);
        const double waste = (double)(t.tiles_x * tx) * (t.tiles_y * ty) / ((double)geo.nx * geo.ny) *
                             (double)(t.tiles_z * (kc + 1)) / geo.nz * ((double)threads / (tx * ty)) *
                             std::ceil(t.n_tiles / slots) / (t.n_tiles / slots);
        cands.push_back({waste, t});
      }
    }
  std::sort(cands.begin() + 1, cands.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  if ((int)cands.size() > max_candidates) cands.resize(max_candidates);
  cudaEvent_t e0, e1;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (err) *err = cudaGetErrorString(ce);
    return ELAS_ERR_CUDA;
  }
  double best = 1e300;
  Tiling best_t = base;
  const int kind = eb == 4 ? AK_F32_DOT : AK_F64_DOT;
  int rc = ELAS_OK;
  for (auto& cand : cands) {
    Prob p = proto;
    p.tx = cand.second.tx; p.ty = cand.second.ty; p.kc = cand.second.kc;
    p.tiles_x = cand.second.tiles_x; p.tiles_y = cand.second.tiles_y;
    p.n_tiles = (int)cand.second.n_tiles;
    rc = engine_set_problems(e, {p}, err);
    if (rc != ELAS_OK) break;
    ce = launch_apply(e.bd, kind, POST_NONE, GATE_NONE, e.stream);  // warm-up
    float tot = 0.f;
    for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) {
      cudaEventRecord(e0, e.stream);
      ce = launch_apply(e.bd, kind, POST_NONE, GATE_NONE, e.stream);
      cudaEventRecord(e1, e.stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    if (ce != cudaSuccess) {
      if (err) *err = cudaGetErrorString(ce);
      rc = ELAS_ERR_CUDA;
      break;
    }
    if (tot / 3 < best) {
      best = tot / 3;
      best_t = cand.second;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != ELAS_OK) return rc;
  record_tuned_tiling(geo, eb, sm_count, best_t);
  *best_out = best_t;
  if (best_ms) *best_ms = best;
  return ELAS_OK;
}

}  // namespace elas

// ==========================================================================================
// Context
// ==========================================================================================
struct elas_ctx {
  Geo geo{};
  int n_phases = 0;
  int precision = ELAS_PREC_FP64;
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 0;
  GridHost grid;
  // workspace views
  int32_t* phase = nullptr;
  double* coef64 = nullptr;
  float* coef32 = nullptr;
  double* cfull = nullptr;
  double* sig = nullptr;
  void* minv = nullptr;        // FP64 (plain) or FP32 (mixed) Jacobi inverse planes
  double* w = nullptr;
  float *w_hi = nullptr, *w_lo = nullptr;
  void *g = nullptr, *h = nullptr, *Ah = nullptr, *z = nullptr;
  double *parts = nullptr, *parts64 = nullptr, *parts32 = nullptr, *parts_stress = nullptr;
  long long stride = 0;
  Engine main, aux64, aux32;   // the solve, stand-alone FP64 products, stand-alone FP32 products
  Tiling tl_main{}, tl64{}, tl32{};
  bool has_solution = false;
  std::string err;
};

namespace {

int fail(elas_ctx* c, int code, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_err = msg;
  return code;
}

int cuda_fail(elas_ctx* c, cudaError_t e, const char* what) {
  return fail(c, ELAS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define ELAS_CUDA(ctx, call)                                   \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return cuda_fail((ctx), _e, #call); \
  } while (0)

#define ELAS_TRY(ctx, call)                     \
  do {                                          \
    std::string _m;                             \
    int _r = (call);                            \
    if (_r != ELAS_OK) return fail((ctx), _r, _m.empty() ? std::string(#call) : _m); \
  } while (0)

struct Carve {
  char* base;
  size_t off = 0;
  char* take(size_t bytes) {
    char* p = base ? base + off : nullptr;
    off = align_up(off + bytes);
    return p;
  }
};

// Workspace layout, used both for sizing (base = nullptr) and for assigning the views.
size_t carve(elas_ctx* c, char* base, int nx, int ny, int nz, int n_phases, int precision) {
  const long long N = (long long)nx * ny * nz;
  const bool mixed = precision == ELAS_PREC_MIXED;
  const size_t vb = mixed ? sizeof(float) : sizeof(double);
  const long long stride = std::max(max_tiles_bound(N), chunks_of(N));
  const size_t P = (size_t)std::max(n_phases, 1);
  Carve cv{base};
  char* t_main = cv.take(engine_table_bytes(1, stride, chunks_of(N)));
  char* t_64 = cv.take(engine_table_bytes(1, stride, chunks_of(N)));
  char* t_32 = cv.take(engine_table_bytes(1, stride, chunks_of(N)));
  int32_t* phase = (int32_t*)cv.take(sizeof(int32_t) * N);
  double* coef64 = (double*)cv.take(sizeof(double) * kCoefStride * P);
  float* coef32 = (float*)cv.take(sizeof(float) * kCoef32Stride * P);
  double* cfull = (double*)cv.take(sizeof(double) * kSymStride * P);
  double* sig = (double*)cv.take(sizeof(double) * 6 * P);
  void* minv = cv.take(vb * 6 * N);
  double* w = (double*)cv.take(sizeof(double) * 3 * N);
  float* w_hi = mixed ? (float*)cv.take(sizeof(float) * 3 * N) : nullptr;
  float* w_lo = mixed ? (float*)cv.take(sizeof(float) * 3 * N) : nullptr;
  void* g = cv.take(vb * 3 * N);
  void* h = cv.take(vb * 3 * N);
  void* Ah = cv.take(vb * 3 * N);
  void* z = cv.take(vb * 3 * N);
  double* parts = (double*)cv.take(sizeof(double) * kPartsSlots * stride);
  double* parts64 = (double*)cv.take(sizeof(double) * kPartsSlots * stride);
  double* parts32 = (double*)cv.take(sizeof(double) * kPartsSlots * stride);
  double* parts_stress = (double*)cv.take(sizeof(double) * 6 * kMaxParts);
  if (c) {
    c->phase = phase; c->coef64 = coef64; c->coef32 = coef32; c->cfull = cfull; c->sig = sig; c->minv = minv;
    c->w = w; c->w_hi = w_hi; c->w_lo = w_lo; c->g = g; c->h = h; c->Ah = Ah; c->z = z;
    c->parts = parts; c->parts64 = parts64; c->parts32 = parts32; c->parts_stress = parts_stress;
    c->stride = stride;
    c->main.d_counts = (long long*)t_main;  // engine_init re-carves these regions
    c->aux64.d_counts = (long long*)t_64;
    c->aux32.d_counts = (long long*)t_32;
  }
  return cv.off;
}

Prob make_prob(elas_ctx* c, const Tiling& tl, double* parts) {
  Prob p{};
  p.nx = c->geo.nx; p.ny = c->geo.ny; p.nz = c->geo.nz; p.N = c->geo.N;
  p.tx = tl.tx; p.ty = tl.ty; p.kc = tl.kc; p.tiles_x = tl.tiles_x; p.tiles_y = tl.tiles_y;
  p.n_tiles = (int)tl.n_tiles;
  p.n_chunks = (int)chunks_of(c->geo.N);
  p.parts_stride = (int)c->stride;
  p.phase = c->phase;
  p.coef64 = c->coef64;
  p.coef32 = c->coef32;
  p.sig = c->sig;
  p.minv = c->minv;
  p.w = c->w; p.w_hi = c->w_hi; p.w_lo = c->w_lo;
  p.g = c->g; p.h = c->h; p.Ah = c->Ah; p.z = c->z;
  p.z_bytes = (long long)(c->precision == ELAS_PREC_MIXED ? sizeof(float) : sizeof(double)) * 3 * c->geo.N;
  p.parts = parts;
  return p;
}

// (Re)install the tilings of the three engines.
int install_tilings(elas_ctx* c) {
  std::string m;
  const bool mixed = c->precision == ELAS_PREC_MIXED;
  c->tl_main = mixed ? c->tl32 : c->tl64;
  int r = engine_set_problems(c->main, {make_prob(c, c->tl_main, c->parts)}, &m);
  if (r == ELAS_OK) r = engine_set_problems(c->aux64, {make_prob(c, c->tl64, c->parts64)}, &m);
  if (r == ELAS_OK) r = engine_set_problems(c->aux32, {make_prob(c, c->tl32, c->parts32)}, &m);
  if (r != ELAS_OK) return fail(c, r, m);
  return ELAS_OK;
}

int set_aux_strain(elas_ctx* c, Engine& e, const double* e6) {
  std::vector<SolveSetup> su(1);
  strain_tensor(e6, su[0].E);
  ELAS_CUDA(c, cudaMemcpyAsync(e.d_setups, su.data(), sizeof(SolveSetup), cudaMemcpyHostToDevice, c->stream));
  ELAS_CUDA(c, launch_state_init(e.bd, e.d_setups, nullptr, 1, c->stream));
  return ELAS_OK;
}

// Point one stand-alone engine's problem at caller buffers (uploads only when they changed).
int point_aux(elas_ctx* c, Engine& e, const void* h, void* Ah, const double* w, double* g) {
  Prob& p = e.probs[0];
  if (p.h == h && p.Ah == Ah && p.w == w && p.g == g) return ELAS_OK;
  p.h = const_cast<void*>(h);
  p.Ah = Ah;
  p.w = const_cast<double*>(w);
  p.g = g;
  std::string m;
  int r = engine_upload_probs(e, &m);
  if (r != ELAS_OK) return fail(c, r, m);
  return ELAS_OK;
}

int upload_sigma(elas_ctx* c, const double* e6, double* bscale2) {
  std::vector<double> sig;
  *bscale2 = grid_sigma(c->grid, e6, sig);
  ELAS_CUDA(c, cudaMemcpyAsync(c->sig, sig.data(), sizeof(double) * sig.size(), cudaMemcpyHostToDevice, c->stream));
  return ELAS_OK;
}

}  // namespace

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

int elas_isotropic_stiffness(double E, double nu, double* C6) {
  if (!C6 || !std::isfinite(E) || !std::isfinite(nu) || !(nu > -1.0 && nu < 0.5)) return ELAS_ERR_INVALID_ARG;
  const double mu = E / (2.0 * (1.0 + nu));
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  for (int i = 0; i < 36; ++i) C6[i] = 0.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) C6[i * 6 + j] = lam;
    C6[i * 6 + i] = lam + 2.0 * mu;
    C6[(i + 3) * 6 + (i + 3)] = mu;
  }
  return ELAS_OK;
}

int elas_cubic_stiffness(double c11, double c12, double c44, double* C6) {
  if (!C6 || !std::isfinite(c11) || !std::isfinite(c12) || !std::isfinite(c44)) return ELAS_ERR_INVALID_ARG;
  for (int i = 0; i < 36; ++i) C6[i] = 0.0;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) C6[i * 6 + j] = c12;
    C6[i * 6 + i] = c11;
    C6[(i + 3) * 6 + (i + 3)] = c44;
  }
  return ELAS_OK;
}

int elas_rotated_stiffness(const double* C6_local, const double* rho, double* C6_global) {
  if (!C6_local || !rho || !C6_global || !finite_all(C6_local, 36) || !finite_all(rho, 3)) return ELAS_ERR_INVALID_ARG;
  bond_rotate(C6_local, rho, C6_global);
  return ELAS_OK;
}

int elas_workspace_bytes(int nx, int ny, int nz, int n_phases, int precision, size_t* bytes) {
  if (!bytes || nx < 2 || ny < 2 || nz < 2 || n_phases < 0 ||
      (precision != ELAS_PREC_FP64 && precision != ELAS_PREC_MIXED))
    return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_workspace_bytes: dims must be >= 2 and precision valid");
  *bytes = carve(nullptr, nullptr, nx, ny, nz, n_phases, precision);
  return ELAS_OK;
}

const char* elas_last_error(const elas_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int elas_create(elas_ctx** out, int nx, int ny, int nz, const int32_t* phase_id, int n_phases, const double* C_local,
                const double* rodrigues, int precision, void* workspace, size_t ws_bytes, void* cuda_stream) {
  if (!out) return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: out is NULL");
  *out = nullptr;
  if (precision != ELAS_PREC_FP64 && precision != ELAS_PREC_MIXED)
    return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: unknown precision");
  if (nx < 2 || ny < 2 || nz < 2)
    return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: every grid dimension must be >= 2");
  GridHost grid;
  std::string m;
  int r = grid_prepare(grid, nx, ny, nz, phase_id, n_phases, C_local, rodrigues, &m);
  if (r != ELAS_OK) return fail(nullptr, r, "elas_create: " + m);
  const size_t need = carve(nullptr, nullptr, nx, ny, nz, n_phases, precision);
  if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || ws_bytes < need) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "elas_create: workspace needs %zu bytes, 256-byte aligned (got %zu at %p)", need,
                  ws_bytes, workspace);
    return fail(nullptr, ELAS_ERR_WORKSPACE, buf);
  }
  elas_ctx* c = new elas_ctx();
  c->geo = Geo{nx, ny, nz, grid.N};
  c->n_phases = n_phases;
  c->precision = precision;
  c->stream = (cudaStream_t)cuda_stream;
  c->grid = std::move(grid);
  auto bail = [&](int code) {
    g_create_err = c->err;
    engine_destroy(c->main);
    engine_destroy(c->aux64);
    engine_destroy(c->aux32);
    delete c;
    return code;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "elas_create: device query"));
  carve(c, (char*)workspace, nx, ny, nz, n_phases, precision);
  const bool mixed = precision == ELAS_PREC_MIXED;
  const long long nch = chunks_of(c->geo.N);
  char* t_main = (char*)c->main.d_counts;
  char* t_64 = (char*)c->aux64.d_counts;
  char* t_32 = (char*)c->aux32.d_counts;
  r = engine_init(c->main, mixed, c->sm_count, apply_max_threads(mixed ? 4 : 8), 1, c->stride, nch, t_main, c->stream, &m);
  if (r == ELAS_OK) r = engine_init(c->aux64, false, c->sm_count, apply_max_threads(8), 1, c->stride, nch, t_64, c->stream, &m);
  if (r == ELAS_OK) r = engine_init(c->aux32, true, c->sm_count, apply_max_threads(4), 1, c->stride, nch, t_32, c->stream, &m);
  if (r != ELAS_OK) return bail(fail(c, r, "elas_create: " + m));
  c->tl64 = choose_tiling(c->geo, 8, c->sm_count);
  c->tl32 = choose_tiling(c->geo, 4, c->sm_count);
  if (c->tl64.n_tiles <= 0 || c->tl32.n_tiles <= 0 || c->tl64.n_tiles > c->stride || c->tl32.n_tiles > c->stride)
    return bail(fail(c, ELAS_ERR_INVALID_ARG, "elas_create: no operator tiling fits this grid"));
  cudaStream_t s = c->stream;
  const GridHost& G = c->grid;
  e = cudaMemcpyAsync(c->phase, phase_id, sizeof(int32_t) * G.N, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->coef64, G.coef64.data(), sizeof(double) * G.coef64.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->coef32, G.coef32.data(), sizeof(float) * G.coef32.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->cfull, G.cfull.data(), sizeof(double) * G.cfull.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "elas_create: upload"));
  if (install_tilings(c) != ELAS_OK) return bail(ELAS_ERR_CUDA);
  *out = c;
  return ELAS_OK;
}

void elas_destroy(elas_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  engine_destroy(ctx->main);
  engine_destroy(ctx->aux64);
  engine_destroy(ctx->aux32);
  delete ctx;
}

int elas_apply(elas_ctx* c, const double* u, double* y) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (!u || !y || (const void*)u == (const void*)y) return fail(c, ELAS_ERR_INVALID_ARG, "elas_apply: bad u / y");
  int r = point_aux(c, c->aux64, u, y, nullptr, nullptr);
  if (r != ELAS_OK) return r;
  // the in-solve kernel variant (u.Au partials), without a scalar update
  ELAS_CUDA(c, launch_apply(c->aux64.bd, AK_F64_DOT, POST_NONE, GATE_NONE, c->stream));
  return ELAS_OK;
}

int elas_apply_f32(elas_ctx* c, const float* u, float* y) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (!u || !y || (const void*)u == (const void*)y) return fail(c, ELAS_ERR_INVALID_ARG, "elas_apply_f32: bad u / y");
  int r = point_aux(c, c->aux32, u, y, nullptr, nullptr);
  if (r != ELAS_OK) return r;
  ELAS_CUDA(c, launch_apply(c->aux32.bd, AK_F32_DOT, POST_NONE, GATE_NONE, c->stream));
  return ELAS_OK;
}

int elas_rhs(elas_ctx* c, const double* strain, double* b) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (!strain || !b || !finite_all(strain, 6)) return fail(c, ELAS_ERR_INVALID_ARG, "elas_rhs: bad strain / b");
  double bs;
  int r = upload_sigma(c, strain, &bs);
  if (r != ELAS_OK) return r;
  ELAS_CUDA(c, launch_rhs(c->geo, c->phase, c->sig, b, c->sm_count, c->stream));
  return ELAS_OK;
}

int elas_residual(elas_ctx* c, const double* strain, const double* w, double* g, double* rnorm) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (!strain || !w || !g || !finite_all(strain, 6)) return fail(c, ELAS_ERR_INVALID_ARG, "elas_residual: bad args");
  int r = set_aux_strain(c, c->aux64, strain);
  if (r == ELAS_OK) r = point_aux(c, c->aux64, nullptr, nullptr, w, g);
  if (r != ELAS_OK) return r;
  ELAS_CUDA(c, launch_apply(c->aux64.bd, AK_F64_AFFINE, POST_NONE, GATE_NONE, c->stream));
  if (rnorm) {
    ELAS_CUDA(c, launch_apply(c->aux64.bd, AK_F64_NORM, POST_TRUE_NORM, GATE_NONE, c->stream));
    ELAS_CUDA(c, cudaMemcpyAsync(c->aux64.h_states, c->aux64.d_states, sizeof(DevState), cudaMemcpyDeviceToHost,
                                 c->stream));
    ELAS_CUDA(c, cudaStreamSynchronize(c->stream));
    *rnorm = std::sqrt(c->aux64.h_states[0].rr_true);
  }
  return ELAS_OK;
}

int elas_jacobi(elas_ctx* c, double* Minv) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (!Minv) return fail(c, ELAS_ERR_INVALID_ARG, "elas_jacobi: Minv is NULL");
  // the FP64 inverse is built straight into the caller's buffer (a mixed context keeps only FP32)
  ELAS_CUDA(c, launch_jacobi(c->geo, c->phase, c->coef64, Minv, nullptr, c->sm_count, c->stream));
  return ELAS_OK;
}

int elas_pcg_solve(elas_ctx* c, const double* strain, double tol, int max_iter, const elas_solve_opts* opts,
                   double* w_out, elas_solve_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (!strain || !finite_all(strain, 6) || !(tol >= 0.0) || max_iter < 0)
    return fail(c, ELAS_ERR_INVALID_ARG, "elas_pcg_solve: bad strain / tol / max_iter");
  const bool mixed = c->precision == ELAS_PREC_MIXED;
  int stop_rule = mixed ? ELAS_STOP_TRUE : ELAS_STOP_PRECOND;
  int replace_every = mixed ? 50 : 0;
  int check_every = 0;
  double drop2 = 0.0;
  int precond = ELAS_PRECOND_BLOCK;
  if (opts) {
    if (opts->precond < ELAS_PRECOND_BLOCK || opts->precond > ELAS_PRECOND_NONE)
      return fail(c, ELAS_ERR_INVALID_ARG, "elas_pcg_solve: unknown precond");
    precond = opts->precond;
    if (opts->stop_rule == ELAS_STOP_PRECOND || opts->stop_rule == ELAS_STOP_TRUE) stop_rule = opts->stop_rule;
    if (opts->replace_every > 0) replace_every = opts->replace_every;
    if (opts->check_every > 0) check_every = opts->check_every;
    if (opts->replace_drop > 0) drop2 = std::pow(10.0, -2.0 * opts->replace_drop);
  }
  int K = check_every;
  if (K <= 0) {
    if (mixed)
      K = replace_every > 0 ? std::min(replace_every, 50) : 50;
    else
      K = (int)std::max<long long>(4, std::min<long long>(64, 20000000LL / std::max<long long>(c->geo.N, 1)));
  }
  cudaStream_t s = c->stream;
  double bscale2 = 0.0;
  int r = upload_sigma(c, strain, &bscale2);
  if (r != ELAS_OK) return r;
  std::vector<SolveSetup> su(1);
  su[0].tol = tol;
  su[0].tol2_true = tol * tol;
  su[0].bscale2 = bscale2;
  strain_tensor(strain, su[0].E);
  su[0].max_iter = max_iter;
  su[0].stop_rule = stop_rule;
  su[0].replace_every = mixed ? replace_every : 0;
  su[0].drop2 = mixed ? drop2 : 0.0;
  // Algorithm 2 part 1: point-block Jacobi inverse (Eq. 9), FP64, stored in the path's precision
  // (or the scalar / identity preconditioner of the comparison solvers)
  ELAS_CUDA(c, launch_jacobi(c->geo, c->phase, c->coef64, mixed ? nullptr : (double*)c->minv,
                             mixed ? (float*)c->minv : nullptr, c->sm_count, s, precond));
  int launches = 0;
  std::string m;
  r = engine_solve(c->main, su, K, &launches, &m);
  if (r != ELAS_OK) return fail(c, r, "elas_pcg_solve: " + m);
  launches += 1;
  if (w_out) ELAS_CUDA(c, cudaMemcpyAsync(w_out, c->w, sizeof(double) * 3 * c->geo.N, cudaMemcpyDeviceToDevice, s));
  const DevState& hs = c->main.h_states[0];
  c->has_solution = true;
  int status = hs.done ? hs.status : ELAS_MAX_ITER;
  if (status == ST_RUNNING) status = ELAS_MAX_ITER;
  if (info) {
    info->iters = hs.iter;
    info->status = status;
    info->relres_precond = hs.gg0 > 0 ? std::sqrt(std::max(hs.gg, 0.0) / hs.gg0) : 0.0;
    info->relres_true = hs.bb > 0 ? std::sqrt(hs.rr_true / hs.bb) : std::sqrt(hs.rr_true);
    info->n_replacements = hs.n_repl;
    info->launches = launches;
    if (w_out) ELAS_CUDA(c, cudaStreamSynchronize(s));
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status == ELAS_NONFINITE) return fail(c, ELAS_ERR_NONFINITE, "elas_pcg_solve: non-finite value in the iteration");
  return ELAS_OK;
}

int elas_stress(elas_ctx* c, const double* strain, const double* w, double* stress, double* von_mises,
                double* macro_stress) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (!strain || !finite_all(strain, 6)) return fail(c, ELAS_ERR_INVALID_ARG, "elas_stress: bad strain");
  if (!w) {
    if (!c->has_solution) return fail(c, ELAS_ERR_STATE, "elas_stress: no solve has run on this context");
    w = c->w;
  }
  DevState* st = c->aux64.d_states;
  ELAS_CUDA(c, launch_stress(c->geo, c->phase, c->cfull, strain, w, stress, von_mises, c->parts_stress, &st->ctr[3],
                             st->macro, c->sm_count, c->stream));
  if (macro_stress) {
    ELAS_CUDA(c, cudaMemcpyAsync(c->aux64.h_states, st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    ELAS_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < 6; ++q) macro_stress[q] = c->aux64.h_states[0].macro[q];
  }
  return ELAS_OK;
}

int elas_hotspot(elas_ctx* c, const double* von_mises, double s_kernel, int neighbours, double* smoothed,
                 double* sigma_max, long long* voxel) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (!von_mises || !smoothed || !sigma_max)
    return fail(c, ELAS_ERR_INVALID_ARG, "elas_hotspot: von_mises, smoothed and sigma_max are required");
  if (!(s_kernel > 0.0) || !std::isfinite(s_kernel))
    return fail(c, ELAS_ERR_INVALID_ARG, "elas_hotspot: the kernel width must be positive");
  if (neighbours != ELAS_HOTSPOT_ALL && neighbours != ELAS_HOTSPOT_SOLID)
    return fail(c, ELAS_ERR_INVALID_ARG, "elas_hotspot: neighbours must be ELAS_HOTSPOT_ALL or ELAS_HOTSPOT_SOLID");
  unsigned long long* best2 = reinterpret_cast<unsigned long long*>(c->parts_stress);
  ELAS_CUDA(c, launch_hotspot(c->geo, c->phase, von_mises, s_kernel, neighbours == ELAS_HOTSPOT_SOLID, smoothed, best2,
                              c->sm_count, c->stream));
  unsigned long long h[2] = {0, 0};
  ELAS_CUDA(c, cudaMemcpyAsync(h, best2, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  ELAS_CUDA(c, cudaStreamSynchronize(c->stream));
  const bool none = h[1] == ~0ull;
  double v = 0.0;
  std::memcpy(&v, &h[0], sizeof v);
  *sigma_max = none ? 0.0 : v;
  if (voxel) *voxel = none ? -1 : (long long)h[1];
  return ELAS_OK;
}

int elas_set_fp64_operator(elas_ctx* c, int form) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  if (form != ELAS_FP64_OP_PAIRED && form != ELAS_FP64_OP_NATIVE)
    return fail(c, ELAS_ERR_INVALID_ARG, "elas_set_fp64_operator: form must be ELAS_FP64_OP_PAIRED or _NATIVE");
  const bool on = form == ELAS_FP64_OP_PAIRED;
  engine_set_ff64(c->main, on);
  engine_set_ff64(c->aux64, on);
  return ELAS_OK;
}

int elas_tuning_export(char* buf, size_t cap, size_t* len) {
  std::string out;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    char line[128];
    for (const auto& kv : g_tuned) {
      const auto& k = kv.first;
      std::snprintf(line, sizeof line, "%d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
                    std::get<3>(k), std::get<4>(k), kv.second.tx, kv.second.ty, kv.second.kc);
      out += line;
    }
  }
  if (len) *len = out.size();
  if (buf && cap > 0) {
    const size_t n = std::min(cap - 1, out.size());
    std::memcpy(buf, out.data(), n);
    buf[n] = '\0';
  }
  return ELAS_OK;
}

int elas_tuning_import(const char* text) {
  if (!text) return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_tuning_import: text is NULL");
  std::vector<std::pair<std::tuple<int, int, int, int, int>, Tiling>> rows;
  const char* p = text;
  int line_no = 0;
  while (*p) {
    const char* e = std::strchr(p, '\n');
    std::string line(p, e ? (size_t)(e - p) : std::strlen(p));
    p = e ? e + 1 : p + line.size();
    ++line_no;
    if (line.find_first_not_of(" \t\r") == std::string::npos) continue;
    int v[8];
    char extra = 0;
    if (std::sscanf(line.c_str(), "%d %d %d %d %d %d %d %d %c", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &v[7],
                    &extra) != 8 ||
        v[0] < 2 || v[1] < 2 || v[2] < 2 || (v[3] != 4 && v[3] != 8) || v[4] < 1 || v[5] < 1 || v[6] < 1 || v[7] < 1) {
      char m[96];
      std::snprintf(m, sizeof m, "elas_tuning_import: line %d is not 'nx ny nz elem_bytes sm_count tx ty kc'", line_no);
      return fail(nullptr, ELAS_ERR_INVALID_ARG, m);
    }
    const Geo geo{v[0], v[1], v[2], (long long)v[0] * v[1] * v[2]};
    const Tiling t = make_tiling(geo, v[3], v[4], v[5], v[6], v[7]);
    if (t.n_tiles <= 0 || t.tx != v[5] || t.ty != v[6] || t.kc != v[7]) {
      char m[96];
      std::snprintf(m, sizeof m, "elas_tuning_import: line %d is not a valid tiling for its grid", line_no);
      return fail(nullptr, ELAS_ERR_INVALID_ARG, m);
    }
    rows.push_back({std::make_tuple(v[0], v[1], v[2], v[3], v[4]), t});
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& r : rows) g_tuned[r.first] = r.second;
  return ELAS_OK;
}

int elas_autotune(elas_ctx* c, int max_candidates, double* best_ms) {
  if (!c) return ELAS_ERR_INVALID_ARG;
  const bool mixed = c->precision == ELAS_PREC_MIXED;
  const int eb = mixed ? 4 : 8;
  Prob proto = make_prob(c, mixed ? c->tl32 : c->tl64, mixed ? c->parts32 : c->parts64);
  const size_t vb = mixed ? sizeof(float) : sizeof(double);
  ELAS_CUDA(c, cudaMemsetAsync(c->h, 0, vb * 3 * c->geo.N, c->stream));
  Tiling best_t{};
  double best = 0.0;
  std::string m;
  int r = tune_tiling(mixed ? c->aux32 : c->aux64, proto, eb, c->sm_count, c->stride, max_candidates, &best_t, &best, &m);
  if (r != ELAS_OK) return fail(c, r, "elas_autotune: " + m);
  if (mixed)
    c->tl32 = best_t;
  else
    c->tl64 = best_t;
  // stand-alone engines point at the caller's last buffers again on their next call
  r = install_tilings(c);
  if (r != ELAS_OK) return r;
  if (best_ms) *best_ms = best;
  return ELAS_OK;
}

}  // extern "C"
