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
#include <string>
#include <vector>

#include "elas_internal.h"

using namespace elas;

struct elas_ctx {
  Geo geo{};
  int n_phases = 0;
  int precision = ELAS_PREC_FP64;
  cudaStream_t stream = nullptr;     // caller's stream: all work is ordered on it
  cudaStream_t cap_stream = nullptr; // private stream used only to record graphs
  int device = 0, sm_count = 0;
  // workspace views
  DevState* st = nullptr;      // solve state
  DevState* st_aux = nullptr;  // state of stand-alone products (strain for residual, stress sums)
  double* parts = nullptr;
  int32_t* phase = nullptr;
  double* coef64 = nullptr;
  float* coef32 = nullptr;
  double* cfull = nullptr;
  double* sig = nullptr;
  double* minv64 = nullptr;
  float* minv32 = nullptr;
  double* w = nullptr;
  float *w_hi = nullptr, *w_lo = nullptr;  // mixed path
  void *g = nullptr, *h = nullptr, *Ah = nullptr, *z = nullptr;
  // host copies
  std::vector<double> cglob;            // n_phases x 36, sample-frame stiffness
  std::vector<long long> phase_count;   // voxels per phase
  Tiling tl64{}, tl32{};
  int vec_blocks = 0, vec_threads = 256;
  bool has_solution = false;
  double last_strain[6] = {0, 0, 0, 0, 0, 0};
  // recorded iteration batches
  cudaGraphExec_t batch_exec = nullptr;
  int batch_k = 0;
  DevState* host_state = nullptr;  // pinned mirror for status reads
  std::string err;
};

namespace {

thread_local std::string g_create_err;

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

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Workspace carving, used both for sizing (base = nullptr) and for assigning the views.
size_t carve(elas_ctx* c, char* base, long long N, int n_phases, int precision) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off = align_up(off + bytes);
    return p;
  };
  const size_t vb = precision == ELAS_PREC_MIXED ? sizeof(float) : sizeof(double);
  DevState* st = (DevState*)take(sizeof(DevState));
  DevState* st_aux = (DevState*)take(sizeof(DevState));
  double* parts = (double*)take(sizeof(double) * kMaxParts * kPartSlots);
  int32_t* phase = (int32_t*)take(sizeof(int32_t) * N);
  double* coef64 = (double*)take(sizeof(double) * kCoefStride * std::max(n_phases, 1));
  float* coef32 = (float*)take(sizeof(float) * kCoefStride * std::max(n_phases, 1));
  double* cfull = (double*)take(sizeof(double) * kSymStride * std::max(n_phases, 1));
  double* sig = (double*)take(sizeof(double) * 6 * std::max(n_phases, 1));
  double* minv64 = precision == ELAS_PREC_FP64 ? (double*)take(sizeof(double) * 6 * N) : nullptr;
  float* minv32 = precision == ELAS_PREC_MIXED ? (float*)take(sizeof(float) * 6 * N) : nullptr;
  double* w = (double*)take(sizeof(double) * 3 * N);
  float* w_hi = precision == ELAS_PREC_MIXED ? (float*)take(sizeof(float) * 3 * N) : nullptr;
  float* w_lo = precision == ELAS_PREC_MIXED ? (float*)take(sizeof(float) * 3 * N) : nullptr;
  void* g = take(vb * 3 * N);
  void* h = take(vb * 3 * N);
  void* Ah = take(vb * 3 * N);
  void* z = take(vb * 3 * N);
  if (c) {
    c->st = st; c->st_aux = st_aux; c->parts = parts; c->phase = phase;
    c->coef64 = coef64; c->coef32 = coef32; c->cfull = cfull; c->sig = sig;
    c->minv64 = minv64; c->minv32 = minv32; c->w = w; c->g = g; c->h = h; c->Ah = Ah; c->z = z;
    c->w_hi = w_hi; c->w_lo = w_lo;
  }
  return off;
}

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

void strain_tensor(const double* e6, double E[9]) {
  E[0] = e6[0]; E[4] = e6[1]; E[8] = e6[2];
  E[5] = E[7] = e6[3];
  E[2] = E[6] = e6[4];
  E[1] = E[3] = e6[5];
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

namespace {

ApplyLaunch base_apply(elas_ctx* c, bool f32) {
  ApplyLaunch a{};
  a.geo = c->geo;
  a.tl = f32 ? c->tl32 : c->tl64;
  a.phase = c->phase;
  a.coef = f32 ? (const void*)c->coef32 : (const void*)c->coef64;
  a.parts = c->parts;
  a.st = c->st;
  a.post = POST_NONE;
  a.gate = GATE_NONE;
  return a;
}

VecLaunch base_vec(elas_ctx* c) {
  VecLaunch v{};
  v.geo = c->geo;
  v.blocks = c->vec_blocks;
  v.threads = c->vec_threads;
  v.phase = c->phase;
  v.sig = c->sig;
  v.w = c->w;
  v.w_hi = c->w_hi;
  v.w_lo = c->w_lo;
  v.g = c->g; v.h = c->h; v.Ah = c->Ah; v.z = c->z;
  v.minv = c->precision == ELAS_PREC_MIXED ? (const void*)c->minv32 : (const void*)c->minv64;
  v.parts = c->parts;
  v.st = c->st;
  return v;
}

// Per-phase sigma = C E (tensor components 11,22,33,23,13,12) for the closed-form right-hand side,
// and the no-cancellation scale of b: sum_e sum_a |sigma_e s_a / 4|^2 = 1/2 sum_e |sigma_e|_F^2.
int upload_sigma(elas_ctx* c, const double* e6, double* bscale2) {
  const double ev[6] = {e6[0], e6[1], e6[2], 2 * e6[3], 2 * e6[4], 2 * e6[5]};
  std::vector<double> sig(6 * (size_t)std::max(c->n_phases, 1), 0.0);
  double s2 = 0.0;
  for (int p = 0; p < c->n_phases; ++p) {
    for (int r = 0; r < 6; ++r) {
      double a = 0.0;
      for (int q = 0; q < 6; ++q) a += c->cglob[36 * p + 6 * r + q] * ev[q];
      sig[6 * p + r] = a;
    }
    const double* S = &sig[6 * p];
    const double f2 = S[0] * S[0] + S[1] * S[1] + S[2] * S[2] + 2 * (S[3] * S[3] + S[4] * S[4] + S[5] * S[5]);
    s2 += 0.5 * f2 * (double)c->phase_count[p];
  }
  *bscale2 = s2;
  ELAS_CUDA(c, cudaMemcpyAsync(c->sig, sig.data(), sizeof(double) * sig.size(), cudaMemcpyHostToDevice, c->stream));
  return ELAS_OK;
}

int set_aux_strain(elas_ctx* c, const double* e6) {
  SolveSetup s{};
  strain_tensor(e6, s.E);
  ELAS_CUDA(c, launch_state_init(c->st_aux, s, c->stream));
  return ELAS_OK;
}

// Record one batch of K PCG iterations (Algorithm 2 steps A-E, K times) as a CUDA graph; the
// last iteration carries the FP64 residual check/replacement between steps D and E.
int record_batch(elas_ctx* c, int K) {
  if (c->batch_exec && c->batch_k == K) return ELAS_OK;
  if (c->batch_exec) {
    cudaGraphExecDestroy(c->batch_exec);
    c->batch_exec = nullptr;
  }
  const bool mixed = c->precision == ELAS_PREC_MIXED;
  cudaStream_t s = c->cap_stream;
  ELAS_CUDA(c, cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  cudaError_t e = cudaSuccess;
  VecLaunch v = base_vec(c);
  for (int it = 0; it < K && e == cudaSuccess; ++it) {
    ApplyLaunch a = base_apply(c, mixed);
    a.u = c->h;
    a.y = c->Ah;
    a.post = POST_LAMBDA;
    a.gate = GATE_RUNNING;
    e = mixed ? launch_apply_f32(a, EPI_STORE_DOT, s) : launch_apply_f64(a, EPI_STORE_DOT, false, s);
    if (e == cudaSuccess) e = launch_pcg_update(v, mixed, s);
    if (e == cudaSuccess && it == K - 1 && mixed) e = launch_w_combine(v, true, s);
    if (e == cudaSuccess && it == K - 1) {
      ApplyLaunch r = base_apply(c, false);
      r.u = c->w;
      r.g_out = c->g;
      r.z_out = c->z;
      r.minv = mixed ? (const void*)c->minv32 : (const void*)c->minv64;
      r.post = POST_REPLACE;
      r.gate = GATE_REPLACE;
      e = mixed ? launch_residual_mixed(r, s) : launch_apply_f64(r, EPI_RESIDUAL, true, s);
    }
    if (e == cudaSuccess) e = launch_pcg_direction(v, mixed, s);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(c, e, "recording the PCG batch");
  }
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
  cudaError_t e3 = cudaGraphInstantiate(&c->batch_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return cuda_fail(c, e3, "cudaGraphInstantiate");
  c->batch_k = K;
  return ELAS_OK;
}

int validate_ctx(elas_ctx* c) {
  if (!c) return ELAS_ERR_INVALID_ARG;
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
  *bytes = carve(nullptr, nullptr, (long long)nx * ny * nz, n_phases, precision);
  return ELAS_OK;
}

const char* elas_last_error(const elas_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int elas_create(elas_ctx** out, int nx, int ny, int nz, const int32_t* phase_id, int n_phases, const double* C_local,
                const double* rodrigues, int precision, void* workspace, size_t ws_bytes, void* cuda_stream) {
  if (!out) return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: out is NULL");
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 2)
    return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: every grid dimension must be >= 2");
  if (precision != ELAS_PREC_FP64 && precision != ELAS_PREC_MIXED)
    return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: unknown precision");
  if (!phase_id || n_phases < 0 || (n_phases > 0 && !C_local))
    return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: phase_id / C_local missing");
  const long long N = (long long)nx * ny * nz;
  if (N > (1LL << 31) - 1) return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: more than 2^31-1 voxels");
  size_t need = carve(nullptr, nullptr, N, n_phases, precision);
  if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || ws_bytes < need) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "elas_create: workspace needs %zu bytes, 256-byte aligned (got %zu at %p)", need,
                  ws_bytes, workspace);
    return fail(nullptr, ELAS_ERR_WORKSPACE, buf);
  }
  std::vector<long long> count(std::max(n_phases, 1), 0);
  for (long long e = 0; e < N; ++e) {
    const int p = phase_id[e];
    if (p < -1 || p >= n_phases) {
      char buf[128];
      std::snprintf(buf, sizeof buf, "elas_create: phase_id[%lld] = %d outside [-1, %d)", e, p, n_phases);
      return fail(nullptr, ELAS_ERR_INVALID_ARG, buf);
    }
    if (p >= 0) ++count[p];
  }
  if (n_phases > 0 && !finite_all(C_local, 36 * (size_t)n_phases))
    return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: C_local has a non-finite entry");
  if (rodrigues && !finite_all(rodrigues, 3 * (size_t)n_phases))
    return fail(nullptr, ELAS_ERR_INVALID_ARG, "elas_create: rodrigues has a non-finite entry");
  for (int p = 0; p < n_phases; ++p) {
    const double* C = C_local + 36 * p;
    double mx = 0.0;
    for (int i = 0; i < 36; ++i) mx = std::max(mx, std::fabs(C[i]));
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j)
        if (std::fabs(C[i * 6 + j] - C[j * 6 + i]) > 1e-12 * mx) {
          char buf[96];
          std::snprintf(buf, sizeof buf, "elas_create: C_local of phase %d is not symmetric", p);
          return fail(nullptr, ELAS_ERR_INVALID_ARG, buf);
        }
  }

  elas_ctx* c = new elas_ctx();
  c->geo = Geo{nx, ny, nz, N};
  c->n_phases = n_phases;
  c->precision = precision;
  c->stream = (cudaStream_t)cuda_stream;
  c->phase_count = count;
  auto bail = [&](int code) {
    g_create_err = c->err;
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->host_state) cudaFreeHost(c->host_state);
    delete c;
    return code;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->host_state, sizeof(DevState));
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "elas_create: device setup"));
  carve(c, (char*)workspace, N, n_phases, precision);

  // per-phase tables (FP64 on the host): sample-frame C, scaled modal blocks, solid flags
  c->cglob.assign(36 * (size_t)std::max(n_phases, 1), 0.0);
  std::vector<double> coef64(kCoefStride * (size_t)std::max(n_phases, 1), 0.0);
  std::vector<float> coef32(coef64.size(), 0.0f);
  std::vector<double> cfull(kSymStride * (size_t)std::max(n_phases, 1), 0.0);
  const double zero_rho[3] = {0, 0, 0};
  for (int p = 0; p < n_phases; ++p) {
    double* Cg = &c->cglob[36 * p];
    bond_rotate(C_local + 36 * p, rodrigues ? rodrigues + 3 * p : zero_rho, Cg);
    for (int i = 0; i < 6; ++i)  // symmetrise the rotated matrix (round-off only)
      for (int j = i + 1; j < 6; ++j) Cg[i * 6 + j] = Cg[j * 6 + i] = 0.5 * (Cg[i * 6 + j] + Cg[j * 6 + i]);
    bool solid = false;
    for (int i = 0; i < 36; ++i) solid |= (C_local[36 * p + i] != 0.0);
    for (int i = 0; i < 6; ++i)
      for (int j = i; j < 6; ++j) {
        const double v = solid ? Cg[i * 6 + j] : 0.0;
        cfull[kSymStride * p + pk(i, j)] = v;
        coef64[kCoefStride * p + kCoefMode0 + pk(i, j)] = v / 16.0;
        coef64[kCoefStride * p + kCoefMode1 + pk(i, j)] = v / 48.0;
        coef64[kCoefStride * p + kCoefMode2 + pk(i, j)] = v / 144.0;
      }
    coef64[kCoefStride * p + kCoefFlag] = solid ? 1.0 : 0.0;
    if (!solid)
      for (int i = 0; i < 36; ++i) Cg[i] = 0.0;
  }
  for (size_t i = 0; i < coef64.size(); ++i) coef32[i] = (float)coef64[i];

  cudaStream_t s = c->stream;
  e = cudaMemsetAsync(c->st, 0, sizeof(DevState), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->st_aux, 0, sizeof(DevState), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->phase, phase_id, sizeof(int32_t) * N, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->coef64, coef64.data(), sizeof(double) * coef64.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->coef32, coef32.data(), sizeof(float) * coef32.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->cfull, cfull.data(), sizeof(double) * cfull.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "elas_create: upload"));

  c->tl64 = make_tiling(c->geo, sizeof(double), c->sm_count);
  c->tl32 = make_tiling(c->geo, sizeof(float), c->sm_count);
  long long vb = (N + c->vec_threads - 1) / c->vec_threads;
  c->vec_blocks = (int)std::min<long long>(vb, (long long)c->sm_count * 8);
  if (c->tl64.blocks <= 0 || c->tl32.blocks <= 0) return bail(fail(c, ELAS_ERR_INVALID_ARG, "elas_create: no tiling"));

  *out = c;
  return ELAS_OK;
}

void elas_destroy(elas_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->host_state) cudaFreeHost(ctx->host_state);
  delete ctx;
}

int elas_apply(elas_ctx* c, const double* u, double* y) {
  if (validate_ctx(c) != ELAS_OK) return ELAS_ERR_INVALID_ARG;
  if (!u || !y || (const void*)u == (const void*)y) return fail(c, ELAS_ERR_INVALID_ARG, "elas_apply: bad u / y");
  ApplyLaunch a = base_apply(c, false);
  a.st = c->st_aux;  // the in-solve kernel variant (u.Au partials), without a scalar update
  a.u = u;
  a.y = y;
  ELAS_CUDA(c, launch_apply_f64(a, EPI_STORE_DOT, false, c->stream));
  return ELAS_OK;
}

int elas_apply_f32(elas_ctx* c, const float* u, float* y) {
  if (validate_ctx(c) != ELAS_OK) return ELAS_ERR_INVALID_ARG;
  if (!u || !y || (const void*)u == (const void*)y) return fail(c, ELAS_ERR_INVALID_ARG, "elas_apply_f32: bad u / y");
  ApplyLaunch a = base_apply(c, true);
  a.st = c->st_aux;
  a.u = u;
  a.y = y;
  ELAS_CUDA(c, launch_apply_f32(a, EPI_STORE_DOT, c->stream));
  return ELAS_OK;
}

int elas_rhs(elas_ctx* c, const double* strain, double* b) {
  if (validate_ctx(c) != ELAS_OK) return ELAS_ERR_INVALID_ARG;
  if (!strain || !b || !finite_all(strain, 6)) return fail(c, ELAS_ERR_INVALID_ARG, "elas_rhs: bad strain / b");
  double bs;
  int r = upload_sigma(c, strain, &bs);
  if (r != ELAS_OK) return r;
  ELAS_CUDA(c, launch_rhs(c->geo, c->phase, c->sig, b, c->sm_count, c->stream));
  return ELAS_OK;
}

int elas_residual(elas_ctx* c, const double* strain, const double* w, double* g, double* rnorm) {
  if (validate_ctx(c) != ELAS_OK) return ELAS_ERR_INVALID_ARG;
  if (!strain || !w || !g || !finite_all(strain, 6)) return fail(c, ELAS_ERR_INVALID_ARG, "elas_residual: bad args");
  int r = set_aux_strain(c, strain);
  if (r != ELAS_OK) return r;
  ApplyLaunch a = base_apply(c, false);
  a.st = c->st_aux;
  a.u = w;
  a.y = g;
  ELAS_CUDA(c, launch_apply_f64(a, EPI_STORE, true, c->stream));
  if (rnorm) {
    a.post = POST_TRUE_NORM;
    ELAS_CUDA(c, launch_apply_f64(a, EPI_NORM, true, c->stream));
    ELAS_CUDA(c, cudaMemcpyAsync(c->host_state, c->st_aux, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    ELAS_CUDA(c, cudaStreamSynchronize(c->stream));
    *rnorm = std::sqrt(c->host_state->rr_true);
  }
  return ELAS_OK;
}

int elas_jacobi(elas_ctx* c, double* Minv) {
  if (validate_ctx(c) != ELAS_OK) return ELAS_ERR_INVALID_ARG;
  if (!Minv) return fail(c, ELAS_ERR_INVALID_ARG, "elas_jacobi: Minv is NULL");
  // the FP64 inverse is built straight into the caller's buffer (a mixed context keeps only FP32)
  ELAS_CUDA(c, launch_jacobi(c->geo, c->phase, c->cfull, Minv, nullptr, c->sm_count, c->stream));
  return ELAS_OK;
}

int elas_pcg_solve(elas_ctx* c, const double* strain, double tol, int max_iter, const elas_solve_opts* opts,
                   double* w_out, elas_solve_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (validate_ctx(c) != ELAS_OK) return ELAS_ERR_INVALID_ARG;
  if (!strain || !finite_all(strain, 6) || !(tol >= 0.0) || max_iter < 0)
    return fail(c, ELAS_ERR_INVALID_ARG, "elas_pcg_solve: bad strain / tol / max_iter");
  const bool mixed = c->precision == ELAS_PREC_MIXED;
  int stop_rule = mixed ? ELAS_STOP_TRUE : ELAS_STOP_PRECOND;
  int replace_every = mixed ? 50 : 0;
  int check_every = 0;
  if (opts) {
    if (opts->stop_rule == ELAS_STOP_PRECOND || opts->stop_rule == ELAS_STOP_TRUE) stop_rule = opts->stop_rule;
    if (opts->replace_every > 0) replace_every = opts->replace_every;
    if (opts->check_every > 0) check_every = opts->check_every;
  }
  int K = check_every;
  if (K <= 0) {
    if (mixed)
      K = replace_every > 0 ? replace_every : 50;
    else
      K = (int)std::max<long long>(4, std::min<long long>(64, 20000000LL / std::max<long long>(c->geo.N, 1)));
  }
  cudaStream_t s = c->stream;
  double bscale2 = 0.0;
  int r = upload_sigma(c, strain, &bscale2);
  if (r != ELAS_OK) return r;
  SolveSetup su{};
  su.tol = tol;
  su.tol2_true = tol * tol;
  su.bscale2 = bscale2;
  strain_tensor(strain, su.E);
  su.max_iter = max_iter;
  su.stop_rule = stop_rule;
  su.replace_every = mixed ? replace_every : 0;
  int launches = 0;
  // Algorithm 2 part 1: point-block Jacobi inverse (Eq. 9) in FP64, FP32 copy for the mixed path
  ELAS_CUDA(c, launch_jacobi(c->geo, c->phase, c->cfull, c->minv64, c->minv32, c->sm_count, s));
  ELAS_CUDA(c, launch_state_init(c->st, su, s));
  VecLaunch v = base_vec(c);
  ELAS_CUDA(c, launch_pcg_init(v, mixed, s));
  launches += 3;
  r = record_batch(c, K);
  if (r != ELAS_OK) return r;
  for (;;) {
    ELAS_CUDA(c, cudaMemcpyAsync(c->host_state, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    ELAS_CUDA(c, cudaStreamSynchronize(s));
    if (c->host_state->done) break;
    if (max_iter == 0) break;
    ELAS_CUDA(c, cudaGraphLaunch(c->batch_exec, s));
    launches += 3 * K + 1 + (mixed ? 1 : 0);
  }
  if (mixed) {
    ELAS_CUDA(c, launch_w_combine(v, false, s));
    launches += 1;
  }
  // final FP64 true residual of the returned w
  ApplyLaunch a = base_apply(c, false);
  a.u = c->w;
  a.post = POST_TRUE_NORM;
  ELAS_CUDA(c, launch_apply_f64(a, EPI_NORM, true, s));
  launches += 1;
  if (w_out) ELAS_CUDA(c, cudaMemcpyAsync(w_out, c->w, sizeof(double) * 3 * c->geo.N, cudaMemcpyDeviceToDevice, s));
  ELAS_CUDA(c, cudaMemcpyAsync(c->host_state, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  ELAS_CUDA(c, cudaStreamSynchronize(s));
  const DevState& hs = *c->host_state;
  c->has_solution = true;
  std::memcpy(c->last_strain, strain, sizeof(double) * 6);
  int status = hs.done ? hs.status : (hs.iter >= max_iter ? ELAS_MAX_ITER : hs.status);
  if (status == ST_RUNNING) status = ELAS_MAX_ITER;
  if (info) {
    info->iters = hs.iter;
    info->status = status;
    info->relres_precond = hs.gg0 > 0 ? std::sqrt(std::max(hs.gg, 0.0) / hs.gg0) : 0.0;
    info->relres_true = hs.bb > 0 ? std::sqrt(hs.rr_true / hs.bb) : std::sqrt(hs.rr_true);
    info->n_replacements = hs.n_repl;
    info->launches = launches;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (status == ELAS_NONFINITE) return fail(c, ELAS_ERR_NONFINITE, "elas_pcg_solve: non-finite value in the iteration");
  return ELAS_OK;
}

int elas_stress(elas_ctx* c, const double* strain, const double* w, double* stress, double* von_mises,
                double* macro_stress) {
  if (validate_ctx(c) != ELAS_OK) return ELAS_ERR_INVALID_ARG;
  if (!strain || !finite_all(strain, 6)) return fail(c, ELAS_ERR_INVALID_ARG, "elas_stress: bad strain");
  if (!w) {
    if (!c->has_solution) return fail(c, ELAS_ERR_STATE, "elas_stress: no solve has run on this context");
    w = c->w;
  }
  ELAS_CUDA(c, launch_stress(c->geo, c->phase, c->cfull, strain, w, stress, von_mises, c->parts, &c->st_aux->ctr[3],
                             c->st_aux->macro, c->sm_count, c->stream));
  if (macro_stress) {
    ELAS_CUDA(c, cudaMemcpyAsync(c->host_state, c->st_aux, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    ELAS_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int r = 0; r < 6; ++r) macro_stress[r] = c->host_state->macro[r];
  }
  return ELAS_OK;
}

}  // extern "C"
