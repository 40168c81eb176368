// Microstructure generator on the device (ELAS3D-Xtal, arXiv 2602.07354, Sec. 2.2): grain
// assignment by the weighted ellipsoidal distance of Algorithm 4 and the pore overwrite of
// Algorithm 5 (with rotated ellipsoids as well as spheres), on a periodic cell.
//
// Grain assignment: the seeds are binned on the host into a uniform grid of cells (about one seed
// per cell, like the coarse cell grid of the paper's seeding stage).  One thread per voxel scans
// the 5 x 5 x 5 cells around its own and keeps the lowest (D^2, grain index); seeds outside that
// block lie at least the distance from the voxel to the block's faces away, so when the best D^2
// is below (that distance / largest semi-axis)^2 the result is exact, and otherwise the thread
// scans every seed.  D^2 is evaluated with explicitly rounded FP64 operations in the order
// (dx*dx + dy*dy) / (rt*rt) + (dz*dz) / (rl*rl), with the periodic minimum-image differences, and
// ties go to the lowest grain index: every voxel gets exactly the grain of a brute-force scan.
//
// Pore overwrite: one block per pore scans the pore's bounding box (periodically wrapped) and
// writes -1 into every voxel whose centre satisfies (q0/a0)^2 + (q1/a1)^2 + (q2/a2)^2 <= 1 with
// q = R^T d; the writes are idempotent, so the order of pores and threads does not matter.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "elas_internal.h"

namespace elas {

namespace {

thread_local std::string g_gen_err;

constexpr int kGenWin = 2;         // cells scanned on each side of a voxel's own cell
constexpr int kGenMaxCells = 128;  // per dimension
constexpr int kGenThreads = 256;
constexpr int kPoreDoubles = 15;

int gen_fail(int code, const std::string& m) {
  g_gen_err = m;
  return code;
}

struct GenGrid {
  int g[3];        // cells per dimension
  double cs[3];    // cell size per dimension
  double inv_rmax2;  // 1 / (largest semi-axis)^2
};

GenGrid gen_grid(int nx, int ny, int nz, int n) {
  GenGrid G{};
  const double L[3] = {(double)nx, (double)ny, (double)nz};
  const double target = std::cbrt(L[0] * L[1] * L[2] / std::max(n, 1));  // ~1 seed per cell
  for (int d = 0; d < 3; ++d) {
    G.g[d] = (int)std::lround(L[d] / target);
    G.g[d] = std::max(1, std::min(kGenMaxCells, G.g[d]));
    G.cs[d] = L[d] / G.g[d];
  }
  return G;
}

struct GenLayout {
  size_t seeds, semi, start, items, pores, counter, total;
};

GenLayout gen_layout(const GenGrid& G, int n_grains, int n_pores) {
  GenLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = (o + b + 255) / 256 * 256;
    return at;
  };
  const size_t cells = (size_t)G.g[0] * G.g[1] * G.g[2];
  L.seeds = take(sizeof(double) * 3 * std::max(n_grains, 1));
  L.semi = take(sizeof(double) * 2 * std::max(n_grains, 1));
  L.start = take(sizeof(int) * (cells + 1));
  L.items = take(sizeof(int) * std::max(n_grains, 1));
  L.pores = take(sizeof(double) * kPoreDoubles * std::max(n_pores, 1));
  L.counter = take(sizeof(unsigned long long) * 2);
  L.total = o;
  return L;
}

__device__ __forceinline__ double min_image(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

// Algorithm 4's weighted ellipsoidal distance, rounded operation by operation.  Without weights
// (rt = rl = 1) the two divisions by 1 are exact and are left out.
template <bool WEIGHTED>
__device__ __forceinline__ double wdist2(const double (&x)[3], const double* __restrict__ s,
                                         const double* __restrict__ semi, int l, const double (&L)[3]) {
  const double dx = min_image(x[0] - s[0], L[0]);
  const double dy = min_image(x[1] - s[1], L[1]);
  const double dz = min_image(x[2] - s[2], L[2]);
  if (!WEIGHTED) return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double rt = semi[2 * l], rl = semi[2 * l + 1];
  return __dadd_rn(__ddiv_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(rt, rt)),
                   __ddiv_rn(__dmul_rn(dz, dz), __dmul_rn(rl, rl)));
}

__device__ __forceinline__ void consider(double D2, int l, double& best, int& arg) {
  if (D2 < best || (D2 == best && l < arg)) {
    best = D2;
    arg = l;
  }
}

template <bool WEIGHTED>
__global__ void k_assign(int nx, int ny, int nz, const double* __restrict__ seeds, const double* __restrict__ semi,
                         int n, const int* __restrict__ start, const int* __restrict__ items, GenGrid G,
                         int32_t* __restrict__ phase, unsigned long long* __restrict__ fallbacks) {
  const long long N = (long long)nx * ny * nz;
  const double L[3] = {(double)nx, (double)ny, (double)nz};
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((long long)nx * ny));
    const double x[3] = {i + 0.5, j + 0.5, k + 0.5};
    int c[3], lo[3], cnt[3];
    bool all[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      c[d] = min(G.g[d] - 1, max(0, (int)floor(x[d] / G.cs[d])));
      all[d] = G.g[d] <= 2 * kGenWin + 1;
      lo[d] = all[d] ? 0 : c[d] - kGenWin;
      cnt[d] = all[d] ? G.g[d] : 2 * kGenWin + 1;
    }
    double best = INFINITY;
    int arg = 0x7fffffff;
    for (int oz = 0; oz < cnt[2]; ++oz) {
      int cz = lo[2] + oz;
      cz += cz < 0 ? G.g[2] : (cz >= G.g[2] ? -G.g[2] : 0);
      for (int oy = 0; oy < cnt[1]; ++oy) {
        int cy = lo[1] + oy;
        cy += cy < 0 ? G.g[1] : (cy >= G.g[1] ? -G.g[1] : 0);
        for (int ox = 0; ox < cnt[0]; ++ox) {
          int cx = lo[0] + ox;
          cx += cx < 0 ? G.g[0] : (cx >= G.g[0] ? -G.g[0] : 0);
          const int cell = cx + G.g[0] * (cy + G.g[1] * cz);
          for (int t = start[cell]; t < start[cell + 1]; ++t) {
            const int l = items[t];
            consider(wdist2<WEIGHTED>(x, seeds + 3 * l, semi, l, L), l, best, arg);
          }
        }
      }
    }
    // every seed outside the scanned block is at least lb away (Euclidean) in some dimension
    double lb = INFINITY;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (!all[d]) lb = fmin(lb, fmin(x[d] - (c[d] - kGenWin) * G.cs[d], (c[d] + kGenWin + 1) * G.cs[d] - x[d]));
    if (!(best < 0.999999 * lb * lb * G.inv_rmax2)) {
      atomicAdd(fallbacks, 1ull);
      for (int l = 0; l < n; ++l)
        consider(wdist2<WEIGHTED>(x, seeds + 3 * l, semi, l, L), l, best, arg);
    }
    phase[v] = arg;
  }
}

__global__ void k_stamp(int nx, int ny, int nz, const double* __restrict__ pores, int32_t* __restrict__ phase) {
  const double* P = pores + (size_t)kPoreDoubles * blockIdx.x;
  const int n[3] = {nx, ny, nz};
  const double L[3] = {(double)nx, (double)ny, (double)nz};
  const double amax = fmax(P[3], fmax(P[4], P[5]));
  const int ext = (int)ceil(amax) + 1;
  int lo[3], cnt[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    cnt[d] = 2 * ext + 1;
    lo[d] = (int)floor(P[d]) - ext;
    if (cnt[d] >= n[d]) {
      cnt[d] = n[d];
      lo[d] = 0;
    }
  }
  const long long total = (long long)cnt[0] * cnt[1] * cnt[2];
  for (long long t = threadIdx.x; t < total; t += blockDim.x) {
    int idx[3] = {(int)(t % cnt[0]), (int)((t / cnt[0]) % cnt[1]), (int)(t / ((long long)cnt[0] * cnt[1]))};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int a = lo[d] + idx[d];
      a %= n[d];
      if (a < 0) a += n[d];
      idx[d] = a;
    }
    const double d0 = min_image(idx[0] + 0.5 - P[0], L[0]);
    const double d1 = min_image(idx[1] + 0.5 - P[1], L[1]);
    const double d2 = min_image(idx[2] + 0.5 - P[2], L[2]);
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double q = __dadd_rn(__dadd_rn(__dmul_rn(P[6 + m], d0), __dmul_rn(P[9 + m], d1)), __dmul_rn(P[12 + m], d2));
      const double u = __ddiv_rn(q, P[3 + m]);
      s = __dadd_rn(s, __dmul_rn(u, u));
    }
    if (s <= 1.0) phase[idx[0] + (long long)nx * (idx[1] + (long long)ny * idx[2])] = -1;
  }
}

__global__ void k_count_pores(const int32_t* __restrict__ phase, long long N, unsigned long long* __restrict__ count) {
  unsigned long long c = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x)
    c += phase[v] < 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

bool finite_all(const double* p, size_t n) {
  for (size_t t = 0; t < n; ++t)
    if (!std::isfinite(p[t])) return false;
  return true;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

}  // namespace

int gen_error(int code, const std::string& m) { return gen_fail(code, m); }
}  // namespace elas

using namespace elas;

extern "C" {

const char* elas_generate_last_error(void) { return g_gen_err.c_str(); }

int elas_generate_workspace_bytes(int nx, int ny, int nz, int n_grains, int n_pores, size_t* bytes) {
  if (!bytes || nx < 1 || ny < 1 || nz < 1 || n_grains < 0 || n_pores < 0)
    return gen_fail(ELAS_ERR_INVALID_ARG, "elas_generate_workspace_bytes: bad arguments");
  *bytes = gen_layout(gen_grid(nx, ny, nz, n_grains), n_grains, n_pores).total;
  return ELAS_OK;
}

int elas_assign_grains(int nx, int ny, int nz, const double* seeds, const double* semi_axes, int n_grains,
                       int32_t* phase, void* workspace, size_t ws_bytes, void* cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1 || n_grains < 1 || !seeds || !phase)
    return gen_fail(ELAS_ERR_INVALID_ARG, "elas_assign_grains: bad dimensions, grain count or pointer");
  if ((long long)nx * ny * nz > (1LL << 31) - 1) return gen_fail(ELAS_ERR_INVALID_ARG, "elas_assign_grains: grid too large");
  const double L[3] = {(double)nx, (double)ny, (double)nz};
  for (int l = 0; l < n_grains; ++l)
    for (int d = 0; d < 3; ++d)
      if (!(seeds[3 * l + d] >= 0.0 && seeds[3 * l + d] < L[d]))
        return gen_fail(ELAS_ERR_INVALID_ARG, "elas_assign_grains: a seed lies outside [0, n) in some dimension");
  double rmax = 1.0;
  if (semi_axes) {
    rmax = 0.0;
    for (int t = 0; t < 2 * n_grains; ++t) {
      if (!(semi_axes[t] > 0.0) || !std::isfinite(semi_axes[t]))
        return gen_fail(ELAS_ERR_INVALID_ARG, "elas_assign_grains: semi-axes must be positive and finite");
      rmax = std::max(rmax, semi_axes[t]);
    }
  }
  GenGrid G = gen_grid(nx, ny, nz, n_grains);
  G.inv_rmax2 = 1.0 / (rmax * rmax);
  const GenLayout Ly = gen_layout(G, n_grains, 0);
  if (!workspace || ((uintptr_t)workspace % 256) != 0 || ws_bytes < Ly.total)
    return gen_fail(ELAS_ERR_WORKSPACE, "elas_assign_grains: workspace too small or not 256-byte aligned");
  // bin the seeds (counting sort by cell, grain order kept within a cell)
  const int cells = G.g[0] * G.g[1] * G.g[2];
  std::vector<int> start(cells + 1, 0), items(n_grains), cell_of(n_grains);
  for (int l = 0; l < n_grains; ++l) {
    int c[3];
    for (int d = 0; d < 3; ++d) c[d] = std::min(G.g[d] - 1, std::max(0, (int)std::floor(seeds[3 * l + d] / G.cs[d])));
    cell_of[l] = c[0] + G.g[0] * (c[1] + G.g[1] * c[2]);
    ++start[cell_of[l] + 1];
  }
  for (int c = 0; c < cells; ++c) start[c + 1] += start[c];
  std::vector<int> fill(start.begin(), start.end() - 1);
  for (int l = 0; l < n_grains; ++l) items[fill[cell_of[l]]++] = l;
  char* base = (char*)workspace;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemcpyAsync(base + Ly.seeds, seeds, sizeof(double) * 3 * n_grains, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && semi_axes)
    e = cudaMemcpyAsync(base + Ly.semi, semi_axes, sizeof(double) * 2 * n_grains, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + Ly.start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + Ly.items, items.data(), sizeof(int) * items.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + Ly.counter, 0, sizeof(unsigned long long) * 2, s);
  if (e != cudaSuccess) return gen_fail(ELAS_ERR_CUDA, std::string("elas_assign_grains: ") + cudaGetErrorString(e));
  const long long N = (long long)nx * ny * nz;
  const int sms = std::max(sm_count(), 1);
  const long long blocks = std::min<long long>((N + kGenThreads - 1) / kGenThreads, (long long)sms * 32);
  auto kern = semi_axes ? k_assign<true> : k_assign<false>;
  kern<<<(int)blocks, kGenThreads, 0, s>>>(nx, ny, nz, (const double*)(base + Ly.seeds),
                                           semi_axes ? (const double*)(base + Ly.semi) : nullptr, n_grains,
                                           (const int*)(base + Ly.start), (const int*)(base + Ly.items), G, phase,
                                           (unsigned long long*)(base + Ly.counter));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables above go out of scope
  if (e != cudaSuccess) return gen_fail(ELAS_ERR_CUDA, std::string("elas_assign_grains: ") + cudaGetErrorString(e));
  return ELAS_OK;
}

int elas_stamp_pores(int nx, int ny, int nz, const double* pores, int n_pores, int32_t* phase,
                     long long* n_pore_voxels, void* workspace, size_t ws_bytes, void* cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1 || n_pores < 0 || (n_pores > 0 && !pores) || !phase)
    return gen_fail(ELAS_ERR_INVALID_ARG, "elas_stamp_pores: bad dimensions, pore count or pointer");
  if ((long long)nx * ny * nz > (1LL << 31) - 1) return gen_fail(ELAS_ERR_INVALID_ARG, "elas_stamp_pores: grid too large");
  const double L[3] = {(double)nx, (double)ny, (double)nz};
  if (n_pores > 0 && !finite_all(pores, (size_t)kPoreDoubles * n_pores))
    return gen_fail(ELAS_ERR_INVALID_ARG, "elas_stamp_pores: non-finite pore parameter");
  for (int p = 0; p < n_pores; ++p) {
    const double* P = pores + kPoreDoubles * p;
    for (int d = 0; d < 3; ++d) {
      if (!(P[d] >= 0.0 && P[d] < L[d]))
        return gen_fail(ELAS_ERR_INVALID_ARG, "elas_stamp_pores: a pore centre lies outside the grid");
      // the minimum image sees a pore whole only when it is shorter than half the cell
      if (!(P[3 + d] > 0.0) || !(P[3 + d] < 0.5 * std::min(L[0], std::min(L[1], L[2]))))
        return gen_fail(ELAS_ERR_INVALID_ARG, "elas_stamp_pores: semi-axes must be positive and below half the cell");
    }
  }
  const GenLayout Ly = gen_layout(gen_grid(nx, ny, nz, 1), 0, n_pores);
  if (!workspace || ((uintptr_t)workspace % 256) != 0 || ws_bytes < Ly.total)
    return gen_fail(ELAS_ERR_WORKSPACE, "elas_stamp_pores: workspace too small or not 256-byte aligned");
  char* base = (char*)workspace;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSuccess;
  if (n_pores > 0)
    e = cudaMemcpyAsync(base + Ly.pores, pores, sizeof(double) * kPoreDoubles * n_pores, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + Ly.counter, 0, sizeof(unsigned long long) * 2, s);
  if (e == cudaSuccess && n_pores > 0) {
    k_stamp<<<n_pores, kGenThreads, 0, s>>>(nx, ny, nz, (const double*)(base + Ly.pores), phase);
    e = cudaGetLastError();
  }
  const long long N = (long long)nx * ny * nz;
  if (e == cudaSuccess) {
    const int sms = std::max(sm_count(), 1);
    const long long blocks = std::min<long long>((N + kGenThreads - 1) / kGenThreads, (long long)sms * 8);
    k_count_pores<<<(int)blocks, kGenThreads, 0, s>>>(phase, N, (unsigned long long*)(base + Ly.counter));
    e = cudaGetLastError();
  }
  unsigned long long cnt = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, base + Ly.counter, sizeof cnt, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return gen_fail(ELAS_ERR_CUDA, std::string("elas_stamp_pores: ") + cudaGetErrorString(e));
  if (n_pore_voxels) *n_pore_voxels = (long long)cnt;
  return ELAS_OK;
}

}  // extern "C"
