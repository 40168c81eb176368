// Maximum-stress extraction (ELAS3D-Xtal, arXiv 2602.07354, App. C): the von Mises field is
// smoothed by a normalised (masked) Gaussian convolution, smooth = G * (vm M) / G * M with M the
// solid indicator, on the periodic cell; the hotspots are the solid voxels that no competing
// 26-neighbour exceeds (every neighbour, or the solid ones only), and the stress concentration
// uses the largest of them.  The sums run over dz, dy, dx
// with the weight (w[dz] * w[dy]) * w[dx], every operation explicitly rounded, so the field is
// bitwise the same as a plain loop in that order; the maximum (and the lowest voxel id holding it)
// are formed with order-independent atomics.
#include <cuda_runtime.h>

#include "elas_internal.h"

namespace elas {

namespace {

constexpr int kHotThreads = 256;

struct Weights {
  double w[2 * kHotMaxRadius + 1];
};

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__global__ void k_smooth(int nx, int ny, int nz, const int32_t* __restrict__ phase, const double* __restrict__ vm,
                         Weights W, int r, double* __restrict__ smooth) {
  const long long N = (long long)nx * ny * nz;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((long long)nx * ny));
    double num = 0.0, den = 0.0;
    for (int dz = -r; dz <= r; ++dz) {
      const long long kz = wrap1(k + dz, nz);
      for (int dy = -r; dy <= r; ++dy) {
        const long long jy = wrap1(j + dy, ny);
        const double wzy = __dmul_rn(W.w[dz + r], W.w[dy + r]);
        for (int dx = -r; dx <= r; ++dx) {
          const long long u = wrap1(i + dx, nx) + nx * (jy + ny * kz);
          const double wt = __dmul_rn(wzy, W.w[dx + r]);
          if (phase[u] >= 0) {
            num = __dadd_rn(num, __dmul_rn(wt, vm[u]));
            den = __dadd_rn(den, wt);
          }
        }
      }
    }
    smooth[v] = den > 0.0 ? __ddiv_rn(num, den) : 0.0;
  }
}

// pass 0: the largest hotspot value (bits of a non-negative double order like the values);
// pass 1: the lowest voxel id holding it
__global__ void k_hotspot(int nx, int ny, int nz, const int32_t* __restrict__ phase, const double* __restrict__ smooth,
                          bool solid_only, int pass, unsigned long long* __restrict__ best) {
  const long long N = (long long)nx * ny * nz;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
    if (phase[v] < 0) continue;
    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((long long)nx * ny));
    const double s = smooth[v];
    bool is_max = true;
    for (int dz = -1; dz <= 1 && is_max; ++dz)
      for (int dy = -1; dy <= 1 && is_max; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const long long u = wrap1(i + dx, nx) + nx * (wrap1(j + dy, ny) + (long long)ny * wrap1(k + dz, nz));
          if (smooth[u] > s && !(solid_only && phase[u] < 0)) {
            is_max = false;
            break;
          }
        }
    if (!is_max) continue;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(s);
    if (pass == 0)
      atomicMax(&best[0], bits);
    else if (bits == best[0])
      atomicMin(&best[1], (unsigned long long)v);
  }
}

}  // namespace

cudaError_t launch_hotspot(const Geo& g, const int32_t* phase, const double* vm, double s_kernel, bool solid_only,
                           double* smooth, unsigned long long* best2, int sm_count, cudaStream_t s) {
  const int r = hot_radius(s_kernel);
  Weights W{};
  hot_weights(s_kernel, r, W.w);
  const long long blocks = std::min<long long>((g.N + kHotThreads - 1) / kHotThreads, (long long)sm_count * 16);
  k_smooth<<<(int)blocks, kHotThreads, 0, s>>>(g.nx, g.ny, g.nz, phase, vm, W, r, smooth);
  cudaError_t e = cudaGetLastError();
  const unsigned long long init[2] = {0ull, ~0ull};
  if (e == cudaSuccess) e = cudaMemcpyAsync(best2, init, sizeof init, cudaMemcpyHostToDevice, s);
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    k_hotspot<<<(int)blocks, kHotThreads, 0, s>>>(g.nx, g.ny, g.nz, phase, smooth, solid_only, pass, best2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // init lives on this stack frame
  return e;
}

}  // namespace elas
