// elas_stress_noalloc: the voxel stress / von Mises / macro-stress step for callers that must not
// allocate memory.
//
// Some callers cannot call cudaMalloc (or any routine that allocates) at the point where they
// need this result: code that runs while a CUDA graph is being captured, real-time loops whose
// memory is fixed at start-up, plug-ins living inside a host framework that owns every device
// allocation, or a serving process whose memory budget is already fully handed out.  elas_create
// does not suit them, because a context allocates a pinned status buffer and a private stream.
// This entry point needs no context: the caller passes its own device inputs and outputs, and the
// only other device memory is a fixed scratch array compiled into the library.
//
// The scratch array is file-scope device memory: every GPU that loads the library holds its
// 1 MiB until the process exits, and every call on that GPU shares it.  It keeps what the last
// call left there; the parts that must start at zero (the arrival counter of the block reduction
// and the bad-id counter) are cleared by every call.  Calls whose work overlaps on the GPU (from
// two streams or two host threads) race on the array, so callers must order them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "elas_internal.h"

namespace {

using namespace elas;

constexpr size_t kScratchBytes = size_t(1) << 20;  // 1 MiB per device
constexpr int kMaxDevices = 64;

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffC = 0;  // ELAS_NOALLOC_MAX_PHASES x 21 doubles (packed symmetric stiffness)
constexpr size_t kOffParts = al256(kOffC + sizeof(double) * kSymStride * ELAS_NOALLOC_MAX_PHASES);
constexpr size_t kOffCtr = al256(kOffParts + sizeof(double) * 6 * kMaxParts);
constexpr size_t kOffBad = kOffCtr + 256;
constexpr size_t kOffMacro = kOffBad + 256;
constexpr size_t kScratchUsed = kOffMacro + sizeof(double) * 6;
static_assert(kScratchUsed <= kScratchBytes, "scratch layout exceeds the static array");

// Host code may not dereference this name: on the host it is only a stand-in for the symbol.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
char* g_scratch[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};

// Counts phase ids outside [-1, n_phases): ids live on the device, so they are checked there
// before any kernel indexes the stiffness table with them.
__global__ void k_count_bad_ids(const int32_t* __restrict__ phase, long long N, int n_phases, unsigned int* bad) {
  unsigned int local = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const int p = phase[e];
    local += (p < -1 || p >= n_phases) ? 1u : 0u;
  }
  if (local) atomicAdd(bad, local);
}

// Set-up, once per device with that device current: resolve the array's device address.
int scratch_for(int dev, char** base, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return ELAS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return ELAS_ERR_CUDA;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return ELAS_ERR_CUDA;
    g_scratch[dev] = static_cast<char*>(p);
    g_sms[dev] = n;
  }
  *base = g_scratch[dev];
  *sms = g_sms[dev];
  return ELAS_OK;
}

bool finite_n(const double* p, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

}  // namespace

extern "C" int elas_stress_noalloc(int nx, int ny, int nz, const int32_t* phase_id, int n_phases,
                                   const double* C_local, const double* rodrigues, const double* strain,
                                   const double* w, double* stress, double* von_mises, double* macro_stress,
                                   void* cuda_stream) {
  if (nx < 2 || ny < 2 || nz < 2 || !phase_id || !w || !strain || n_phases < 0 ||
      n_phases > ELAS_NOALLOC_MAX_PHASES || (n_phases > 0 && !C_local))
    return ELAS_ERR_INVALID_ARG;
  const long long N = (long long)nx * ny * nz;
  if (N > (1LL << 31) - 1 || !finite_n(strain, 6)) return ELAS_ERR_INVALID_ARG;
  if (n_phases > 0 && !finite_n(C_local, 36 * n_phases)) return ELAS_ERR_INVALID_ARG;
  if (rodrigues && !finite_n(rodrigues, 3 * n_phases)) return ELAS_ERR_INVALID_ARG;
  // the call synchronises its stream and copies from a stack buffer, neither of which a stream
  // under capture can take: refuse it before any work is enqueued
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return ELAS_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ELAS_ERR_CUDA;
  char* base = nullptr;
  int sms = 0;
  int rc = scratch_for(dev, &base, &sms);
  if (rc != ELAS_OK) return rc;

  // Per-phase sample-frame stiffness (Eq. 4), rotated and packed on the host exactly as
  // elas_create does, staged through a fixed stack buffer (no heap use) into the scratch table.
  constexpr int kChunk = 32;
  double pack[kChunk * kSymStride];
  const double zero_rho[3] = {0, 0, 0};
  for (int p0 = 0; p0 < n_phases; p0 += kChunk) {
    const int np = n_phases - p0 < kChunk ? n_phases - p0 : kChunk;
    for (int q = 0; q < np; ++q) {
      const int p = p0 + q;
      const double* Cl = C_local + 36 * p;
      double mx = 0.0;
      bool solid = false;
      for (int i = 0; i < 36; ++i) {
        mx = std::fmax(mx, std::fabs(Cl[i]));
        solid |= (Cl[i] != 0.0);
      }
      for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j)
          if (std::fabs(Cl[i * 6 + j] - Cl[j * 6 + i]) > 1e-12 * mx) return ELAS_ERR_INVALID_ARG;
      double Cg[36];
      bond_rotate(Cl, rodrigues ? rodrigues + 3 * p : zero_rho, Cg);
      for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) Cg[i * 6 + j] = Cg[j * 6 + i] = 0.5 * (Cg[i * 6 + j] + Cg[j * 6 + i]);
      for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) pack[q * kSymStride + pk(i, j)] = solid ? Cg[i * 6 + j] : 0.0;
    }
    if (cudaMemcpyAsync(base + kOffC + sizeof(double) * kSymStride * p0, pack, sizeof(double) * kSymStride * np,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return ELAS_ERR_CUDA;
  }
  unsigned int* ctr = reinterpret_cast<unsigned int*>(base + kOffCtr);
  unsigned int* bad = reinterpret_cast<unsigned int*>(base + kOffBad);
  if (cudaMemsetAsync(base + kOffCtr, 0, 512, s) != cudaSuccess) return ELAS_ERR_CUDA;  // counter + bad count

  long long blocks = (N + 255) / 256;
  if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
  k_count_bad_ids<<<(int)blocks, 256, 0, s>>>(phase_id, N, n_phases, bad);
  if (cudaGetLastError() != cudaSuccess) return ELAS_ERR_CUDA;
  unsigned int n_bad = 0;
  if (cudaMemcpyAsync(&n_bad, bad, sizeof n_bad, cudaMemcpyDeviceToHost, s) != cudaSuccess) return ELAS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ELAS_ERR_CUDA;
  if (n_bad != 0) return ELAS_ERR_INVALID_ARG;

  Geo g{nx, ny, nz, N};
  double* macro_dev = reinterpret_cast<double*>(base + kOffMacro);
  if (launch_stress(g, phase_id, reinterpret_cast<const double*>(base + kOffC), strain, w, stress, von_mises,
                    reinterpret_cast<double*>(base + kOffParts), ctr, macro_dev, sms, s) != cudaSuccess)
    return ELAS_ERR_CUDA;
  if (macro_stress) {
    if (cudaMemcpyAsync(macro_stress, macro_dev, sizeof(double) * 6, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return ELAS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ELAS_ERR_CUDA;
  }
  return ELAS_OK;
}
