// Issue-rate probe of the arithmetic pipes the operator kernels use (not part of libelas): eight
// independent dependency chains per thread of FADD, packed FADD2 (add.rn.f32x2), FFMA, packed FFMA2,
// DFMA, and the double -> float -> double conversion chain of the double-float split, over
// 8 blocks x 256 threads per SM.  Prints one JSON line per operation with its lane-operation rate;
// the roofline peaks of the benchmark (128 FP32 lanes per SM per clock; the FP64 pipe) are checked
// against these.  Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o pipe_rates pipe_rates_probe.cu && ./pipe_rates
#include <cuda_runtime.h>

#include <cstdio>

namespace {

constexpr int kChains = 8;

template <int OP>
__global__ void k_rate(float* out, int iters, float s) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  float a[kChains];
  float2 b[kChains];
  double d[kChains];
  for (int j = 0; j < kChains; ++j) {
    a[j] = tid * 1e-7f + j;
    b[j] = make_float2(a[j], a[j] + 1.f);
    d[j] = a[j];
  }
  const float2 s2 = make_float2(s, s * 0.5f);
  const double sd = s;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      if (OP == 0) a[j] = __fadd_rn(a[j], s);
      if (OP == 1) b[j] = __fadd2_rn(b[j], s2);
      if (OP == 2) a[j] = fmaf(a[j], s, 0.5f);
      if (OP == 3) b[j] = __ffma2_rn(b[j], s2, s2);
      if (OP == 4) d[j] = fma(d[j], sd, 0.5);
      if (OP == 5) d[j] = (double)__double2float_rn(d[j]) + sd;
    }
  }
  float r = 0.f;
  for (int j = 0; j < kChains; ++j) r += a[j] + b[j].x + b[j].y + (float)d[j];
  out[tid] = r;
}

template <int OP>
float best_ms(float* out, int blocks, int threads, int iters) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_rate<OP><<<blocks, threads>>>(out, iters, 1.0000001f);
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_rate<OP><<<blocks, threads>>>(out, iters, 1.0000001f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int threads = 256, blocks = sms * 8;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 1;
  const double nthr = (double)blocks * threads;
  struct Case {
    const char* name;
    int iters;
    double lanes;  // lane operations per instruction
  } cases[] = {{"fadd", 4096, 1}, {"fadd2", 4096, 2}, {"ffma", 4096, 1}, {"ffma2", 4096, 2}, {"dfma", 2048, 1},
               {"cvt_f64_f32_f64_dadd", 512, 1}};
  for (int c = 0; c < 6; ++c) {
    float ms = 0.f;
    switch (c) {
      case 0: ms = best_ms<0>(out, blocks, threads, cases[c].iters); break;
      case 1: ms = best_ms<1>(out, blocks, threads, cases[c].iters); break;
      case 2: ms = best_ms<2>(out, blocks, threads, cases[c].iters); break;
      case 3: ms = best_ms<3>(out, blocks, threads, cases[c].iters); break;
      case 4: ms = best_ms<4>(out, blocks, threads, cases[c].iters); break;
      default: ms = best_ms<5>(out, blocks, threads, cases[c].iters); break;
    }
    const double instr = nthr * cases[c].iters * kChains;
    std::printf("{\"op\": \"%s\", \"ms\": %.4f, \"lane_ops_per_s\": %.4e, \"sms\": %d}\n", cases[c].name, ms,
                instr * cases[c].lanes / (ms * 1e-3), sms);
  }
  const cudaError_t e = cudaDeviceSynchronize();
  cudaFree(out);
  std::printf("{\"status\": \"%s\"}\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
