// Vector kernels of the point-block Jacobi PCG (ELAS3D-Xtal, arXiv 2602.07354, Algorithm 2).
//
// One iteration of Algorithm 2 is three launches on the device:
//   apply      Ah = A h with the h.Ah partial sums fused into its epilogue; its last block forms
//              lambda = gg / hAh (step B) and applies the breakdown guard
//   update     w -= lambda h, g -= lambda Ah (step C), z = M^-1 g and gg = z.g, g.g (step D);
//              its last block forms gg, gamma = gg / gg_last and decides convergence (step D)
//   direction  h = z + gamma h (step E)
// All scalars live in device memory (DevState), so a batch of iterations runs without the host;
// kernels of a finished (or paused) solve return immediately.  Reductions are FP64 and summed
// in a fixed order, so a solve is bitwise reproducible.
//
// Precision: the vector type Tv is double (FP64 path) or float (mixed path).  The fluctuation
// w is FP64 in both; reductions accumulate FP64.
#include <cuda_runtime.h>

#include "elas_internal.h"

namespace elas {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) r += red[i];
  }
  return r;
}

__device__ bool publish_and_arrive(double* parts, const double* vals, int nvals, unsigned int* ctr) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    for (int q = 0; q < nvals; ++q) parts[q * kMaxParts + blockIdx.x] = vals[q];
    __threadfence();
    const unsigned int t = atomicAdd(ctr, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return s_last != 0;
}

__device__ double total_of(const double* slot, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(slot + i);
  return block_sum(v, red);
}

__device__ __forceinline__ int wrapi(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

template <typename Tv>
struct VecP {
  int nx, ny, nz;
  long long N;
  const int32_t* __restrict__ phase;
  const double* __restrict__ sig;
  double* __restrict__ w;
  float* __restrict__ w_hi;
  float* __restrict__ w_lo;
  Tv* __restrict__ g;
  Tv* __restrict__ h;
  Tv* __restrict__ Ah;
  Tv* __restrict__ z;
  const Tv* __restrict__ minv;
  double* parts;
  DevState* st;
};

template <typename Tv>
__device__ __forceinline__ void jacobi_apply(const Tv* __restrict__ minv, long long N, long long n, const Tv (&g)[3],
                                             Tv (&z)[3]) {
  const Tv m11 = minv[n], m22 = minv[N + n], m33 = minv[2 * N + n];
  const Tv m23 = minv[3 * N + n], m13 = minv[4 * N + n], m12 = minv[5 * N + n];
  z[0] = m11 * g[0] + m12 * g[1] + m13 * g[2];
  z[1] = m12 * g[0] + m22 * g[1] + m23 * g[2];
  z[2] = m13 * g[0] + m23 * g[1] + m33 * g[2];
}

// Solve setup: tolerances and counters (kernel arguments are captured by value in graphs).
__global__ void k_state_init(DevState* st, SolveSetup s) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->tol = s.tol;
  st->tol2_true = s.tol2_true;
  st->bscale2 = s.bscale2;
  st->max_iter = s.max_iter;
  st->stop_rule = s.stop_rule;
  st->replace_every = s.replace_every;
  for (int q = 0; q < 9; ++q) st->E[q] = s.E[q];
  st->iter = 0;
  st->n_repl = 0;
  st->want_check = 0;
  st->last_repl_iter = 0;
  st->done = 0;
  st->status = ST_RUNNING;
  st->gg = st->gg0 = st->gg_last = st->hAh = st->hAh_first = st->lambda = st->gamma = 0.0;
  st->rr = st->bb = st->rr_true = 0.0;
}

// Initial state of Algorithm 2 in fluctuation form: w = 0, g = b (right-hand side of Eqs. 7-8
// from the closed form b_m = sum_e sigma_e . s_a / 4), z = M^-1 g, h = z, gg0 = z.g.
template <typename Tv>
__global__ void k_pcg_init(const VecP<Tv> p) {
  __shared__ double red[32];
  DotAcc<Tv> zg, gg2;
  DotAcc<double> bb;
  const long long N = p.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(n % p.nx), j = (int)((n / p.nx) % p.ny), k = (int)(n / ((long long)p.nx * p.ny));
    double b[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
      const long long e =
          (long long)wrapi(i - ax, p.nx) + (long long)p.nx * (wrapi(j - ay, p.ny) + (long long)p.ny * wrapi(k - az, p.nz));
      const int ph = p.phase[e];
      if (ph < 0) continue;
      const double* S = p.sig + 6 * (long long)ph;
      const double sx = 0.25 * (2 * ax - 1), sy = 0.25 * (2 * ay - 1), sz = 0.25 * (2 * az - 1);
      b[0] += S[0] * sx + S[5] * sy + S[4] * sz;
      b[1] += S[5] * sx + S[1] * sy + S[3] * sz;
      b[2] += S[4] * sx + S[3] * sy + S[2] * sz;
    }
    Tv g[3], z[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      g[c] = (Tv)b[c];
      bb.add(b[c], b[c]);
      gg2.add(g[c], g[c]);
    }
    jacobi_apply(p.minv, N, n, g, z);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p.w[c * N + n] = 0.0;
      if (p.w_hi) {
        p.w_hi[c * N + n] = 0.f;
        p.w_lo[c * N + n] = 0.f;
      }
      p.g[c * N + n] = g[c];
      p.z[c * N + n] = z[c];
      p.h[c * N + n] = z[c];
      zg.add(z[c], g[c]);
    }
  }
  const double vals[3] = {block_sum(zg.value(), red), block_sum(bb.value(), red), block_sum(gg2.value(), red)};
  if (!publish_and_arrive(p.parts, vals, 3, &p.st->ctr[1])) return;
  const double s_zg = total_of(p.parts, gridDim.x, red);
  const double s_bb = total_of(p.parts + kMaxParts, gridDim.x, red);
  const double s_gg = total_of(p.parts + 2 * kMaxParts, gridDim.x, red);
  if (threadIdx.x == 0) {
    DevState* st = p.st;
    st->ctr[1] = 0u;
    st->gg = st->gg0 = s_zg;
    st->bb = s_bb;
    st->rr = s_gg;
    if (!isfinite(s_zg) || !isfinite(s_bb)) {
      st->status = ELAS_NONFINITE;
      st->done = 1;
    } else if (!(s_zg > 0.0) || s_bb <= 1e-24 * st->bscale2) {
      // zero load (round-off of an exactly zero right-hand side): w = 0 is the solution
      st->status = ELAS_CONVERGED;
      st->done = 1;
    }
  }
}

// Steps C and D of Algorithm 2.
template <typename Tv, bool MIXED>
__global__ void k_pcg_update(const VecP<Tv> p) {
  __shared__ double red[32];
  const DevState* cst = p.st;
  if (cst->done || cst->want_check) return;
  const double lam = cst->lambda;
  const Tv lam_v = (Tv)lam;
  // mixed path: lambda as an unevaluated float pair, w updated with error-free transformations
  const float lam_hi = (float)lam, lam_lo = (float)(lam - (double)lam_hi);
  DotAcc<Tv> zg, gg2;
  const long long N = p.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    Tv g[3], z[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const Tv hc = p.h[c * N + n];
      if (MIXED) {
        // (_rn intrinsics: no FMA contraction inside the error-free transformations)
        const float hf = (float)hc;
        const float prod = __fmul_rn(lam_hi, hf);
        const float perr = __fadd_rn(fmaf(lam_hi, hf, -prod), __fmul_rn(lam_lo, hf));  // lambda h = prod + perr
        const float wh = p.w_hi[c * N + n], wl = p.w_lo[c * N + n];
        const float s = __fsub_rn(wh, prod);  // two-sum of wh and -prod
        const float bb = __fsub_rn(s, wh);
        const float e = __fadd_rn(__fadd_rn(__fsub_rn(wh, __fsub_rn(s, bb)), __fsub_rn(-prod, bb)), __fsub_rn(wl, perr));
        const float nh = __fadd_rn(s, e);  // renormalise the pair
        p.w_hi[c * N + n] = nh;
        p.w_lo[c * N + n] = __fsub_rn(e, __fsub_rn(nh, s));
      } else {
        p.w[c * N + n] -= lam * (double)hc;
      }
      g[c] = p.g[c * N + n] - lam_v * p.Ah[c * N + n];
      p.g[c * N + n] = g[c];
      gg2.add(g[c], g[c]);
    }
    jacobi_apply(p.minv, N, n, g, z);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p.z[c * N + n] = z[c];
      zg.add(z[c], g[c]);
    }
  }
  const double vals[2] = {block_sum(zg.value(), red), block_sum(gg2.value(), red)};
  if (!publish_and_arrive(p.parts, vals, 2, &p.st->ctr[2])) return;
  const double s_zg = total_of(p.parts, gridDim.x, red);
  const double s_gg = total_of(p.parts + kMaxParts, gridDim.x, red);
  if (threadIdx.x == 0) {
    DevState* st = p.st;
    st->ctr[2] = 0u;
    st->gg_last = st->gg;
    st->gg = s_zg;
    st->rr = s_gg;
    st->iter += 1;
    if (!isfinite(s_zg) || !isfinite(s_gg)) {
      st->status = ELAS_NONFINITE;
      st->done = 1;
      return;
    }
    const bool est = (st->stop_rule == ELAS_STOP_TRUE) ? (s_gg <= st->tol2_true * st->bb)
                                                        : (s_zg < st->tol * st->tol * st->gg0);
    if (est) {
      if (MIXED || st->stop_rule == ELAS_STOP_TRUE) {
        st->want_check = 1;  // confirm on the FP64 true residual before stopping
      } else {
        st->status = ELAS_CONVERGED;
        st->done = 1;
      }
    } else if (st->iter >= st->max_iter) {
      st->status = ELAS_MAX_ITER;
      st->done = 1;
    }
    st->gamma = s_zg / st->gg_last;
  }
}

// Step E of Algorithm 2 (Fletcher-Reeves direction).
template <typename Tv>
__global__ void k_pcg_direction(const VecP<Tv> p) {
  const DevState* cst = p.st;
  if (cst->done || cst->want_check) return;
  const Tv gam = (Tv)cst->gamma;
  const long long N3 = 3 * p.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N3; t += (long long)gridDim.x * blockDim.x)
    p.h[t] = p.z[t] + gam * p.h[t];
}

// w = w_hi + w_lo (FP64) for the FP64 residual replacement and the solve's output.  When gated it
// runs only where the residual replacement that follows it runs.
__global__ void k_w_combine(const float* __restrict__ w_hi, const float* __restrict__ w_lo, double* __restrict__ w,
                            long long n3, int gated, const DevState* st) {
  if (gated && (st->done || !(st->want_check ||
                              (st->replace_every > 0 && st->iter - st->last_repl_iter >= st->replace_every))))
    return;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3; t += (long long)gridDim.x * blockDim.x)
    w[t] = (double)w_hi[t] + (double)w_lo[t];
}

template <typename Tv>
VecP<Tv> make_p(const VecLaunch& v) {
  VecP<Tv> p;
  p.nx = v.geo.nx; p.ny = v.geo.ny; p.nz = v.geo.nz; p.N = v.geo.N;
  p.phase = v.phase;
  p.sig = v.sig;
  p.w = v.w;
  p.w_hi = v.w_hi;
  p.w_lo = v.w_lo;
  p.g = static_cast<Tv*>(v.g);
  p.h = static_cast<Tv*>(v.h);
  p.Ah = static_cast<Tv*>(v.Ah);
  p.z = static_cast<Tv*>(v.z);
  p.minv = static_cast<const Tv*>(v.minv);
  p.parts = v.parts;
  p.st = v.st;
  return p;
}

}  // namespace

cudaError_t launch_state_init(DevState* st, const SolveSetup& s, cudaStream_t stream) {
  k_state_init<<<1, 32, 0, stream>>>(st, s);
  return cudaGetLastError();
}

cudaError_t launch_pcg_init(const VecLaunch& v, bool mixed, cudaStream_t s) {
  if (mixed)
    k_pcg_init<float><<<v.blocks, v.threads, 0, s>>>(make_p<float>(v));
  else
    k_pcg_init<double><<<v.blocks, v.threads, 0, s>>>(make_p<double>(v));
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(const VecLaunch& v, bool mixed, cudaStream_t s) {
  if (mixed)
    k_pcg_update<float, true><<<v.blocks, v.threads, 0, s>>>(make_p<float>(v));
  else
    k_pcg_update<double, false><<<v.blocks, v.threads, 0, s>>>(make_p<double>(v));
  return cudaGetLastError();
}

cudaError_t launch_pcg_direction(const VecLaunch& v, bool mixed, cudaStream_t s) {
  if (mixed)
    k_pcg_direction<float><<<v.blocks, v.threads, 0, s>>>(make_p<float>(v));
  else
    k_pcg_direction<double><<<v.blocks, v.threads, 0, s>>>(make_p<double>(v));
  return cudaGetLastError();
}

cudaError_t launch_w_combine(const VecLaunch& v, bool gated, cudaStream_t s) {
  k_w_combine<<<v.blocks, v.threads, 0, s>>>(v.w_hi, v.w_lo, v.w, 3 * v.geo.N, gated ? 1 : 0, v.st);
  return cudaGetLastError();
}

}  // namespace elas
