// Vector kernels of the point-block Jacobi PCG (ELAS3D-Xtal, arXiv 2602.07354, Algorithm 2).
//
// One iteration of Algorithm 2 is three launches on the device:
//   apply      Ah = A h with the h.Ah partial sums fused into its epilogue; a problem's last
//              item forms lambda = gg / hAh (step B) and applies the breakdown guard
//   update     w -= lambda h, g -= lambda Ah (step C), z = M^-1 g and gg = z.g, g.g (step D);
//              a problem's last item forms gg, gamma = gg / gg_last and decides convergence
//   direction  h = z + gamma h (step E)
// Every launch walks a flattened list of (problem, node chunk) items over all problems of the
// batch (one problem = one RVE with one load case).  All scalars live in device memory
// (DevState per problem), so a batch of iterations runs without the host; a finished (or
// paused) problem's items return at once.  Each item publishes its partial sums, and the
// problem's last item adds them in chunk order, so a problem's result is bitwise reproducible
// and independent of the other problems in the launch.
//
// Precision: the vector type Tv is double (FP64 path) or float (mixed path).  In the mixed path
// w is an unevaluated pair of floats updated with error-free transformations and the dot
// products accumulate compensated pairs, so no FP64 arithmetic runs per node (GB300 issues FP64
// at 1/64 of the FP32 rate).
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

__device__ double total_of(const double* slot, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(slot + i);
  return block_sum(v, red);
}

// Thread 0 publishes this item's partials; true in every thread of the problem's last item.
__device__ bool publish_item(const Prob& P, int chunk, const double* vals, int nvals, unsigned int* ctr, int* s_last) {
  if (threadIdx.x == 0) {
    for (int q = 0; q < nvals; ++q) P.parts[q * P.parts_stride + chunk] = vals[q];
    __threadfence();
    *s_last = atomicAdd(ctr, 1u) == (unsigned)(P.n_chunks - 1);
  }
  __syncthreads();
  return *s_last != 0;
}

__device__ __forceinline__ int wrapi(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

template <typename Tv>
__device__ __forceinline__ void jacobi_apply(const Tv* __restrict__ minv, long long N, long long n, const Tv (&g)[3],
                                             Tv (&z)[3]) {
  const Tv m11 = minv[n], m22 = minv[N + n], m33 = minv[2 * N + n];
  const Tv m23 = minv[3 * N + n], m13 = minv[4 * N + n], m12 = minv[5 * N + n];
  z[0] = m11 * g[0] + m12 * g[1] + m13 * g[2];
  z[1] = m12 * g[0] + m22 * g[1] + m23 * g[2];
  z[2] = m13 * g[0] + m23 * g[1] + m33 * g[2];
}

// Solve setup per problem: tolerances, applied strain, counters; marks the problem for k_pcg_init.
__global__ void k_state_init(const Prob* __restrict__ probs, const SolveSetup* __restrict__ setups,
                             const int* __restrict__ idx, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  DevState* st = probs[idx ? idx[k] : k].st;
  const SolveSetup s = setups[k];
  st->tol = s.tol;
  st->tol2_true = s.tol2_true;
  st->bscale2 = s.bscale2;
  st->max_iter = s.max_iter;
  st->stop_rule = s.stop_rule;
  st->replace_every = s.replace_every;
  st->drop2 = s.drop2;
  for (int q = 0; q < 9; ++q) st->E[q] = s.E[q];
  st->iter = 0;
  st->n_repl = 0;
  st->want_check = 0;
  st->last_repl_iter = 0;
  st->done = 0;
  st->needs_init = 1;
  st->status = ST_RUNNING;
  st->gg = st->gg0 = st->gg_last = st->hAh = st->hAh_first = st->lambda = st->gamma = 0.0;
  st->rr = st->bb = st->rr_true = 0.0;
  for (int q = 0; q < 8; ++q) st->ctr[q] = 0u;  // in case an earlier solve ended inside a reduction
}

// Initial state of Algorithm 2 in fluctuation form: w = 0, g = b (right-hand side of Eqs. 7-8
// from the closed form b_m = sum_e sigma_e . s_a / 4), z = M^-1 g, h = z, gg0 = z.g.
template <typename Tv>
__global__ void k_pcg_init(const Prob* __restrict__ probs, const int* __restrict__ vitem_prob,
                           const long long* __restrict__ counts) {
  __shared__ double red[32];
  __shared__ int s_last;
  const long long n_items = counts[1];
  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Prob& P = probs[vitem_prob[item]];
    if (!P.st->needs_init) continue;  // only problems set up since their last start
    const int chunk = (int)(item - P.item0_vec);
    const long long N = P.N, n0 = (long long)chunk * kVecChunk, n1 = min(n0 + kVecChunk, N);
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    Tv* __restrict__ g = reinterpret_cast<Tv*>(P.g);
    Tv* __restrict__ h = reinterpret_cast<Tv*>(P.h);
    Tv* __restrict__ z = reinterpret_cast<Tv*>(P.z);
    double* __restrict__ w = P.w;
    float* __restrict__ w_hi = P.w_hi;
    float* __restrict__ w_lo = P.w_lo;
    const int32_t* __restrict__ phase = P.phase;
    const double* __restrict__ sig = P.sig;
    const Tv* __restrict__ minv = reinterpret_cast<const Tv*>(P.minv);
    DotAcc<Tv> zg, gg2;
    DotAcc<double> bb;
#pragma unroll
    for (int q = 0; q < kVecPerThread; ++q) {
      const long long n = n0 + q * kVecThreads + threadIdx.x;
      if (n >= n1) break;
      const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / ((long long)nx * ny));
      double b[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        const long long e = (long long)wrapi(i - ax, nx) +
                            (long long)nx * (wrapi(j - ay, ny) + (long long)ny * wrapi(k - az, nz));
        const int ph = phase[e];
        if (ph < 0) continue;
        const double* S = sig + 6 * (long long)ph;
        const double sx = 0.25 * (2 * ax - 1), sy = 0.25 * (2 * ay - 1), sz = 0.25 * (2 * az - 1);
        b[0] += S[0] * sx + S[5] * sy + S[4] * sz;
        b[1] += S[5] * sx + S[1] * sy + S[3] * sz;
        b[2] += S[4] * sx + S[3] * sy + S[2] * sz;
      }
      Tv gv[3], zv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        gv[c] = (Tv)b[c];
        bb.add(b[c], b[c]);
        gg2.add(gv[c], gv[c]);
      }
      jacobi_apply(minv, N, n, gv, zv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        w[c * N + n] = 0.0;
        if (w_hi) {
          w_hi[c * N + n] = 0.f;
          w_lo[c * N + n] = 0.f;
        }
        g[c * N + n] = gv[c];
        z[c * N + n] = zv[c];
        h[c * N + n] = zv[c];
        zg.add(zv[c], gv[c]);
      }
    }
    const double vals[3] = {block_total(zg, red), block_total(bb, red), block_total(gg2, red)};
    if (publish_item(P, chunk, vals, 3, &P.st->ctr[1], &s_last)) {
      const double s_zg = total_of(P.parts, P.n_chunks, red);
      const double s_bb = total_of(P.parts + P.parts_stride, P.n_chunks, red);
      const double s_gg = total_of(P.parts + 2 * P.parts_stride, P.n_chunks, red);
      if (threadIdx.x == 0) {
        DevState* st = P.st;
        st->ctr[1] = 0u;
        st->needs_init = 0;
        st->gg = st->gg0 = s_zg;
        st->bb = s_bb;
        st->rr = s_gg;
        st->rr_repl = s_gg;
        if (!isfinite(s_zg) || !isfinite(s_bb)) {
          st->status = ELAS_NONFINITE;
          st->done = 1;
        } else if (s_bb <= 1e-24 * st->bscale2) {
          // zero load (round-off of an exactly zero right-hand side): w = 0 is the solution
          st->status = ELAS_CONVERGED;
          st->done = 1;
        } else if (!(s_zg > 0.0)) {
          // z.g of a non-zero load is not positive: the preconditioner is not definite
          st->status = ELAS_BREAKDOWN;
          st->done = 1;
        } else if (st->max_iter <= 0) {
          st->status = ELAS_MAX_ITER;
          st->done = 1;
        }
      }
    }
    __syncthreads();
  }
}

// One node of steps C and D: w -= lambda h, g -= lambda Ah, z = M^-1 g, and the two dot terms.
// Mixed path: w is the unevaluated pair (wh, wl), updated with error-free transformations
// (_rn intrinsics keep the compiler from contracting them into FMAs).
template <bool MIXED, typename Tv>
__device__ __forceinline__ void update_node(const Tv (&h)[3], const Tv (&Ah)[3], Tv (&g)[3], float (&wh)[3],
                                            float (&wl)[3], double* w, long long N, long long n, const Tv (&m)[6],
                                            Tv (&z)[3], double lam, float lam_hi, float lam_lo, Tv lam_v,
                                            DotAcc<Tv>& zg, DotAcc<Tv>& gg2) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MIXED) {
      const float hf = (float)h[c];
      const float prod = __fmul_rn(lam_hi, hf);
      const float perr = __fadd_rn(fmaf(lam_hi, hf, -prod), __fmul_rn(lam_lo, hf));  // lambda h = prod + perr
      const float s = __fsub_rn(wh[c], prod);  // two-sum of wh and -prod
      const float bb = __fsub_rn(s, wh[c]);
      const float e =
          __fadd_rn(__fadd_rn(__fsub_rn(wh[c], __fsub_rn(s, bb)), __fsub_rn(-prod, bb)), __fsub_rn(wl[c], perr));
      const float nh = __fadd_rn(s, e);  // renormalise the pair
      wl[c] = __fsub_rn(e, __fsub_rn(nh, s));
      wh[c] = nh;
    } else {
      w[c * N + n] -= lam * (double)h[c];
    }
    g[c] = g[c] - lam_v * Ah[c];
    gg2.add(g[c], g[c]);
  }
  // point-block Jacobi, symmetric inverse in Voigt slot order 11, 22, 33, 23, 13, 12
  z[0] = m[0] * g[0] + m[5] * g[1] + m[4] * g[2];
  z[1] = m[5] * g[0] + m[1] * g[1] + m[3] * g[2];
  z[2] = m[4] * g[0] + m[3] * g[1] + m[2] * g[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) zg.add(z[c], g[c]);
}

// The scalar step D/E of Algorithm 2 on a problem's totals z.g and g.g (one thread): gg,
// gamma = gg / gg_last, the iteration count and the stopping tests.
__device__ void update_scalar_step(DevState* st, double s_zg, double s_gg, bool mixed) {
  st->ctr[2] = 0u;
  st->gg_last = st->gg;
  st->gg = s_zg;
  st->rr = s_gg;
  st->iter += 1;
  if (!isfinite(s_zg) || !isfinite(s_gg)) {
    st->status = ELAS_NONFINITE;
    st->done = 1;
  } else {
    const bool est = (st->stop_rule == ELAS_STOP_TRUE) ? (s_gg <= st->tol2_true * st->bb)
                                                        : (s_zg < st->tol * st->tol * st->gg0);
    if (est) {
      if (mixed || st->stop_rule == ELAS_STOP_TRUE) {
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
    st->gam_f = (float)st->gamma;
  }
}

// Publishes an update item's partials (z.g, g.g); the problem's last item performs the scalar step.
__device__ void finish_update(const Prob& P, int chunk, const double (&vals)[2], bool mixed, double* red,
                              int* s_last) {
  if (publish_item(P, chunk, vals, 2, &P.st->ctr[2], s_last)) {
    const double s_zg = total_of(P.parts, P.n_chunks, red);
    const double s_gg = total_of(P.parts + P.parts_stride, P.n_chunks, red);
    if (threadIdx.x == 0) update_scalar_step(P.st, s_zg, s_gg, mixed);
  }
}

__device__ __forceinline__ float q4(const float4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }
__device__ __forceinline__ void s4(float4& v, int j, float x) {
  if (j == 0) v.x = x; else if (j == 1) v.y = x; else if (j == 2) v.z = x; else v.w = x;
}

// Steps C and D of Algorithm 2.  FP32 vectors of a grid whose size is a multiple of 4 move as
// float4 (each thread owns 4 consecutive nodes), all other cases node by node.
template <typename Tv, bool MIXED, bool VEC>
__device__ __forceinline__ void update_items(const Prob* __restrict__ probs, const int* __restrict__ vitem_prob,
                                             const long long* __restrict__ counts) {
  __shared__ double red[32];
  __shared__ int s_last;
  const long long n_items = counts[1];
  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Prob& P = probs[vitem_prob[item]];
    const DevState* cst = P.st;
    if (cst->done || cst->want_check) continue;
    const int chunk = (int)(item - P.item0_vec);
    const long long N = P.N, n0 = (long long)chunk * kVecChunk, n1 = min(n0 + kVecChunk, N);
    Tv* __restrict__ gp = reinterpret_cast<Tv*>(P.g);
    const Tv* __restrict__ hp = reinterpret_cast<const Tv*>(P.h);
    const Tv* __restrict__ Ahp = reinterpret_cast<const Tv*>(P.Ah);
    Tv* __restrict__ zp = reinterpret_cast<Tv*>(P.z);
    const Tv* __restrict__ minv = reinterpret_cast<const Tv*>(P.minv);
    double* __restrict__ w = P.w;
    float* __restrict__ w_hi = P.w_hi;
    float* __restrict__ w_lo = P.w_lo;
    const double lam = cst->lambda;
    const float lam_hi = cst->lam_hi, lam_lo = cst->lam_lo;  // formed once per problem
    const Tv lam_v = MIXED ? (Tv)lam_hi : (Tv)lam;
    DotAcc<Tv> zg, gg2;
    const long long nq = n0 + 4 * (long long)threadIdx.x;
    if (VEC && MIXED && (N & 3) == 0 && nq + 3 < n1) {
      // vector path: 4 consecutive nodes per thread, 21 float4 loads and 12 float4 stores
      float4 h4[3], A4[3], g4[3], wh4[3], wl4[3], m4[6], z4[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h4[c] = *reinterpret_cast<const float4*>(hp + c * N + nq);
        A4[c] = *reinterpret_cast<const float4*>(Ahp + c * N + nq);
        g4[c] = *reinterpret_cast<const float4*>(gp + c * N + nq);
        wh4[c] = *reinterpret_cast<const float4*>(w_hi + c * N + nq);
        wl4[c] = *reinterpret_cast<const float4*>(w_lo + c * N + nq);
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) m4[q] = *reinterpret_cast<const float4*>(minv + q * N + nq);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        Tv h[3], Ah[3], g[3], m[6], z[3];
        float wh[3], wl[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          h[c] = q4(h4[c], j); Ah[c] = q4(A4[c], j); g[c] = q4(g4[c], j);
          wh[c] = q4(wh4[c], j); wl[c] = q4(wl4[c], j);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) m[q] = q4(m4[q], j);
        update_node<MIXED>(h, Ah, g, wh, wl, w, N, nq + j, m, z, lam, lam_hi, lam_lo, lam_v, zg, gg2);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s4(g4[c], j, g[c]); s4(z4[c], j, z[c]); s4(wh4[c], j, wh[c]); s4(wl4[c], j, wl[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        *reinterpret_cast<float4*>(gp + c * N + nq) = g4[c];
        *reinterpret_cast<float4*>(zp + c * N + nq) = z4[c];
        *reinterpret_cast<float4*>(w_hi + c * N + nq) = wh4[c];
        *reinterpret_cast<float4*>(w_lo + c * N + nq) = wl4[c];
      }
    } else {
      // node by node: thread t owns nodes n0 + t + q*256 (the vector path's ragged tail and
      // grids whose size is not a multiple of 4 run here; which path a node takes depends only
      // on its problem)
      const bool vec_problem = VEC && MIXED && (N & 3) == 0;
#pragma unroll
      for (int q = 0; q < kVecPerThread; ++q) {
        const long long n = vec_problem ? nq + q : n0 + q * kVecThreads + threadIdx.x;
        if (n >= n1) break;
        Tv h[3], Ah[3], g[3], m[6], z[3];
        float wh[3] = {0.f, 0.f, 0.f}, wl[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          h[c] = hp[c * N + n];
          Ah[c] = Ahp[c * N + n];
          g[c] = gp[c * N + n];
          if (MIXED) {
            wh[c] = w_hi[c * N + n];
            wl[c] = w_lo[c * N + n];
          }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) m[k] = minv[k * N + n];
        update_node<MIXED>(h, Ah, g, wh, wl, w, N, n, m, z, lam, lam_hi, lam_lo, lam_v, zg, gg2);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          gp[c * N + n] = g[c];
          zp[c * N + n] = z[c];
          if (MIXED) {
            w_hi[c * N + n] = wh[c];
            w_lo[c * N + n] = wl[c];
          }
        }
      }
    }
    const double vals[2] = {block_total(zg, red), block_total(gg2, red)};
    finish_update(P, chunk, vals, MIXED, red, &s_last);
    __syncthreads();
  }
}

// FP64: four resident blocks per SM (64 registers): 3.6% faster per FP64 solve than three, 5% than
// two; the update is bound by both the FP64 pipe (21 FP64 operations per node) and HBM.
__global__ void __launch_bounds__(kVecThreads, 4)
    k_pcg_update_f64(const Prob* __restrict__ probs, const int* __restrict__ vitem_prob,
                     const long long* __restrict__ counts) {
  update_items<double, false, false>(probs, vitem_prob, counts);
}
// Mixed path: four consecutive nodes per thread as float4 rows, the compiler's own register choice
// (measured against one node at a time per thread at 3, 4 and 6 blocks per SM: 51-66 ms per
// mixed solve against 47 ms).
__global__ void k_pcg_update_f32(const Prob* __restrict__ probs, const int* __restrict__ vitem_prob,
                                 const long long* __restrict__ counts) {
  update_items<float, true, true>(probs, vitem_prob, counts);
}

// Step E of Algorithm 2 (Fletcher-Reeves direction).
template <typename Tv>
__global__ void k_pcg_direction(const Prob* __restrict__ probs, const int* __restrict__ vitem_prob,
                                const long long* __restrict__ counts) {
  const long long n_items = counts[1];
  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Prob& P = probs[vitem_prob[item]];
    const DevState* cst = P.st;
    if (cst->done || cst->want_check) continue;
    const int chunk = (int)(item - P.item0_vec);
    const long long N = P.N, n0 = (long long)chunk * kVecChunk, n1 = min(n0 + kVecChunk, N);
    const Tv gam = sizeof(Tv) == 4 ? (Tv)cst->gam_f : (Tv)cst->gamma;
    Tv* __restrict__ h = reinterpret_cast<Tv*>(P.h);
    const Tv* __restrict__ z = reinterpret_cast<const Tv*>(P.z);
    const long long nq = n0 + 4 * (long long)threadIdx.x;
    if (sizeof(Tv) == 4 && (N & 3) == 0 && nq + 3 < n1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float4 hv = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(h) + c * N + nq);
        const float4 zv = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(z) + c * N + nq);
        const float gf = (float)gam;
        hv.x = zv.x + gf * hv.x; hv.y = zv.y + gf * hv.y; hv.z = zv.z + gf * hv.z; hv.w = zv.w + gf * hv.w;
        *reinterpret_cast<float4*>(reinterpret_cast<float*>(h) + c * N + nq) = hv;
      }
    } else {
      const bool vec_problem = sizeof(Tv) == 4 && (N & 3) == 0;
#pragma unroll
      for (int q = 0; q < kVecPerThread; ++q) {
        const long long n = vec_problem ? nq + q : n0 + q * kVecThreads + threadIdx.x;
        if (n >= n1) break;
#pragma unroll
        for (int c = 0; c < 3; ++c) h[c * N + n] = z[c * N + n] + gam * h[c * N + n];
      }
    }
  }
}

// w = w_hi + w_lo (FP64) for the FP64 residual replacement and the solve's output.  Gated like the
// kernel that follows it: the residual replacement, or the final true residual of a stopped problem.
__global__ void k_w_combine(const Prob* __restrict__ probs, const int* __restrict__ vitem_prob,
                            const long long* __restrict__ counts, int gate) {
  const long long n_items = counts[1];
  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Prob& P = probs[vitem_prob[item]];
    const DevState* st = P.st;
    if (gate == GATE_REPLACE && (st->done || !replacement_due(st))) continue;
    if (gate == GATE_FINALIZE && (!st->done || st->finalized)) continue;
    const int chunk = (int)(item - P.item0_vec);
    const long long N = P.N, n0 = (long long)chunk * kVecChunk, n1 = min(n0 + kVecChunk, N);
    double* __restrict__ w = P.w;
    const float* __restrict__ w_hi = P.w_hi;
    const float* __restrict__ w_lo = P.w_lo;
#pragma unroll
    for (int q = 0; q < kVecPerThread; ++q) {
      const long long n = n0 + q * kVecThreads + threadIdx.x;
      if (n >= n1) break;
#pragma unroll
      for (int c = 0; c < 3; ++c) w[c * N + n] = (double)w_hi[c * N + n] + (double)w_lo[c * N + n];
    }
  }
}

}  // namespace

cudaError_t launch_state_init(const BatchDev& b, const SolveSetup* setups, const int* idx, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_state_init<<<(n + 127) / 128, 128, 0, s>>>(b.probs, setups, idx, n);
  return cudaGetLastError();
}

cudaError_t launch_pcg_init(const BatchDev& b, bool mixed, cudaStream_t s) {
  if (mixed)
    k_pcg_init<float><<<b.vec_blocks, b.vec_threads, 0, s>>>(b.probs, b.vitem_prob, b.counts);
  else
    k_pcg_init<double><<<b.vec_blocks, b.vec_threads, 0, s>>>(b.probs, b.vitem_prob, b.counts);
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(const BatchDev& b, bool mixed, cudaStream_t s) {
  if (mixed)
    k_pcg_update_f32<<<b.vec_blocks, b.vec_threads, 0, s>>>(b.probs, b.vitem_prob, b.counts);
  else
    k_pcg_update_f64<<<b.vec_blocks, b.vec_threads, 0, s>>>(b.probs, b.vitem_prob, b.counts);
  return cudaGetLastError();
}

cudaError_t launch_pcg_direction(const BatchDev& b, bool mixed, cudaStream_t s) {
  if (mixed)
    k_pcg_direction<float><<<b.vec_blocks, b.vec_threads, 0, s>>>(b.probs, b.vitem_prob, b.counts);
  else
    k_pcg_direction<double><<<b.vec_blocks, b.vec_threads, 0, s>>>(b.probs, b.vitem_prob, b.counts);
  return cudaGetLastError();
}

cudaError_t launch_w_combine(const BatchDev& b, int gate, cudaStream_t s) {
  k_w_combine<<<b.vec_blocks, b.vec_threads, 0, s>>>(b.probs, b.vitem_prob, b.counts, gate);
  return cudaGetLastError();
}

}  // namespace elas
