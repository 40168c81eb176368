// Internal declarations shared by the CUDA translation units of libelas.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include <cstddef>
#include <cstdint>
#include <string>

#include "elas.h"

namespace elas {

// ------------------------------------------------------------------------------------------
// Per-phase coefficient block (device): the three scaled copies of the sample-frame Voigt
// stiffness used by the modal element product, packed symmetric (21 entries each, each copy
// starting on a 32-entry boundary so it loads as aligned vectors):
//   [0,21)   C/16   constant-strain mode
//   [32,53)  C/48   the three linear modes
//   [64,85)  C/144  the three bilinear modes
//   [96]     1 if the phase is solid, 0 for a pore
// plus, in a separate table, the unscaled C (21 entries) for stress and Jacobi.
// ------------------------------------------------------------------------------------------
constexpr int kCoefStride = 128;
constexpr int kCoefMode0 = 0, kCoefMode1 = 32, kCoefMode2 = 64, kCoefFlag = 96;
// the solid flag is also kept in the padding of the C/16 block, so the operator reads it with
// that block's first vector loads
constexpr int kCoefSolid0 = 21;
// FP64 table only: the diagonal 3x3 blocks (K_e)_aa of the element stiffness for the corners
// a = 0..3 (corner 7 - a has the same block), 6 Voigt-ordered entries each.
constexpr int kCoefJac = 100;
constexpr int kSymStride = 21;
// FP32 coefficient table (floats per phase): [0, 128) the FP32 copy of the layout above, then the
// float-pair copy of the three scaled blocks used by the FP64 operator in double-float arithmetic:
// block b at kCoefFF + kCoefFFBlock * b holds 24 (hi, lo) pairs (entry 21 of block 0: solid flag),
// each pair the double value split exactly as hi = fl32(v), lo = fl32(v - hi).
constexpr int kCoefFF = 128, kCoefFFBlock = 48;
constexpr int kCoef32Stride = 288;
constexpr int kMaxThreadsF64 = 384, kMaxThreadsF32 = 384;
// largest dynamic shared memory of an operator tile (the 4-slot node ring and the face buffers)
constexpr size_t kApplySmemMax = 200 * 1024;
// per-thread slots of the double-float operator's carried face forces (6 float4 per thread)
constexpr size_t kFupSlotBytes = (size_t)6 * 16 * kMaxThreadsF64;

__host__ __device__ constexpr int pk(int i, int j) {
  return i <= j ? i * 6 - i * (i - 1) / 2 + (j - i) : j * 6 - j * (j - 1) / 2 + (i - j);
}

// Solver scalars kept on the device between kernels (one per solve).
struct DevState {
  double gg, gg0, gg_last, hAh, hAh_first, lambda, gamma;
  double rr;        // g.g of the current recursive residual (FP64 accumulation)
  double bb;        // ||b||^2 (FP64)
  double rr_true;   // ||A w + b||^2 of the last FP64 residual (replacement / final check)
  double tol, tol2_true, bscale2;
  double rr_repl;   // rr right after the last replacement (or at the start)
  double drop2;     // replace once rr <= drop2 * rr_repl (0: off)
  int iter, max_iter, status, done;
  int stop_rule, n_repl, want_check, last_repl_iter;
  int replace_every, needs_init, finalized, pad2;
  float lam_hi, lam_lo;  // lambda as an unevaluated float pair (mixed path)
  float gam_f, pad_f;    // gamma rounded to float (mixed path)
  double E[9];           // applied strain tensor (row-major) of the current solve / product
  double macro[6];       // macroscopic stress of the last elas_stress
  unsigned int ctr[8];   // arrival counters of the last-block reductions (self-resetting)
};

// Which kernels of a solve skip their work:
//   GATE_NONE     never (stand-alone products)
//   GATE_RUNNING  when the solve is done or paused for an FP64 residual check
//   GATE_REPLACE  unless a residual check is wanted or the replacement interval has elapsed
//   GATE_FINALIZE unless the problem has stopped and its final FP64 w / true residual are not formed
enum { GATE_NONE = 0, GATE_RUNNING = 1, GATE_REPLACE = 2, GATE_FINALIZE = 3 };

#ifdef __CUDACC__
// The mixed path's FP64 residual replacement is due: a convergence check is pending, the
// replacement interval has elapsed, or the residual has dropped by the requested factor.
__device__ __forceinline__ bool replacement_due(const DevState* st) {
  return st->want_check || (st->replace_every > 0 && st->iter - st->last_repl_iter >= st->replace_every) ||
         (st->drop2 > 0.0 && st->rr <= st->drop2 * st->rr_repl);
}
#endif

struct StressE {
  double v[6];
};

#ifdef __CUDACC__
// ---- double-float arithmetic ------------------------------------------------------------------
// An FP64 value carried as an unevaluated pair of floats v = hi + lo (about 48 significant bits),
// operated on with the FP32 pipe, which GB300 issues at 64x the FP64 rate.  The building blocks
// are the error-free transformations of Knuth (TwoSum: the rounding error of a float sum is a
// float, 1969) and Dekker (TwoProd: the rounding error of a float product, obtained here with one
// fused multiply-add, 1971).  Sums keep the exact error of the leading parts and add the trailing
// parts in plain FP32 (the "sloppy" double-float sum), so the error of a sum is a few units of
// 2^-48 of its operands' magnitude; pairs are renormalised (Fast2Sum) where they enter a product.
// The _rn intrinsics keep the compiler from contracting or reordering the error terms.
struct ff {
  float hi, lo;
  ff() = default;
  __device__ __forceinline__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit ff(int v) : hi((float)v), lo(0.f) {}
  // exact split of a double into its rounded leading float and the float nearest the remainder
  __device__ __forceinline__ explicit ff(double v) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
};
// TwoSum: s + e = a + b exactly
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
// Fast2Sum renormalisation of a pair whose leading part dominates
__device__ __forceinline__ ff ff_norm(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  return ff(s, __fsub_rn(lo, __fsub_rn(s, hi)));
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
  float e;
  const float s = two_sum(a.hi, b.hi, e);
  return ff(s, __fadd_rn(__fadd_rn(a.lo, b.lo), e));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
// product: TwoProd of the leading parts plus the cross terms (the lo*lo term is below 2^-48)
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_norm(p, e);
}
__device__ __forceinline__ bool operator!=(ff a, ff b) { return a.hi != b.hi || a.lo != b.lo; }
#endif

#ifdef __CUDACC__
// Dot-product accumulators.  FP64 compute accumulates in FP64.  FP32 compute accumulates a
// compensated pair of floats: each product is split exactly with an FMA and added with an
// error-free two-sum, the rounding errors collect in `lo`, and only the final pair is converted
// to FP64.  GB300 issues FP64 arithmetic and FP32<->FP64 conversions at 1/64 of the FP32 rate,
// so FP64 accumulation inside an FP32 kernel would bound it by the FP64 pipe.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.f, lo = 0.f;
  // (the _rn intrinsics keep the compiler from contracting these steps into FMAs)
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
  // error-free merge of another compensated pair
  __device__ __forceinline__ void merge(float ohi, float olo) {
    const float s = __fadd_rn(hi, ohi);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(ohi, bb));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, olo), e);
  }
};

// double-float operands (the FP64 operator in double-float arithmetic): each product split
// exactly (TwoProd plus cross terms), summed into a compensated float pair.
template <>
struct DotAcc<ff> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    float e;
    hi = two_sum(hi, p, e);
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ void merge(float ohi, float olo) {
    float e;
    hi = two_sum(hi, ohi, e);
    lo = __fadd_rn(__fadd_rn(lo, olo), e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Sum of an accumulator over the block, valid in thread 0 (fixed order).  FP32 pairs are merged
// through the warps and the block in FP32 and converted to FP64 once, in thread 0: an FP64
// instruction costs a warp ~64 scheduler cycles on GB300, which would dominate short work items.
// red: >= 32 doubles of shared memory.
__device__ __forceinline__ double block_total(const DotAcc<double>& a, double* red) {
  double v = a.s;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
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
__device__ __forceinline__ double block_total(const DotAcc<float>& a, double* red) {
  DotAcc<float> v = a;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ohi = __shfl_down_sync(0xffffffffu, v.hi, o);
    const float olo = __shfl_down_sync(0xffffffffu, v.lo, o);
    v.merge(ohi, olo);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float2* r2 = reinterpret_cast<float2*>(red);
  __syncthreads();
  if (lane == 0) r2[wid] = make_float2(v.hi, v.lo);
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    DotAcc<float> t;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t.merge(r2[i].x, r2[i].y);
    r = t.value();
  }
  return r;
}
__device__ __forceinline__ double block_total(const DotAcc<ff>& a, double* red) {
  DotAcc<float> f;
  f.hi = a.hi;
  f.lo = a.lo;
  return block_total(f, red);
}
#endif


enum { ST_RUNNING = -1 };

// Reduction slots in the partials buffer (each kMaxParts doubles).
constexpr int kMaxParts = 4096;
constexpr int kPartSlots = 8;

struct Tiling {
  int tx, ty, kc;            // node tile (tx x ty) and z-chunk kc
  int tiles_x, tiles_y, tiles_z;
  long long n_tiles;
  int threads;               // >= (tx+1)*(ty+1) rounded up to a warp, >= tx*ty
  int blocks;                // persistent grid (<= kMaxParts)
  size_t smem;               // dynamic shared memory bytes
};

struct Ctx;

// Device-side views used by kernel launchers.
struct Geo {
  int nx, ny, nz;
  long long N;
};

// ------------------------------------------------------------------------------------------
// Batched problems.  A "problem" is one RVE grid with one load case: its own vectors, its own
// solver state and per-item partial sums.  Every iteration kernel walks a flattened work list of
// (problem, tile) items (operator) or (problem, node chunk) items (vector kernels); a problem's
// result depends only on its own size and tiling, never on the other problems of the launch.
// A single solve is a batch of one problem.
// ------------------------------------------------------------------------------------------
constexpr int kVecThreads = 256;                    // block size of the vector kernels
constexpr int kVecPerThread = 4;                    // nodes per thread per work item
constexpr int kVecChunk = kVecThreads * kVecPerThread;  // nodes per vector-kernel work item
constexpr int kPartsSlots = 3;

struct Prob {
  int nx, ny, nz;
  long long N;
  int tx, ty, kc, tiles_x, tiles_y, n_tiles;  // operator tiling of this grid
  int n_chunks;                                // vector-kernel items
  int parts_stride;                            // >= max(n_tiles, n_chunks)
  long long item0_apply, item0_vec;            // first work item of this problem
  const int32_t* phase;
  const double* coef64;
  const float* coef32;
  const double* sig;      // per-phase sigma = C E of this load case (6 per phase)
  const void* minv;       // 6N Jacobi inverse planes (vector type)
  double* w;              // FP64 fluctuation (input of FP64 residuals, output)
  float* w_hi;            // mixed path: w as an unevaluated float pair
  float* w_lo;
  void* g;
  void* h;
  void* Ah;
  void* z;
  long long z_bytes;      // capacity of z; 0 keeps the FP64 operator on its recomputed-halo form
  double* parts;          // [kPartsSlots][parts_stride] per-item partial sums
  DevState* st;
};

// Launch description shared by the iteration kernels of one batch (device pointers).
struct BatchDev {
  const Prob* probs;
  const int* item_prob;    // apply item -> problem
  const int* vitem_prob;   // vector item -> problem
  const long long* counts; // [0] apply items, [1] vector items (read on the device)
  int apply_threads;       // block size of every operator launch (>= every tile's voxel count)
  size_t smem32, smem64;   // dynamic shared memory of FP32 / native FP64 operator launches
  size_t smemff;           // ... of double-float FP64 operator launches
  int blocks32, blocks64;  // persistent grids of FP32 / FP64 operator launches
  int vec_blocks, vec_threads;
  int nohalo64;            // native FP64 iteration operator without recomputed x/y halo (+ edge pass)
  int ff64;                // FP64 products in double-float arithmetic (ELAS_FP64_OP_PAIRED)
};

// apply.cu ---------------------------------------------------------------------------------
enum ApplyEpi { EPI_STORE = 0, EPI_STORE_DOT = 1, EPI_RESIDUAL = 2, EPI_NORM = 3 };
enum ApplyRole { ROLE_H = 0, ROLE_W = 1 };  // input h -> Ah, or input w (FP64) -> g / norms
// post actions of a problem's last item
enum { POST_NONE = 0, POST_LAMBDA = 1, POST_TRUE_NORM = 2, POST_REPLACE = 3 };
enum ApplyKind {
  AK_F64_DOT = 0,       // FP64 h -> Ah with h.Ah (FP64 iteration)
  AK_F32_DOT = 1,       // FP32 h -> Ah with h.Ah (mixed iteration)
  AK_F64_RESID = 2,     // FP64 w -> g, z (FP64 vectors): residual check of the FP64 path
  AK_MIX_RESID = 3,     // FP64 w -> g, z (FP32 vectors): residual replacement of the mixed path
  AK_F64_NORM = 4,      // ||A w + b||^2 only
  AK_F64_AFFINE = 5,    // g = A w + b stored (FP64)
};

size_t apply_smem_bytes(int tx, int ty, int elem_bytes);
size_t apply_smem_bytes_ff(int tx, int ty);
Tiling make_tiling(const Geo& g, int elem_bytes, int sm_count, int tx_hint = 0, int ty_hint = 0, int kc_hint = 0);
int apply_max_threads(int elem_bytes);
int apply_resident_blocks(int elem_bytes, int threads, size_t smem);
cudaError_t launch_apply(const BatchDev& b, int kind, int post, int gate, cudaStream_t s);
// Whether a problem's z can hold the tile-edge exports of the FP64 operator without halo.
bool apply_nohalo_fits(const Prob& p);

// other kernels (per grid, outside the iteration loop)
cudaError_t launch_jacobi(const Geo& g, const int32_t* phase, const double* coef64, double* minv64,
                          float* minv32, int sm_count, cudaStream_t s,
                          int mode = ELAS_PRECOND_BLOCK);
cudaError_t launch_rhs(const Geo& g, const int32_t* phase, const double* sig, double* b, int sm_count,
                       cudaStream_t s);
cudaError_t launch_stress(const Geo& g, const int32_t* phase, const double* cfull, const double* E6,
                          const double* w, double* stress, double* vm, double* parts, unsigned int* ctr,
                          double* macro_out, int sm_count, cudaStream_t s);

// pcg.cu -----------------------------------------------------------------------------------
struct SolveSetup {
  double tol, tol2_true, bscale2;
  double E[9];
  double drop2;
  int max_iter, stop_rule, replace_every, pad;
};
// per-problem setups (device array, one per problem)
// setups[k] initialises problem idx[k] (idx == nullptr: problem k) and marks it for k_pcg_init
cudaError_t launch_state_init(const BatchDev& b, const SolveSetup* setups, const int* idx, int n, cudaStream_t s);
cudaError_t launch_pcg_init(const BatchDev& b, bool mixed, cudaStream_t s);
cudaError_t launch_pcg_update(const BatchDev& b, bool mixed, cudaStream_t s);
cudaError_t launch_pcg_direction(const BatchDev& b, bool mixed, cudaStream_t s);
// w = w_hi + w_lo in FP64 (mixed path); gate: GATE_NONE, GATE_REPLACE or GATE_FINALIZE
cudaError_t launch_w_combine(const BatchDev& b, int gate, cudaStream_t s);

// hotspot.cu ---------------------------------------------------------------------------------
// Maximum-stress extraction of App. C.  Gaussian of standard deviation s (voxels) truncated at
// radius ceil(2 s) (the default filter size 2 ceil(2 s) + 1 of the paper's tool), at most 4.
constexpr int kHotMaxRadius = 4;
inline int hot_radius(double s) {
  int r = (int)std::ceil(2.0 * s);
  return r < 1 ? 1 : (r > kHotMaxRadius ? kHotMaxRadius : r);
}
inline void hot_weights(double s, int r, double* w) {
  double sum = 0.0;
  for (int x = -r; x <= r; ++x) {
    w[x + r] = std::exp(-(double)(x * x) / (2.0 * s * s));
    sum += w[x + r];
  }
  for (int x = -r; x <= r; ++x) w[x + r] /= sum;
}
// smooth (device N) written; best2[0]: bits of the largest hotspot value, best2[1]: its lowest
// voxel id (~0 if there is no hotspot); solid_only: pore neighbours do not compete.  Synchronises s.
cudaError_t launch_hotspot(const Geo& g, const int32_t* phase, const double* vm, double s_kernel, bool solid_only,
                           double* smooth, unsigned long long* best2, int sm_count, cudaStream_t s);

// generate.cu: records the message of a failed generator call (elas_generate_last_error)
int gen_error(int code, const std::string& m);

// host-side helpers (api.cu)
void bond_rotate(const double* C6_local, const double* rho, double* C6_global);

}  // namespace elas
