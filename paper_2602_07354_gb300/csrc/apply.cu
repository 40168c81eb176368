// Operator, preconditioner-build, right-hand-side and stress kernels (sm_103a).
//
// Matrix-free product y = A u of ELAS3D-Xtal (arXiv 2602.07354), Sec. 2.1.2 / Algorithm 2
// step A.  The paper evaluates it node by node as a 27-point stencil with 3x3 blocks gathered
// from the 8 surrounding element matrices.  Here every voxel's element product K_e u_e is
// computed once, voxel-centred, and its 8 corner forces are gathered per node from shared
// memory, marching along z through a tile of nodes:
//
//   * Exact modal split of K_e u_e.  With centred coordinates (xi, eta, zeta) in [-1/2,1/2]^3 the
//     trilinear field is u = A0 + A_x xi + A_y eta + A_z zeta + A_xy xi eta + A_yz eta zeta +
//     A_xz xi zeta + A_xyz xi eta zeta, whose coefficients are the Walsh-Hadamard transform of
//     the 8 corner values.  The displacement gradient splits into monomials {1, xi, eta, zeta,
//     eta zeta, xi zeta, xi eta} that are orthogonal on the voxel, so the element energy
//     int eps:C:eps (Eq. 7) is a sum of 7 independent quadratic forms with weights 1, 1/12 and
//     1/144.  The corner forces follow by the transposed transform.  This is the same K_e as
//     the 2x2x2 Gauss integral of B^T C B (exact for trilinear elements), at 432 instead of
//     1,152 flops per voxel (30 MUL + 108 FMA in the mode products, 186 adds).
//   * Per-phase coefficients are the sample-frame stiffness scaled by 1/16, 1/48 and 1/144
//     (the products of the transform scalings and mode weights), built on the host in FP64.
//   * Periodic wrap (Eq. 1) is applied when node layers are staged into shared memory.
//   * Node sums are gathered in a fixed order and block partial sums are combined in a fixed
//     order by the last block to finish, so every result is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "elas_internal.h"

namespace elas {

namespace {

// ---- deterministic block / grid reductions ------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order; result valid in thread 0.  red: >= 32 doubles of smem.
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

// Thread 0 publishes this block's partials, then the last block to arrive sees them all.
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

// Fixed-order total of one partial slot (called by every thread of the last block).
__device__ double total_of(const double* slot, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(slot + i);
  return block_sum(v, red);
}

// Ampere-style asynchronous global->shared element copies (cp.async), used to prefetch the
// periodically wrapped halo of the next node layer while the current one is computed.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_i32(void* smem, const int32_t* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
// element copy to a shared-memory address (4 or 8 bytes)
template <typename E>
__device__ __forceinline__ void cp_async_to(unsigned s, const E* gmem) {
  static_assert(sizeof(E) == 4 || sizeof(E) == 8, "4- or 8-byte elements");
  if (sizeof(E) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
// Node-layer ring of the operator: kRing slots, layers staged kAhead = kRing - 1 ahead; a thread
// waits for a layer's copies kAhead - 2 iterations after issuing them.
constexpr int kRing = 4, kAhead = kRing - 1;
__device__ __forceinline__ void cp_async_wait_ahead() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kAhead - 2) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int wrapi(int i, int n) {
  while (i < 0) i += n;
  while (i >= n) i -= n;
  return i;
}

// ---- modal element product ------------------------------------------------------------------
// The mode coefficients are the Walsh-Hadamard transform over the corner index
// a = ax + 2 ay + 4 az: W[m] = sum_a chi_m(a) u[a], chi_m(a) = product over the set bits d of m of
// s_d(a) = 2 a_d - 1.  It factors into an x, a y and a z stage; the kernel applies the x and y
// stages per face (4 corners) and the z stage per voxel, and the transposed stages in reverse.
// s = C e restricted to the Voigt slots in MASK (rows and columns); k: packed symmetric C.
template <int MASK, typename T>
__device__ __forceinline__ void symv(const T (&k)[24], const T (&e)[6], T (&s)[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (!((MASK >> i) & 1)) continue;
    T acc = T(0);
    bool first = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (!((MASK >> j) & 1)) continue;
      acc = first ? k[pk(i, j)] * e[j] : fma(k[pk(i, j)], e[j], acc);
      first = false;
    }
    s[i] = acc;
  }
}

// Double-float form: every row is a compensated dot product (Ogita-Rump-Oishi "Dot2" on pairs):
// each term's product is split exactly (TwoProd plus the two cross terms), the leading parts are
// summed with TwoSum and all error terms collect in one float, renormalised once per row.
// Coefficients of the double-float form read from the table (L1) at the point of use instead of
// being held in registers (the products' pairs and transforms already fill the register file).
struct LazyK {
  const ff* p;
  __device__ __forceinline__ ff operator[](int i) const {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p) + i);
    return ff(v.x, v.y);
  }
};
template <int MASK, typename KA>
__device__ __forceinline__ void symv_ff(const KA& k, const ff (&e)[6], ff (&s)[6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (!((MASK >> i) & 1)) continue;
    float hi = 0.f, lo = 0.f;
    bool first = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (!((MASK >> j) & 1)) continue;
      const ff a = k[pk(i, j)], b = e[j];
      const float p = __fmul_rn(a.hi, b.hi);
      float pe = fmaf(a.hi, b.hi, -p);
      pe = fmaf(a.hi, b.lo, pe);
      pe = fmaf(a.lo, b.hi, pe);
      if (first) {
        hi = p;
        lo = pe;
      } else {
        float t;
        hi = two_sum(hi, p, t);
        lo = __fadd_rn(lo, __fadd_rn(t, pe));
      }
      first = false;
    }
    s[i] = ff_norm(hi, lo);
  }
}
template <int MASK>
__device__ __forceinline__ void symv(const LazyK& k, const ff (&e)[6], ff (&s)[6]) {
  symv_ff<MASK>(k, e, s);
}

// 24 consecutive coefficients (16-byte aligned) through the read-only path as vectors.
__device__ __forceinline__ void load_k(const float* __restrict__ K, float (&k)[24]) {
  const float4* K4 = reinterpret_cast<const float4*>(K);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float4 v = __ldg(K4 + q);
    k[4 * q] = v.x; k[4 * q + 1] = v.y; k[4 * q + 2] = v.z; k[4 * q + 3] = v.w;
  }
}
__device__ __forceinline__ void load_k(const double* __restrict__ K, double (&k)[24]) {
  const double2* K2 = reinterpret_cast<const double2*>(K);
#pragma unroll
  for (int q = 0; q < 12; ++q) {
    const double2 v = __ldg(K2 + q);
    k[2 * q] = v.x; k[2 * q + 1] = v.y;
  }
}


// Where the operator's per-phase coefficient blocks live for each arithmetic: the FP64 table, the
// FP32 copy, or the float-pair copy inside the FP32 table (strides and offsets in elements).
template <typename T>
struct CoefOf;
template <>
struct CoefOf<double> {
  static constexpr int stride = kCoefStride, base = 0, m1 = kCoefMode1, m2 = kCoefMode2;
  static __device__ __forceinline__ const double* table(const Prob& P) { return P.coef64; }
};
template <>
struct CoefOf<float> {
  static constexpr int stride = kCoef32Stride, base = 0, m1 = kCoefMode1, m2 = kCoefMode2;
  static __device__ __forceinline__ const float* table(const Prob& P) { return P.coef32; }
};
template <>
struct CoefOf<ff> {
  static constexpr int stride = kCoef32Stride / 2, base = kCoefFF / 2, m1 = kCoefFFBlock / 2, m2 = kCoefFFBlock;
  static __device__ __forceinline__ const ff* table(const Prob& P) { return reinterpret_cast<const ff*>(P.coef32); }
};

// ---- the x and y components as one packed lane pair --------------------------------------------
// The transforms treat the three displacement components alike; the x and y components travel as
// one pair, operated on with the packed FP32 instructions of sm_100+ (add/sub.rn.f32x2: two IEEE
// operations per lane and instruction), the z component alone.  FP64 pairs are two scalars.
template <typename T>
struct P2;
template <>
struct P2<float> {
  float2 v;
};
template <>
struct P2<double> {
  double x, y;
};
template <>
struct P2<ff> {
  float2 hi, lo;  // (x.hi, y.hi), (x.lo, y.lo)
};
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<const float2*>(&r);
}
__device__ __forceinline__ P2<float> operator+(P2<float> a, P2<float> b) { return {add2(a.v, b.v)}; }
__device__ __forceinline__ P2<float> operator-(P2<float> a, P2<float> b) { return {sub2(a.v, b.v)}; }
__device__ __forceinline__ P2<double> operator+(P2<double> a, P2<double> b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ P2<double> operator-(P2<double> a, P2<double> b) { return {a.x - b.x, a.y - b.y}; }
// two double-float sums at once: TwoSum of the leading parts, trailing parts and error in FP32
__device__ __forceinline__ P2<ff> operator+(P2<ff> a, P2<ff> b) {
  const float2 s = add2(a.hi, b.hi);
  const float2 bb = sub2(s, a.hi);
  const float2 e = add2(sub2(a.hi, sub2(s, bb)), sub2(b.hi, bb));
  return {s, add2(add2(a.lo, b.lo), e)};
}
__device__ __forceinline__ P2<ff> operator-(P2<ff> a, P2<ff> b) {
  return a + P2<ff>{make_float2(-b.hi.x, -b.hi.y), make_float2(-b.lo.x, -b.lo.y)};
}
__device__ __forceinline__ P2<float> pk2(float x, float y) { return {make_float2(x, y)}; }
__device__ __forceinline__ P2<double> pk2(double x, double y) { return {x, y}; }
__device__ __forceinline__ P2<ff> pk2(ff x, ff y) { return {make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)}; }
__device__ __forceinline__ float lane0(P2<float> a) { return a.v.x; }
__device__ __forceinline__ float lane1(P2<float> a) { return a.v.y; }
__device__ __forceinline__ double lane0(P2<double> a) { return a.x; }
__device__ __forceinline__ double lane1(P2<double> a) { return a.y; }
__device__ __forceinline__ ff lane0(P2<ff> a) { return ff(a.hi.x, a.lo.x); }
__device__ __forceinline__ ff lane1(P2<ff> a) { return ff(a.hi.y, a.lo.y); }

// (x, y, z, 4th) shared-memory records: float [x y z id], double [x y | z id], double-float
// [x.hi y.hi x.lo y.lo | z.hi z.lo id -]; the 4th element holds a phase id in the node ring
__device__ __forceinline__ void ld_xyz(const float* p, P2<float>& xy, float& z) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  xy.v = make_float2(v.x, v.y);
  z = v.z;
}
__device__ __forceinline__ void ld_xyz(const double* p, P2<double>& xy, double& z) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  xy = {a.x, a.y};
  z = p[2];
}
__device__ __forceinline__ void ld_xyz(const ff* p, P2<ff>& xy, ff& z) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float2 b = *reinterpret_cast<const float2*>(p + 2);
  xy = {make_float2(a.x, a.y), make_float2(a.z, a.w)};
  z = ff(b.x, b.y);
}
__device__ __forceinline__ void st_xyz(float* p, P2<float> xy, float z) {
  *reinterpret_cast<float4*>(p) = make_float4(xy.v.x, xy.v.y, z, 0.f);
}
__device__ __forceinline__ void st_xyz(double* p, P2<double> xy, double z) {
  *reinterpret_cast<double2*>(p) = make_double2(xy.x, xy.y);
  p[2] = z;
}
__device__ __forceinline__ void st_xyz(ff* p, P2<ff> xy, ff z) {
  *reinterpret_cast<float4*>(p) = make_float4(xy.hi.x, xy.hi.y, xy.lo.x, xy.lo.y);
  *reinterpret_cast<float2*>(p + 2) = make_float2(z.hi, z.lo);
}

// the butterflies of one face: corners b = ax + 2 ay -> face modes q = mx + 2 my (any lane type)
template <typename L>
__device__ __forceinline__ void face_bf(const L& c0, const L& c1, const L& c2, const L& c3, L (&V)[4]) {
  const L s01 = c0 + c1, d01 = c1 - c0;
  const L s23 = c2 + c3, d23 = c3 - c2;
  V[0] = s01 + s23;
  V[1] = d01 + d23;
  V[2] = s23 - s01;
  V[3] = d23 - d01;
}
// the transposed butterflies: face modes m -> corners (a0 = m0 - m1, ...)
template <typename L>
__device__ __forceinline__ void face_bf_t(const L (&m)[4], L (&cor)[4]) {
  const L a0 = m[0] - m[1], a1 = m[0] + m[1], a2 = m[2] - m[3], a3 = m[2] + m[3];
  cor[0] = a0 - a2;
  cor[2] = a0 + a2;
  cor[1] = a1 - a3;
  cor[3] = a1 + a3;
}

// Forward transform of one face (4 corners b = ax + 2 ay) into face modes q = mx + 2 my, the x and
// y components as a pair.  face: the record of corner 0; row: elements per record row; RS: elements
// per node record of the ring.
template <int RS, typename T>
__device__ __forceinline__ void face_forward(const T* face, int row, P2<T> (&Vxy)[4], T (&Vz)[4]) {
  P2<T> cxy[4];
  T cz[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) ld_xyz(face + (b >> 1) * row + RS * (b & 1), cxy[b], cz[b]);
  face_bf(cxy[0], cxy[1], cxy[2], cxy[3], Vxy);
  face_bf(cz[0], cz[1], cz[2], cz[3], Vz);
}

// Modal element forces F[c][m] (m = 1..7; F[c][0] = 0) from the mode coefficients W[c][m]:
// seven orthogonal gradient monomials, each a symmetric-stiffness product (see file header).
// k0 holds the C/16 block (already loaded).  FP64 reads the C/48 and C/144 blocks as well; FP32
// instead scales the linear-mode coefficients by 1/3 and the trilinear one by 1/9 and uses C/16
// for all seven products (C/48 e = C/16 (e/3)), which trades 12 multiplies for 12 of the 18
// vector loads of the coefficient blocks.
template <typename T, typename K0>
__device__ __forceinline__ void modal_forces(T (&W)[3][8], const K0& k0, const T* __restrict__ K,
                                             T (&F)[3][8]) {
  constexpr bool f32 = sizeof(T) == 4;
  constexpr bool lazy = std::is_same<K0, LazyK>::value;
  T s[6];
  const K0& k = k0;
  {  // constant-strain mode: gradient columns are the linear coefficients (modes 1, 2, 4)
    const T e[6] = {W[0][1], W[1][2], W[2][4], W[1][4] + W[2][2], W[0][4] + W[2][1], W[0][2] + W[1][1]};
    symv<0x3f>(k, e, s);
    F[0][1] = s[0]; F[1][1] = s[5]; F[2][1] = s[4];
    F[0][2] = s[5]; F[1][2] = s[1]; F[2][2] = s[3];
    F[0][4] = s[4]; F[1][4] = s[3]; F[2][4] = s[2];
  }
  auto linear_modes = [&](const auto& k1) {
    {  // mode xi: gradient [0 | A_xy | A_xz]
      const T e[6] = {T(0), W[1][3], W[2][5], W[2][3] + W[1][5], W[0][5], W[0][3]};
      symv<0x3e>(k1, e, s);
      F[0][3] = s[5]; F[1][3] = s[1]; F[2][3] = s[3];
      F[0][5] = s[4]; F[1][5] = s[3]; F[2][5] = s[2];
    }
    {  // mode eta: gradient [A_xy | 0 | A_yz]
      const T e[6] = {W[0][3], T(0), W[2][6], W[1][6], W[0][6] + W[2][3], W[1][3]};
      symv<0x3d>(k1, e, s);
      F[0][3] += s[0]; F[1][3] += s[5]; F[2][3] += s[4];
      F[0][6] = s[4]; F[1][6] = s[3]; F[2][6] = s[2];
    }
    {  // mode zeta: gradient [A_xz | A_yz | 0]
      const T e[6] = {W[0][5], W[1][6], T(0), W[2][6], W[2][5], W[0][6] + W[1][5]};
      symv<0x3b>(k1, e, s);
      F[0][5] += s[0]; F[1][5] += s[5]; F[2][5] += s[4];
      F[0][6] += s[5]; F[1][6] += s[1]; F[2][6] += s[3];
    }
  };
  // bilinear modes: eta zeta -> [A_xyz|0|0], xi zeta -> [0|A_xyz|0], xi eta -> [0|0|A_xyz]
  auto bilinear_modes = [&](const auto& k2) {
    {
      const T e[6] = {W[0][7], T(0), T(0), T(0), W[2][7], W[1][7]};
      symv<0x31>(k2, e, s);
      F[0][7] = s[0]; F[1][7] = s[5]; F[2][7] = s[4];
    }
    {
      const T e[6] = {T(0), W[1][7], T(0), W[2][7], T(0), W[0][7]};
      symv<0x2a>(k2, e, s);
      F[0][7] += s[5]; F[1][7] += s[1]; F[2][7] += s[3];
    }
    {
      const T e[6] = {T(0), T(0), W[2][7], W[1][7], W[0][7], T(0)};
      symv<0x1c>(k2, e, s);
      F[0][7] += s[4]; F[1][7] += s[3]; F[2][7] += s[2];
    }
  };
  if constexpr (f32) {
    const T third = T(1.0 / 3.0), ninth = T(1.0 / 9.0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      W[c][3] *= third;
      W[c][5] *= third;
      W[c][6] *= third;
      W[c][7] *= ninth;
    }
    linear_modes(k0);
    bilinear_modes(k0);
  } else if constexpr (lazy) {
    linear_modes(LazyK{K + CoefOf<T>::m1});
    bilinear_modes(LazyK{K + CoefOf<T>::m2});
  } else {
    T kb[24];
    load_k(K + CoefOf<T>::m1, kb);
    linear_modes(kb);
    load_k(K + CoefOf<T>::m2, kb);
    bilinear_modes(kb);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) F[c][0] = T(0);
}

// ---- the tile kernel --------------------------------------------------------------------------
// elements of one face-force buffer: 4 corners x NV columns x 4-wide records
__host__ __device__ constexpr int fbuf_elems(int NV) { return 4 * NV * 4; }
// Double-float face-force records, compact: record r (= buffer x 4 NV + corner x NV + column) keeps
// its x and y pairs (x.hi, y.hi, x.lo, y.lo) at pair offset 2 r and its z pair at 16 NV + r (both
// buffers' xy parts first), 24 bytes a record instead of a padded 32.
__device__ __forceinline__ void st_face_ff(ff* Fc, int NV, int r, const P2<ff>& xy, ff z) {
  *reinterpret_cast<float4*>(Fc + 2 * r) = make_float4(xy.hi.x, xy.hi.y, xy.lo.x, xy.lo.y);
  *reinterpret_cast<float2*>(Fc + 16 * NV + r) = make_float2(z.hi, z.lo);
}
__device__ __forceinline__ void ld_face_ff(const ff* Fc, int NV, int r, P2<ff>& xy, ff& z) {
  const float4 a = *reinterpret_cast<const float4*>(Fc + 2 * r);
  const float2 b = *reinterpret_cast<const float2*>(Fc + 16 * NV + r);
  xy = {make_float2(a.x, a.y), make_float2(a.z, a.w)};
  z = ff(b.x, b.y);
}
// the same helpers for the other forms are never called (their records stay 4-wide)
template <typename T, typename P>
__device__ __forceinline__ void st_face_ff(T*, int, int, const P&, T) {}
template <typename T, typename P>
__device__ __forceinline__ void ld_face_ff(const T*, int, int, P&, T&) {}

__device__ __forceinline__ bool gate_skips(int gate, const DevState* st) {
  if (gate == GATE_RUNNING) return st->done || st->want_check;
  if (gate == GATE_REPLACE)
    return st->done || !replacement_due(st);
  if (gate == GATE_FINALIZE) return !st->done || st->finalized;
  return false;
}

// Voigt slot order of the 6 stored symmetric inverse entries: 11, 22, 33, 23, 13, 12.
template <typename Tv>
__device__ __forceinline__ void block_jacobi_apply(const Tv* __restrict__ minv, long long N, long long n,
                                                   const Tv (&g)[3], Tv (&z)[3]) {
  const Tv m11 = minv[n], m22 = minv[N + n], m33 = minv[2 * N + n];
  const Tv m23 = minv[3 * N + n], m13 = minv[4 * N + n], m12 = minv[5 * N + n];
  z[0] = m11 * g[0] + m12 * g[1] + m13 * g[2];
  z[1] = m12 * g[0] + m22 * g[1] + m23 * g[2];
  z[2] = m13 * g[0] + m23 * g[1] + m33 * g[2];
}

// The scalar step a problem's last item performs on the problem's totals (s0: h.Ah or z.g, s1: r.r).
__device__ void post_scalars(DevState* st, int post, double s0, double s1) {
  if (post == POST_LAMBDA) {  // Algorithm 2 step B
    st->hAh = s0;
    if (st->iter == 0) st->hAh_first = s0;
    if (!isfinite(s0)) {
      st->status = ELAS_NONFINITE;
      st->done = 1;
    } else if (!(s0 > 0.0)) {
      st->status = ELAS_BREAKDOWN;
      st->done = 1;
    } else {
      st->lambda = st->gg / s0;
      st->lam_hi = (float)st->lambda;
      st->lam_lo = (float)(st->lambda - (double)st->lam_hi);
    }
  } else if (post == POST_TRUE_NORM) {
    st->rr_true = s1;
    st->finalized = 1;
  } else if (post == POST_REPLACE) {
    // the FP64 true residual replaces the recursive one; convergence is decided on it
    st->rr_true = s1;
    st->rr = s1;
    st->rr_repl = s1;
    st->n_repl += 1;
    const double gg_new = s0;
    const bool conv = (st->stop_rule == ELAS_STOP_TRUE) ? (s1 <= st->tol2_true * st->bb)
                                                         : (gg_new < st->tol * st->tol * st->gg0);
    if (!isfinite(s1) || !isfinite(gg_new)) {
      st->status = ELAS_NONFINITE;
      st->done = 1;
    } else if (conv) {
      st->status = ELAS_CONVERGED;
      st->done = 1;
    } else if (st->iter >= st->max_iter) {
      st->status = ELAS_MAX_ITER;
      st->done = 1;
    }
    st->gg = gg_new;
    st->gamma = gg_new / st->gg_last;
    st->gam_f = (float)st->gamma;
    st->want_check = 0;
    st->last_repl_iter = st->iter;
  }
}

// Persistent operator kernel over (problem, tile) items.  For one item the CTA owns a tx x ty
// node tile and a chunk of kc node layers of its problem.  Thread t < (tx+1)(ty+1) owns voxel
// column (vi, vj) of the tile (global voxel i0-1+vi, j0-1+vj) and marches it along z, keeping
// in registers the modes of its lower face and the forces its previous voxel left on the shared
// face (the double-float form keeps those forces in a per-thread shared-memory slot); thread
// t < tx*ty owns node (ni, nj).  Shared memory: a 4-slot ring of node layers ((tx+2)(ty+2)
// records of x, y, z and the phase id of the voxel whose low corner is that node) filled by
// cp.async three layers ahead, so neither the node values nor the phase ids of a layer are waited
// for in the layer that uses them, and two buffers of per-column face corner forces
// ([corner][column] records).  One barrier per layer.  Each item publishes its own partial sums;
// the problem's last item sums them in tile order.
template <typename Tin, typename T, typename Tvec, int EPI, bool AFFINE, int MAXT, int MINB, bool NOHALO = false>
__global__ void __launch_bounds__(MAXT, MINB)
    k_apply(const Prob* __restrict__ probs, const int* __restrict__ item_prob, const long long* __restrict__ counts,
            int role, int post, int gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  __shared__ int s_last;
  static_assert(sizeof(Tin) == sizeof(T), "node layers are staged in the input's size");
  // double-float arithmetic: node layers arrive as doubles and are split into pairs in place
  constexpr bool kFF = std::is_same<T, ff>::value;
  using Tst = typename std::conditional<kFF, double, T>::type;  // type of the stored products
  const int t = threadIdx.x;
  const long long n_items = counts[0];

  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Prob& P = probs[item_prob[item]];
    if (gate != GATE_NONE && gate_skips(gate, P.st)) continue;  // uniform over the block
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long N = P.N;
    const int tx = P.tx, ty = P.ty;
    const int NXv = tx + 1, NV = (tx + 1) * (ty + 1);
    const int NXp = tx + 2, NP = (tx + 2) * (ty + 2);
    constexpr int RS = 4;                       // elements per node record
    T* ring = reinterpret_cast<T*>(smem_raw);  // [kRing][NP][RS]
    T* Fc = ring + kRing * NP * RS;             // [2][4 corners][NV][4] (double-float: compact, below)
    const long long plane = (long long)nx * ny;
    const int32_t* __restrict__ phase = P.phase;
    const T* __restrict__ coef = CoefOf<T>::table(P) + CoefOf<T>::base;
    const Tin* __restrict__ u = role == ROLE_W ? reinterpret_cast<const Tin*>(P.w) : reinterpret_cast<const Tin*>(P.h);
    Tst* __restrict__ y = role == ROLE_W ? reinterpret_cast<Tst*>(P.g) : reinterpret_cast<Tst*>(P.Ah);
    Tvec* __restrict__ g_v = reinterpret_cast<Tvec*>(P.g);
    Tvec* __restrict__ z_v = reinterpret_cast<Tvec*>(P.z);
    const Tvec* __restrict__ minv_v = reinterpret_cast<const Tvec*>(P.minv);
    T E4[3][3];
    if (AFFINE) {
#pragma unroll
      for (int q = 0; q < 9; ++q) E4[q / 3][q % 3] = (T)(4.0 * P.st->E[q]);
    }
    DotAcc<T> dot0;       // h.Ah (the product's own precision, compensated in FP32)
    DotAcc<double> dot1;  // r.r of the FP64 residual variants
    DotAcc<double> dot0r; // z.g of the residual replacement
    const int ni = t % tx, nj = t / tx;
    // voxel column of this thread; NOHALO puts the tile's own columns (1..tx x 1..ty) on the
    // first threads and the halo columns (row 0, then column 0) on the last ones, so that whole
    // warps of halo columns skip the element product
    int vi, vj;
    if (!NOHALO) {
      vi = t % NXv;
      vj = t / NXv;
    } else if (t < tx * ty) {
      vi = 1 + t % tx;
      vj = 1 + t / tx;
    } else {
      const int hh = t - tx * ty;
      vi = hh <= tx ? hh : 0;
      vj = hh <= tx ? 0 : hh - tx;
    }
    const int vcol = vi + NXv * vj;  // the column's slot in the face-force buffer

    const int tile = (int)(item - P.item0_apply);
    const int bx = tile % P.tiles_x;
    const int by = (tile / P.tiles_x) % P.tiles_y;
    const int bz = tile / (P.tiles_x * P.tiles_y);
    const int i0 = bx * tx, j0 = by * ty, k0 = bz * P.kc;
    const int k1 = min(k0 + P.kc, nz);

    const bool has_vox = t < NV;
    // nodes of this tile inside the grid (NOHALO: its own voxel columns are 1..rx x 1..ry)
    const int rx = min(tx, nx - i0), ry = min(ty, ny - j0);
    const int kbase = k0;  // (the voxel block's coefficient array is also called k0)
    const bool has_node = (t < tx * ty) && (i0 + ni < nx) && (j0 + nj < ny);
    const long long node_xy = has_node ? (long long)(j0 + nj) * nx + (i0 + ni) : 0;

    // this thread's staging records of the node layer (at most 3, since blockDim >= (tx+1)(ty+1)):
    // their periodically wrapped in-plane offsets and the shared-memory addresses of the records in
    // ring slot 0, fixed for the whole tile
    int soff[3];
    unsigned srec[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int sl = t + r * (int)blockDim.x;
      soff[r] = sl < NP ? wrapi(j0 - 1 + sl / NXp, ny) * nx + wrapi(i0 - 1 + sl % NXp, nx) : -1;
      srec[r] = (unsigned)__cvta_generic_to_shared(ring + RS * (sl < NP ? sl : 0));
    }
    const unsigned slot_bytes = (unsigned)(NP * RS * sizeof(T));
    const Tin* __restrict__ u1 = u + N;
    const Tin* __restrict__ u2 = u + 2 * N;
    // the layers are staged in order from k0 - 1: the offset of the next one, wrapped periodically
    int kofs_next = (k0 == 0 ? nz - 1 : k0 - 1) * (int)plane;
    // asynchronous copy of the next node layer and of the phase ids of the voxels above it into
    // ring slot b (the id goes to the record's fourth element)
    auto stage = [&](int b) {
      const int kofs = kofs_next;
      const unsigned sb = (unsigned)b * slot_bytes;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        if (soff[r] < 0) break;
        const int e = kofs + soff[r];
        const unsigned d = srec[r] + sb;
        cp_async_to(d, u + e);
        cp_async_to(d + sizeof(T), u1 + e);
        cp_async_to(d + 2 * sizeof(T), u2 + e);
        cp_async_to(d + 3 * sizeof(T), phase + e);
      }
      cp_async_commit();
      kofs_next = kofs + (int)plane < (int)N ? kofs + (int)plane : kofs + (int)plane - (int)N;
    };
    // per-thread shared-memory offsets fixed for the tile: the voxel column's lower face corner
    // record in a ring slot, the owned node's record, the column's slots in a face-force buffer and
    // the 4 records the owned node gathers
    const T* const face0 = ring + RS * (vj * NXp + vi);
    const int row = RS * NXp, slot_elems = NP * RS, fbuf = 4 * NV * 4;
    const T* const hrec0 = ring + RS * ((nj + 1) * NXp + ni + 1);
    T* const fcol = Fc + 4 * vcol;
    int goff[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) goff[b] = 4 * (b * NV + (ni + 1 - (b & 1)) + NXv * (nj + 1 - (b >> 1)));
    // linear index of the owned node on the layer the next gather writes (layer kv - 1; the first
    // gather, at kv = k0 + 1, writes layer k0)
    int nrow = k0 * (int)plane + (int)node_xy;
    // double-float form: once this thread's own copies of ring slot b have landed, split its node
    // records' doubles into float pairs in place (before the barrier that publishes the slot)
    auto split_slot = [&](int b) {
      if constexpr (kFF) {
        T* dst = ring + b * NP * RS;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          if (soff[r] < 0) break;
          T* rec = dst + RS * (t + r * (int)blockDim.x);
          const double* d = reinterpret_cast<const double*>(rec);
          const double v0 = d[0], v1 = d[1], v2 = d[2];
          asm volatile("" ::: "memory");  // the pairs overwrite the doubles they are made from
          st_xyz(rec, pk2(T(v0), T(v1)), T(v2));
        }
      }
    };

    P2<T> Vlo_xy[4], FUp_xy[4];  // modes of the lower face, forces the previous voxel left on it
    T Vlo_z[4], FUp_z[4];
    // double-float form: the forces the previous voxel left on the lower face wait in a per-thread
    // shared-memory slot (6 float4 planes after the face-force buffers, conflict-free) instead of
    // 24 registers, which this form's products need
    float4* const fup = reinterpret_cast<float4*>(Fc + (kFF ? 24 * NV : 2 * fbuf_elems(NV))) + t;
    const int fup_plane = (int)blockDim.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      FUp_xy[q] = pk2(T(0), T(0));
      FUp_z[q] = T(0);
    }
    if constexpr (kFF) {
#pragma unroll
      for (int e = 0; e < 6; ++e) fup[e * fup_plane] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // Node layers are staged kAhead ahead into the kRing-slot ring.  Iteration kv: one barrier
    // publishes node layer kv+1 and the corner forces of node layer kv-1 (written in iteration
    // kv-1); after it every thread has left iteration kv-1, so the slot of layer kv-1 takes layer
    // kv+kAhead, and each thread waits for its own copies of layer kv+2 (issued kAhead-2 iterations
    // earlier) and, in the double-float form, splits them into pairs off the barrier's path (the
    // next barrier publishes them).  Then layer kv-1 is gathered and voxel layer kv computed.  Face
    // forces are double-buffered by layer parity.
#pragma unroll
    for (int a = 0; a < kAhead; ++a) {
      if (k0 - 1 + a <= k1)
        stage(a);
      else
        cp_async_commit();
    }
    cp_async_wait_ahead();  // layers k0-1 and k0 have landed
    if (kFF) {
      split_slot(0);
      split_slot(1);
    }
    // NOHALO: only the tile's own voxel columns take the element product; the others (halo row and
    // column, columns beyond a ragged tile's edge) would put zero forces on their faces in every
    // layer, so their face-force records are zeroed once here and their threads skip the z-march
    // (published by the loop's first barrier; the previous item's gathers ended at its last one)
    const bool own_col = !NOHALO || (vi >= 1 && vj >= 1 && vi <= rx && vj <= ry);
    if (NOHALO && has_vox && !own_col) {
      const P2<T> zxy = pk2(T(0), T(0));
#pragma unroll
      for (int buf = 0; buf < 2; ++buf)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if constexpr (kFF)
            st_face_ff(Fc, NV, buf * 4 * NV + b * NV + vcol, zxy, T(0));
          else
            st_xyz(fcol + buf * fbuf + b * 4 * NV, zxy, T(0));
        }
    }
    T hown[3] = {T(0), T(0), T(0)};  // the owned node's operand on the previous layer (h.Ah)
    for (int kv = k0 - 1; kv <= k1; ++kv) {
      const int L = kv - k0 + 1;
      __syncthreads();
      if (kv + kAhead <= k1)
        stage((L + kAhead) % kRing);  // prefetch layer kv + kAhead: overlaps the next layers' arithmetic
      else
        cp_async_commit();
      cp_async_wait_ahead();  // this thread's copies of layer kv+2 have landed
      if (kFF && kv + 2 <= k1) split_slot((L + 2) % kRing);
      if (kv > k0 && has_node) {
        // node (ni,nj) of layer kv-1 is corner 3 of column (ni,nj), 2 of (ni+1,nj), 1 of
        // (ni,nj+1) and 0 of (ni+1,nj+1)
        const T* fp = Fc + ((kv - 1) & 1) * fbuf;
        P2<T> oxy = pk2(T(0), T(0));
        T oz = T(0);
#pragma unroll
        for (int b = 3; b >= 0; --b) {
          P2<T> xy;
          T z;
          if constexpr (kFF) {
            ld_face_ff(Fc, NV, ((kv - 1) & 1) * 4 * NV + goff[b] / 4, xy, z);
          } else {
            ld_xyz(fp + goff[b], xy, z);
          }
          oxy = oxy + xy;
          oz = oz + z;
        }
        const T out[3] = {lane0(oxy), lane1(oxy), oz};
        const long long n = nrow;
        if (EPI == EPI_STORE || EPI == EPI_STORE_DOT) {
#pragma unroll
          for (int c = 0; c < 3; ++c) y[c * N + n] = (Tst)out[c];
          if (EPI == EPI_STORE_DOT && (!NOHALO || (ni >= 1 && nj >= 1))) {
            dot0.add(hown[0], out[0]);
            dot0.add(hown[1], out[1]);
            dot0.add(hown[2], out[2]);
          }
        } else if (EPI == EPI_RESIDUAL) {
          Tvec gv[3], zv[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            gv[c] = (Tvec)out[c];
            dot1.add((double)out[c], (double)out[c]);
          }
          block_jacobi_apply(minv_v, N, n, gv, zv);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            g_v[c * N + n] = gv[c];
            z_v[c * N + n] = zv[c];
            dot0r.add((double)zv[c], (double)gv[c]);
          }
        } else {  // EPI_NORM
#pragma unroll
          for (int c = 0; c < 3; ++c) dot1.add((double)out[c], (double)out[c]);
        }
      }
      if (kv < k1 && has_vox && own_col) {
        const bool own = own_col;
        if (L == 0) face_forward<RS>(face0, row, Vlo_xy, Vlo_z);
        P2<T> Vup_xy[4];
        T Vup_z[4];
        face_forward<RS>(face0 + ((L + 1) % kRing) * slot_elems, row, Vup_xy, Vup_z);
        P2<T> FL_xy[4], FU_xy[4];
        T FL_z[4], FU_z[4];
        const int ph = own ? *reinterpret_cast<const int*>(face0 + (L % kRing) * slot_elems + 3) : -1;
        const T* K = ph >= 0 ? coef + (long long)ph * CoefOf<T>::stride : nullptr;
        T k0[24];
        bool solid = false;
        if (K != nullptr) {
          if constexpr (kFF) {
            solid = __ldg(reinterpret_cast<const float*>(K + kCoefSolid0)) != 0.f;
          } else {
            load_k(K + kCoefMode0, k0);
            solid = k0[kCoefSolid0] != T(0);
          }
        }
        if (solid) {
          // z stage of the forward transform (x and y components paired)
          P2<T> Wxy[8];
          T Wz[8];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            Wxy[q] = Vlo_xy[q] + Vup_xy[q];
            Wxy[q + 4] = Vup_xy[q] - Vlo_xy[q];
            Wz[q] = Vlo_z[q] + Vup_z[q];
            Wz[q + 4] = Vup_z[q] - Vlo_z[q];
          }
          T W[3][8], F[3][8];
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            W[0][m] = lane0(Wxy[m]);
            W[1][m] = lane1(Wxy[m]);
            W[2][m] = Wz[m];
          }
          if (AFFINE) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              W[c][1] += E4[c][0];
              W[c][2] += E4[c][1];
              W[c][4] += E4[c][2];
            }
          }
          if constexpr (kFF)
            modal_forces(W, LazyK{K + kCoefMode0}, K, F);
          else
            modal_forces(W, k0, K, F);
          // transposed z stage: forces on the lower (this node layer) and upper face
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const P2<T> a = pk2(F[0][q], F[1][q]), b = pk2(F[0][q + 4], F[1][q + 4]);
            FL_xy[q] = a - b;
            FU_xy[q] = a + b;
            FL_z[q] = F[2][q] - F[2][q + 4];
            FU_z[q] = F[2][q] + F[2][q + 4];
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            FL_xy[q] = FU_xy[q] = pk2(T(0), T(0));
            FL_z[q] = FU_z[q] = T(0);
          }
        }
        // face of node layer kv: lower-face forces of this voxel + upper-face forces of the one below,
        // back-transformed to the 4 corners (transposed x and y stages)
        P2<T> m_xy[4], cor_xy[4];
        T m_z[4], cor_z[4];
        if constexpr (kFF) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 a = fup[q * fup_plane];
            FUp_xy[q] = P2<T>{make_float2(a.x, a.y), make_float2(a.z, a.w)};
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float4 a = fup[(4 + h) * fup_plane];
            FUp_z[2 * h] = ff(a.x, a.y);
            FUp_z[2 * h + 1] = ff(a.z, a.w);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          m_xy[q] = FUp_xy[q] + FL_xy[q];
          m_z[q] = FUp_z[q] + FL_z[q];
        }
        face_bf_t(m_xy, cor_xy);
        face_bf_t(m_z, cor_z);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if constexpr (kFF)
            st_face_ff(Fc, NV, (kv & 1) * 4 * NV + b * NV + vcol, cor_xy[b], cor_z[b]);
          else
            st_xyz(fcol + (kv & 1) * fbuf + b * 4 * NV, cor_xy[b], cor_z[b]);
        }
        if (NOHALO && own && kv >= kbase && (vi == rx || vj == ry)) {
          // the tile's last voxel column and row also act on the nodes just beyond the tile: their
          // corners with a_x = 1 (column) and a_y = 1 (row) go to the edge pass, per node layer
          Tst* ex = reinterpret_cast<Tst*>(P.z) + 6 * ((long long)tile * P.kc + (kv - kbase)) * (tx + ty);
          auto put = [&](Tst* d, int b) {
            d[0] = (Tst)lane0(cor_xy[b]); d[1] = (Tst)lane1(cor_xy[b]); d[2] = (Tst)cor_z[b];
          };
          if (vi == rx) {
            Tst* d = ex + 6 * (vj - 1);
            put(d, 1);
            put(d + 3, 3);
          }
          if (vj == ry) {
            Tst* d = ex + 6 * (ty + vi - 1);
            put(d, 2);
            put(d + 3, 3);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Vlo_xy[q] = Vup_xy[q];
          Vlo_z[q] = Vup_z[q];
        }
        if constexpr (kFF) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            fup[q * fup_plane] = make_float4(FU_xy[q].hi.x, FU_xy[q].hi.y, FU_xy[q].lo.x, FU_xy[q].lo.y);
#pragma unroll
          for (int h = 0; h < 2; ++h)
            fup[(4 + h) * fup_plane] =
                make_float4(FU_z[2 * h].hi, FU_z[2 * h].lo, FU_z[2 * h + 1].hi, FU_z[2 * h + 1].lo);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            FUp_xy[q] = FU_xy[q];
            FUp_z[q] = FU_z[q];
          }
        }
      }
      if (EPI == EPI_STORE_DOT && kv < k1 && has_node) {
        P2<T> hxy;
        ld_xyz(hrec0 + (L % kRing) * slot_elems, hxy, hown[2]);
        hown[0] = lane0(hxy);
        hown[1] = lane1(hxy);
      }
      if (kv > k0) nrow += (int)plane;
    }
    cp_async_wait_all();
    __syncthreads();

    if (NOHALO) {
      // interior nodes' h.Ah; the edge pass adds the tile-edge nodes and takes the scalar step
      const double b0 = block_total(dot0, red);
      if (t == 0) P.parts[tile] = b0;
      __syncthreads();
    } else if (EPI != EPI_STORE) {
      const double b0 = EPI == EPI_RESIDUAL ? block_total(dot0r, red) : block_total(dot0, red);
      const double b1 = block_total(dot1, red);
      if (t == 0) {
        P.parts[tile] = b0;
        P.parts[P.parts_stride + tile] = b1;
        __threadfence();
        s_last = atomicAdd(&P.st->ctr[0], 1u) == (unsigned)(P.n_tiles - 1);
      }
      __syncthreads();
      if (s_last) {
        const double s0 = total_of(P.parts, P.n_tiles, red);
        const double s1 = total_of(P.parts + P.parts_stride, P.n_tiles, red);
        if (t == 0) {
          P.st->ctr[0] = 0u;
          post_scalars(P.st, post, s0, s1);
        }
      }
      __syncthreads();
    }
  }
}

// Tile-edge pass of the FP64 operator without recomputed halo.  The operator leaves a tile's
// first node column and row (ni = 0 or nj = 0) with its own voxels' forces only, and exports per
// node layer the forces its last voxel column and row put on the nodes just beyond it, into z
// (which Algorithm 2 does not read between the direction and the next update).  Each edge node
// here adds, in this fixed order, the exports of its left, front and diagonal neighbour tiles
// (periodic), stores Ah and its h.Ah term; the problem's last item sums the operator's and this
// pass's partial sums in tile order and takes the scalar step.
constexpr int kEdgeThreads = 256;
__global__ void __launch_bounds__(kEdgeThreads)
    k_edge64(const Prob* __restrict__ probs, const int* __restrict__ item_prob, const long long* __restrict__ counts,
             int post, int gate) {
  __shared__ double red[32];
  __shared__ int s_last;
  const long long n_items = counts[0];
  for (long long item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Prob& P = probs[item_prob[item]];
    if (gate != GATE_NONE && gate_skips(gate, P.st)) continue;  // uniform over the block
    const int nx = P.nx, ny = P.ny, nz = P.nz, tx = P.tx, ty = P.ty;
    const long long N = P.N, plane = (long long)nx * ny;
    const int tile = (int)(item - P.item0_apply);
    const int bx = tile % P.tiles_x, by = (tile / P.tiles_x) % P.tiles_y, bz = tile / (P.tiles_x * P.tiles_y);
    const int i0 = bx * tx, j0 = by * ty, k0 = bz * P.kc, k1 = min(k0 + P.kc, nz);
    const int rx = min(tx, nx - i0), ry = min(ty, ny - j0);
    const int bxl = (bx + P.tiles_x - 1) % P.tiles_x, byf = (by + P.tiles_y - 1) % P.tiles_y;
    const int ryf = min(ty, ny - byf * ty);
    const long long E = 6LL * (tx + ty);  // per tile and node layer: column records, then row records
    const long long tl = bxl + (long long)P.tiles_x * (by + (long long)P.tiles_y * bz);
    const long long tf = bx + (long long)P.tiles_x * (byf + (long long)P.tiles_y * bz);
    const long long td = bxl + (long long)P.tiles_x * (byf + (long long)P.tiles_y * bz);
    const int nb = rx + ry - 1;  // edge nodes per layer: (0, 0..ry-1), then (1..rx-1, 0)
    const double* __restrict__ ex = reinterpret_cast<const double*>(P.z);
    const double* __restrict__ h = reinterpret_cast<const double*>(P.h);
    double* __restrict__ y = reinterpret_cast<double*>(P.Ah);
    DotAcc<double> dot;
    const long long total = (long long)nb * (k1 - k0);
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int l = (int)(idx / nb), q = (int)(idx % nb);
      const int ni = q < ry ? 0 : q - ry + 1, nj = q < ry ? q : 0;
      const long long n = (long long)(k0 + l) * plane + (long long)(j0 + nj) * nx + (i0 + ni);
      double v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = y[c * N + n];
      // column record j of a tile: its last column's voxel at row j+1, corners (1,0) then (1,1);
      // row record i: its last row's voxel at column i+1, corners (0,1) then (1,1)
      if (ni == 0) {  // the left tile's last column: corner (1,1) of row nj (nj >= 1), (1,0) of row nj+1
        const double* s = ex + (tl * P.kc + l) * E;
        if (nj >= 1) {
#pragma unroll
          for (int c = 0; c < 3; ++c) v[c] += s[6 * (nj - 1) + 3 + c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] += s[6 * nj + c];
      }
      if (nj == 0) {  // the front tile's last row: corner (1,1) of column ni (ni >= 1), (0,1) of column ni+1
        const double* s = ex + (tf * P.kc + l) * E + 6LL * ty;
        if (ni >= 1) {
#pragma unroll
          for (int c = 0; c < 3; ++c) v[c] += s[6 * (ni - 1) + 3 + c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] += s[6 * ni + c];
      }
      if (ni == 0 && nj == 0) {  // the diagonal tile's corner column: corner (1,1)
        const double* s = ex + (td * P.kc + l) * E;
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] += s[6 * (ryf - 1) + 3 + c];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        y[c * N + n] = v[c];
        dot.add(h[c * N + n], v[c]);
      }
    }
    const double b1 = block_total(dot, red);
    if (threadIdx.x == 0) {
      P.parts[P.parts_stride + tile] = b1;
      __threadfence();
      s_last = atomicAdd(&P.st->ctr[0], 1u) == (unsigned)(P.n_tiles - 1);
    }
    __syncthreads();
    if (s_last) {
      const double s_in = total_of(P.parts, P.n_tiles, red);
      const double s_edge = total_of(P.parts + P.parts_stride, P.n_tiles, red);
      if (threadIdx.x == 0) {
        P.st->ctr[0] = 0u;
        post_scalars(P.st, post, s_in + s_edge, 0.0);
      }
    }
    __syncthreads();
  }
}

template <typename Tin, typename T, typename Tvec, int EPI, bool AFFINE, bool NOHALO = false>
cudaError_t launch_t(const BatchDev& b, int role, int post, int gate, cudaStream_t s) {
  constexpr bool f64 = sizeof(T) == 8;  // FP64 and double-float share the 8-byte configuration
  constexpr bool kFF = std::is_same<T, ff>::value;
  static_assert(!NOHALO || (f64 && EPI == EPI_STORE_DOT && !AFFINE), "no-halo form: FP64 h -> Ah with h.Ah only");
  // one block of up to 384 threads per SM for every arithmetic (FP32: 168 registers a thread; two
  // blocks of 256 at 128 registers measured 6% slower)
  auto kern = k_apply<Tin, T, Tvec, EPI, AFFINE, f64 ? kMaxThreadsF64 : kMaxThreadsF32, 1, NOHALO>;
  // the native FP64 form does without the double-float form's carried-force slots
  const size_t smem = kFF ? b.smemff : f64 ? b.smem64 : b.smem32;
  const int blocks = f64 ? b.blocks64 : b.blocks32;
  if (b.apply_threads > (f64 ? kMaxThreadsF64 : kMaxThreadsF32)) return cudaErrorInvalidConfiguration;
  if (smem > kApplySmemMax) return cudaErrorInvalidValue;
  // The dynamic shared-memory limit is a property of the kernel, shared by every context of the
  // process: it is raised once to the largest tile any tiling may choose and never lowered, so a
  // context launching a smaller tile on another thread cannot shrink it under a larger one.
  static std::once_flag once;
  static cudaError_t set_err = cudaSuccess;
  std::call_once(once, [&] {
    set_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApplySmemMax);
  });
  if (set_err != cudaSuccess) return set_err;
  kern<<<blocks, b.apply_threads, smem, s>>>(b.probs, b.item_prob, b.counts, role, post, gate);
  cudaError_t e = cudaGetLastError();
  if (NOHALO && e == cudaSuccess) {
    k_edge64<<<4 * blocks, kEdgeThreads, 0, s>>>(b.probs, b.item_prob, b.counts,
                                                                                   post, gate);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace

cudaError_t launch_apply(const BatchDev& b, int kind, int post, int gate, cudaStream_t s) {
  if (b.ff64) {  // FP64 products in double-float arithmetic
    switch (kind) {
      case AK_F64_DOT:
        // the recomputed-halo form: its halo columns cost the FP32 pipe less than the no-halo
        // form's edge pass and layout cost it (173 against 223 us per product at 100^3); the
        // no-halo form pays for native FP64, whose halo columns would occupy the FP64 pipe
        return launch_t<double, ff, double, EPI_STORE_DOT, false>(b, ROLE_H, post, gate, s);
      case AK_F64_RESID: return launch_t<double, ff, double, EPI_RESIDUAL, true>(b, ROLE_W, post, gate, s);
      case AK_MIX_RESID: return launch_t<double, ff, float, EPI_RESIDUAL, true>(b, ROLE_W, post, gate, s);
      case AK_F64_NORM: return launch_t<double, ff, double, EPI_NORM, true>(b, ROLE_W, post, gate, s);
      case AK_F64_AFFINE: return launch_t<double, ff, double, EPI_STORE, true>(b, ROLE_W, post, gate, s);
      default: break;
    }
  }
  switch (kind) {
    case AK_F64_DOT:
      if (b.nohalo64) return launch_t<double, double, double, EPI_STORE_DOT, false, true>(b, ROLE_H, post, gate, s);
      return launch_t<double, double, double, EPI_STORE_DOT, false>(b, ROLE_H, post, gate, s);
    case AK_F32_DOT: return launch_t<float, float, float, EPI_STORE_DOT, false>(b, ROLE_H, post, gate, s);
    case AK_F64_RESID: return launch_t<double, double, double, EPI_RESIDUAL, true>(b, ROLE_W, post, gate, s);
    case AK_MIX_RESID: return launch_t<double, double, float, EPI_RESIDUAL, true>(b, ROLE_W, post, gate, s);
    case AK_F64_NORM: return launch_t<double, double, double, EPI_NORM, true>(b, ROLE_W, post, gate, s);
    case AK_F64_AFFINE: return launch_t<double, double, double, EPI_STORE, true>(b, ROLE_W, post, gate, s);
  }
  return cudaErrorInvalidValue;
}

int apply_max_threads(int elem_bytes) { return elem_bytes == 8 ? kMaxThreadsF64 : kMaxThreadsF32; }

bool apply_nohalo_fits(const Prob& p) {
  const long long need = (long long)sizeof(double) * 6 * p.n_tiles * p.kc * (p.tx + p.ty);
  return p.z != nullptr && p.z_bytes > 0 && need <= p.z_bytes;
}

int apply_resident_blocks(int elem_bytes, int threads, size_t smem) {
  int R = elem_bytes == 8 ? 1 : std::max(1, (int)(65536 / (threads * 168)));
  R = std::min(R, (int)((227 * 1024) / (smem + 1024)));
  return std::max(R, 1);
}

size_t apply_smem_bytes(int tx, int ty, int elem_bytes) {
  const size_t NP = (size_t)(tx + 2) * (ty + 2), NV = (size_t)(tx + 1) * (ty + 1);
  return 4 * (kRing * NP + 8 * NV) * elem_bytes;  // node ring + 2 face-force buffers, 4-wide records
}

size_t apply_smem_bytes_ff(int tx, int ty) {
  const size_t NP = (size_t)(tx + 2) * (ty + 2), NV = (size_t)(tx + 1) * (ty + 1);
  // node ring (double records, split in place), 2 compact face-force buffers (24 bytes a record),
  // the per-thread slots of the carried face forces
  return 4 * kRing * NP * sizeof(double) + 2 * 4 * NV * 24 + kFupSlotBytes;
}

Tiling make_tiling(const Geo& g, int elem_bytes, int sm_count, int tx_hint, int ty_hint, int kc_hint) {
  // Model: the SM is throughput-bound, so the time of a launch is the busiest SM's work.  With R
  // blocks resident per SM (registers ~128/thread, shared memory per block), tiles are handed out
  // round-robin to sm_count*R blocks; the busiest SM runs ceil(n_tiles/(sm_count*R)) rounds of R
  // tiles, each (kc + 1) voxel layers of `threads` voxel slots plus a fixed per-layer overhead
  // (the barrier and the staging).  FP32 tiles also pay for latency not hidden by fewer
  // than two resident blocks.
  Tiling best{};
  double best_cost = 1e300;
  const int tx_lo = tx_hint ? tx_hint : 4, tx_hi = tx_hint ? tx_hint : 40;
  const int ty_lo = ty_hint ? ty_hint : 2, ty_hi = ty_hint ? ty_hint : 24;
  const int min_threads = elem_bytes == 8 ? 192 : 96;
  const int max_threads = elem_bytes == 8 ? kMaxThreadsF64 : kMaxThreadsF32;
  for (int tx = tx_lo; tx <= tx_hi; ++tx)
    for (int ty = ty_lo; ty <= ty_hi; ++ty) {
      // every item of a launch runs with the same block size; threads beyond the tile idle
      const int nv = (tx + 1) * (ty + 1);
      const int threads = max_threads;
      if (nv > threads || tx * ty > threads) continue;
      if (nv < min_threads && !(tx_hint && ty_hint)) continue;
      const size_t smem = elem_bytes == 8 ? std::max(apply_smem_bytes(tx, ty, 8), apply_smem_bytes_ff(tx, ty))
                                          : apply_smem_bytes(tx, ty, elem_bytes);
      if (smem > kApplySmemMax) continue;
      const int R = apply_resident_blocks(elem_bytes, threads, smem);
      const int tiles_x = (g.nx + tx - 1) / tx, tiles_y = (g.ny + ty - 1) / ty;
      for (int kc = (kc_hint ? kc_hint : 1); kc <= (kc_hint ? kc_hint : std::min(64, g.nz)); ++kc) {
        const int tiles_z = (g.nz + kc - 1) / kc;
        const long long n_tiles = (long long)tiles_x * tiles_y * tiles_z;
        const long long slots = (long long)sm_count * R;
        const long long blocks = n_tiles < slots ? n_tiles : slots;
        const long long rounds = (n_tiles + slots - 1) / slots;
        const double per_sm_tiles = (double)rounds * std::min<long long>(R, (n_tiles + sm_count - 1) / sm_count);
        double cost = per_sm_tiles * (kc + 1 + 0.5) * (threads + 64);
        if (n_tiles > (1LL << 30)) continue;
        if (elem_bytes == 4 && blocks < 2LL * sm_count) cost *= 1.0 + 0.5 * (2.0 - (double)blocks / sm_count) / 2.0;
        if (cost < best_cost * 0.999) {
          best_cost = cost;
          best.tx = tx; best.ty = ty; best.kc = kc;
          best.tiles_x = tiles_x; best.tiles_y = tiles_y; best.tiles_z = tiles_z;
          best.n_tiles = n_tiles;
          best.threads = threads;
          best.blocks = (int)blocks;
          best.smem = smem;
        }
      }
    }
  return best;
}

// ---- point-block Jacobi (Eq. 9) --------------------------------------------------------------
// A_mm = sum over the 8 voxels around node m of the corner's diagonal block of K_e, read from the
// per-phase table (corner a and 7 - a share one block); a node without solid voxels gets the
// identity, so that the preconditioner stays defined on fully void regions.
// mode: ELAS_PRECOND_BLOCK (the inverse block), ELAS_PRECOND_SCALAR (inverse diagonal entries
// only, M = diag A) or ELAS_PRECOND_NONE (identity: plain CG), all in the same 6-plane layout.
__global__ void k_jacobi(int nx, int ny, int nz, long long N, const int32_t* __restrict__ phase,
                         const double* __restrict__ coef64, double* __restrict__ minv64, float* __restrict__ minv32,
                         int mode) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / ((long long)nx * ny));
    double D[6] = {0, 0, 0, 0, 0, 0};  // 11 22 33 23 13 12
    int solid = 0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
      const long long e = (long long)wrapi(i - ax, nx) + (long long)nx * (wrapi(j - ay, ny) + (long long)ny * wrapi(k - az, nz));
      const int ph = phase[e];
      if (ph < 0) continue;
      const double* T = coef64 + (long long)ph * kCoefStride;
      if (__ldg(T + kCoefFlag) == 0.0) continue;
      ++solid;
      const double* Da = T + kCoefJac + 6 * (a < 4 ? a : 7 - a);
#pragma unroll
      for (int q = 0; q < 6; ++q) D[q] += __ldg(Da + q);
    }
    double inv[6];
    if (solid == 0 || mode == ELAS_PRECOND_NONE) {
      inv[0] = inv[1] = inv[2] = 1.0;
      inv[3] = inv[4] = inv[5] = 0.0;
    } else if (mode == ELAS_PRECOND_SCALAR) {
      inv[0] = 1.0 / D[0];
      inv[1] = 1.0 / D[1];
      inv[2] = 1.0 / D[2];
      inv[3] = inv[4] = inv[5] = 0.0;
    } else {
      const double a11 = D[0], a22 = D[1], a33 = D[2], a23 = D[3], a13 = D[4], a12 = D[5];
      const double c11 = a22 * a33 - a23 * a23, c22 = a11 * a33 - a13 * a13, c33 = a11 * a22 - a12 * a12;
      const double c23 = a12 * a13 - a11 * a23, c13 = a12 * a23 - a22 * a13, c12 = a13 * a23 - a33 * a12;
      const double det = a11 * c11 + a12 * c12 + a13 * c13;
      const double r = 1.0 / det;
      inv[0] = c11 * r; inv[1] = c22 * r; inv[2] = c33 * r;
      inv[3] = c23 * r; inv[4] = c13 * r; inv[5] = c12 * r;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      if (minv64) minv64[q * N + n] = inv[q];
      if (minv32) minv32[q * N + n] = (float)inv[q];
    }
  }
}

cudaError_t launch_jacobi(const Geo& g, const int32_t* phase, const double* coef64, double* minv64, float* minv32,
                          int sm_count, cudaStream_t s, int mode) {
  const int threads = 256;
  long long blocks = (g.N + threads - 1) / threads;
  if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
  k_jacobi<<<(int)blocks, threads, 0, s>>>(g.nx, g.ny, g.nz, g.N, phase, coef64, minv64, minv32, mode);
  return cudaGetLastError();
}

// ---- right-hand side b_m = sum over the 8 voxels around m of sigma_e . n_a, n_a = s_a / 4 ------
// (K_e Ebar)_a = int grad N_a dV . (C:E) = sigma . n_a exactly, so b needs only sigma per phase.
__global__ void k_rhs(int nx, int ny, int nz, long long N, const int32_t* __restrict__ phase,
                      const double* __restrict__ sig, double* __restrict__ b) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / ((long long)nx * ny));
    double f[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
      const long long e = (long long)wrapi(i - ax, nx) + (long long)nx * (wrapi(j - ay, ny) + (long long)ny * wrapi(k - az, nz));
      const int ph = phase[e];
      if (ph < 0) continue;
      const double* S = sig + 6 * (long long)ph;  // 11 22 33 23 13 12
      const double sx = 0.25 * (2 * ax - 1), sy = 0.25 * (2 * ay - 1), sz = 0.25 * (2 * az - 1);
      f[0] += S[0] * sx + S[5] * sy + S[4] * sz;
      f[1] += S[5] * sx + S[1] * sy + S[3] * sz;
      f[2] += S[4] * sx + S[3] * sy + S[2] * sz;
    }
    b[n] = f[0];
    b[N + n] = f[1];
    b[2 * N + n] = f[2];
  }
}

cudaError_t launch_rhs(const Geo& g, const int32_t* phase, const double* sig, double* b, int sm_count, cudaStream_t s) {
  const int threads = 256;
  long long blocks = (g.N + threads - 1) / threads;
  if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
  k_rhs<<<(int)blocks, threads, 0, s>>>(g.nx, g.ny, g.nz, g.N, phase, sig, b);
  return cudaGetLastError();
}

// ---- stress (stress_OpenMP / stress_fullfield_OpenMP) ---------------------------------------
// Centroid gradient: d w_c / d x_d = (sum_a s_d(a) w_a,c) / 4.
__global__ void k_stress(int nx, int ny, int nz, long long N, const int32_t* __restrict__ phase,
                         const double* __restrict__ cfull, StressE E6, const double* __restrict__ w,
                         double* __restrict__ stress, double* __restrict__ vm, double* parts, unsigned int* ctr,
                         double* macro_out) {
  __shared__ double red[32];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
    const int ph = phase[e];
    double s6[6] = {0, 0, 0, 0, 0, 0};
    if (ph >= 0) {
      double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // G[c][d]
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
        const long long n = (long long)wrapi(i + ax, nx) + (long long)nx * (wrapi(j + ay, ny) + (long long)ny * wrapi(k + az, nz));
        const double sd[3] = {0.25 * (2 * ax - 1), 0.25 * (2 * ay - 1), 0.25 * (2 * az - 1)};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double wc = w[c * N + n];
#pragma unroll
          for (int d = 0; d < 3; ++d) G[c][d] += sd[d] * wc;
        }
      }
      const double ev[6] = {E6.v[0] + G[0][0], E6.v[1] + G[1][1], E6.v[2] + G[2][2],
                            2.0 * E6.v[3] + G[1][2] + G[2][1], 2.0 * E6.v[4] + G[0][2] + G[2][0],
                            2.0 * E6.v[5] + G[0][1] + G[1][0]};
      const double* C = cfull + (long long)ph * kSymStride;
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        double t = 0.0;
#pragma unroll
        for (int c = 0; c < 6; ++c) t += C[pk(r, c)] * ev[c];
        s6[r] = t;
      }
    }
    if (stress) {
#pragma unroll
      for (int r = 0; r < 6; ++r) stress[r * N + e] = s6[r];
    }
    if (vm) {
      const double d1 = s6[0] - s6[1], d2 = s6[1] - s6[2], d3 = s6[2] - s6[0];
      vm[e] = sqrt(0.5 * (d1 * d1 + d2 * d2 + d3 * d3) + 3.0 * (s6[3] * s6[3] + s6[4] * s6[4] + s6[5] * s6[5]));
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) acc[r] += s6[r];
  }
  double b[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) b[r] = block_sum(acc[r], red);
  if (!publish_and_arrive(parts, b, 6, ctr)) return;
  for (int r = 0; r < 6; ++r) {
    const double tot = total_of(parts + r * kMaxParts, gridDim.x, red);
    if (threadIdx.x == 0) macro_out[r] = tot / (double)N;
  }
  if (threadIdx.x == 0) *ctr = 0u;
}

cudaError_t launch_stress(const Geo& g, const int32_t* phase, const double* cfull, const double* E6,
                          const double* w, double* stress, double* vm, double* parts, unsigned int* ctr,
                          double* macro_out, int sm_count, cudaStream_t s) {
  const int threads = 256;
  long long blocks = (g.N + threads - 1) / threads;
  if (blocks > (long long)sm_count * 8) blocks = (long long)sm_count * 8;
  if (blocks > kMaxParts) blocks = kMaxParts;  // one partial-sum slot per block
  StressE e;
  for (int i = 0; i < 6; ++i) e.v[i] = E6[i];
  k_stress<<<(int)blocks, threads, 0, s>>>(g.nx, g.ny, g.nz, g.N, phase, cfull, e, w, stress, vm, parts, ctr, macro_out);
  return cudaGetLastError();
}

}  // namespace elas
