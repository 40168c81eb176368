// Grain seeding (Algorithm 3) and crystallographic orientation assignment (Algorithm 6) of
// ELAS3D-Xtal (arXiv 2602.07354, Sec. 2.2.1 and 2.2.3) on the device, one thread per grain.
//
// The random draws of both algorithms are inputs (standard normal and uniform variates, angles),
// so a caller's generator decides the statistics and every result is reproducible.  Seeding:
// lognormal diameter and aspect ratio (Eq. 10), given by the mean and standard deviation of the
// variate itself, prolate semi-axes rt = d/2, rl = alpha rt, and uniform seed positions.
// Orientations: the fibre texture (crystal axis turned onto the build direction, uniform spin
// about it, Gaussian wobble about an in-plane axis) or Shoemake's uniform quaternions, both
// returned as Rodrigues vectors rho = tan(theta/2) n.  The rotation matrix of the fibre texture is
// turned into its quaternion by the largest-component (Shepperd) rule, which stays accurate up to
// the half turn; the half-turn guard of the random branch (|q_w| < 1e-8: rho = 1e9 (x, y, z)) is
// applied to both branches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "elas_internal.h"

namespace elas {

namespace {

constexpr int kTexThreads = 256;

// lognormal parameters (log-space mean m, spread s) of a variate with mean mu and deviation sd
void lognormal_params(double mu, double sd, double* m, double* s) {
  const double r = sd / mu;
  *s = std::sqrt(std::log(1.0 + r * r));
  *m = std::log(mu) - 0.5 * (*s) * (*s);
}

struct SeedArgs {
  double lo[3], span[3];
  double m_d, s_d, m_a, s_a;
};

// Explicitly rounded operations: the products and sums are rounded one at a time, never fused,
// so that seeds equal lo + u (hi - lo) as written.
__global__ void k_seed_grains(int n, SeedArgs a, const double* __restrict__ z, const double* __restrict__ u,
                              double* __restrict__ seeds, double* __restrict__ semi) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double d = exp(__dadd_rn(a.m_d, __dmul_rn(a.s_d, z[2 * i])));
    const double alpha = exp(__dadd_rn(a.m_a, __dmul_rn(a.s_a, z[2 * i + 1])));
    const double rt = d / 2.0;
    semi[2 * i] = rt;
    semi[2 * i + 1] = __dmul_rn(alpha, rt);
#pragma unroll
    for (int c = 0; c < 3; ++c) seeds[3 * i + c] = __dadd_rn(a.lo[c], __dmul_rn(u[3 * i + c], a.span[c]));
  }
}

struct OrientArgs {
  int texture;
  double Rb[9];  // fibre texture: rotation taking the crystal axis onto the sample axis (row-major)
};

__device__ __forceinline__ void store_rodrigues(double w, double x, double y, double z, double* rho) {
  if (fabs(w) < 1e-8) {
    rho[0] = x * 1e9;
    rho[1] = y * 1e9;
    rho[2] = z * 1e9;
  } else {
    rho[0] = x / w;
    rho[1] = y / w;
    rho[2] = z / w;
  }
}

__global__ void k_orientations(int n, OrientArgs a, const double* __restrict__ draws, double* __restrict__ rho) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double d0 = draws[3 * k], d1 = draws[3 * k + 1], d2 = draws[3 * k + 2];
    if (a.texture == ELAS_TEXTURE_RANDOM) {
      // Shoemake: (q_w, q_x, q_y, q_z) from u1, u2, u3
      double s2, c2, s3, c3;
      sincos(2.0 * M_PI * d1, &s2, &c2);
      sincos(2.0 * M_PI * d2, &s3, &c3);
      const double r1 = sqrt(1.0 - d0), r0 = sqrt(d0);
      store_rodrigues(r1 * s2, r1 * c2, r0 * s3, r0 * c3, rho + 3 * k);
      continue;
    }
    // fibre: R = R_spin(phi) R_wobble(theta about (cos alpha, sin alpha, 0)) R_base
    double sp, cp, sa, ca, st, ct;
    sincos(d0, &sp, &cp);
    sincos(d1, &sa, &ca);
    sincos(d2, &st, &ct);
    // wobble: I + sin t K + (1 - cos t) K^2 for the unit axis k = (ca, sa, 0)
    const double v = 1.0 - ct;
    const double W[9] = {1.0 + v * (ca * ca - 1.0), v * ca * sa, st * sa,
                         v * ca * sa, 1.0 + v * (sa * sa - 1.0), -st * ca,
                         -st * sa, st * ca, 1.0 - v};
    double SW[9];
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // spin about X3 applied to the wobble's rows
      SW[j] = cp * W[j] - sp * W[3 + j];
      SW[3 + j] = sp * W[j] + cp * W[3 + j];
      SW[6 + j] = W[6 + j];
    }
    double R[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        R[3 * i + j] = SW[3 * i] * a.Rb[j] + SW[3 * i + 1] * a.Rb[3 + j] + SW[3 * i + 2] * a.Rb[6 + j];
    // quaternion of R by its largest component
    const double tr = R[0] + R[4] + R[8];
    double w, x, y, z;
    if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
      w = 0.5 * sqrt(1.0 + tr);
      const double f = 0.25 / w;
      x = (R[7] - R[5]) * f; y = (R[2] - R[6]) * f; z = (R[3] - R[1]) * f;
    } else if (R[0] >= R[4] && R[0] >= R[8]) {
      x = 0.5 * sqrt(1.0 + R[0] - R[4] - R[8]);
      const double f = 0.25 / x;
      w = (R[7] - R[5]) * f; y = (R[1] + R[3]) * f; z = (R[2] + R[6]) * f;
    } else if (R[4] >= R[8]) {
      y = 0.5 * sqrt(1.0 - R[0] + R[4] - R[8]);
      const double f = 0.25 / y;
      w = (R[2] - R[6]) * f; x = (R[1] + R[3]) * f; z = (R[5] + R[7]) * f;
    } else {
      z = 0.5 * sqrt(1.0 - R[0] - R[4] + R[8]);
      const double f = 0.25 / z;
      w = (R[3] - R[1]) * f; x = (R[2] + R[6]) * f; y = (R[5] + R[7]) * f;
    }
    store_rodrigues(w, x, y, z, rho + 3 * k);
  }
}

int blocks_for(int n) { return std::max(1, std::min((n + kTexThreads - 1) / kTexThreads, 4096)); }

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

}  // namespace

}  // namespace elas

using namespace elas;

extern "C" {

int elas_grain_count(double lx, double ly, double lz, double mean_d, double mean_alpha, long long* n_grains) {
  if (!n_grains || !(lx > 0) || !(ly > 0) || !(lz > 0) || !(mean_d > 0) || !(mean_alpha > 0) || !std::isfinite(lx) ||
      !std::isfinite(ly) || !std::isfinite(lz) || !std::isfinite(mean_d) || !std::isfinite(mean_alpha))
    return gen_error(ELAS_ERR_INVALID_ARG, "elas_grain_count: lengths and means must be positive and finite");
  const double V = lx * ly * lz;
  const double Vg = M_PI * (mean_d / 2.0) * (mean_d / 2.0) * (mean_alpha * mean_d);
  const double n = std::ceil(V / Vg);
  if (!(n < 2147483647.0)) return gen_error(ELAS_ERR_INVALID_ARG, "elas_grain_count: more than 2^31-1 grains");
  *n_grains = (long long)n;
  return ELAS_OK;
}

int elas_seed_grains(int n_grains, const double* lo, const double* hi, double mean_d, double sd_d, double mean_alpha,
                     double sd_alpha, const double* z, const double* u, double* seeds, double* semi_axes,
                     void* cuda_stream) {
  if (n_grains < 0 || !lo || !hi || (n_grains > 0 && (!z || !u || !seeds || !semi_axes)))
    return gen_error(ELAS_ERR_INVALID_ARG, "elas_seed_grains: missing argument");
  if (!finite3(lo) || !finite3(hi) || !(hi[0] > lo[0]) || !(hi[1] > lo[1]) || !(hi[2] > lo[2]))
    return gen_error(ELAS_ERR_INVALID_ARG, "elas_seed_grains: the box needs finite lo < hi on every axis");
  if (!(mean_d > 0) || !(mean_alpha > 0) || !(sd_d >= 0) || !(sd_alpha >= 0) || !std::isfinite(mean_d) ||
      !std::isfinite(mean_alpha) || !std::isfinite(sd_d) || !std::isfinite(sd_alpha))
    return gen_error(ELAS_ERR_INVALID_ARG, "elas_seed_grains: means must be positive, deviations >= 0, all finite");
  if (n_grains == 0) return ELAS_OK;
  SeedArgs a{};
  for (int c = 0; c < 3; ++c) {
    a.lo[c] = lo[c];
    a.span[c] = hi[c] - lo[c];
  }
  lognormal_params(mean_d, sd_d, &a.m_d, &a.s_d);
  lognormal_params(mean_alpha, sd_alpha, &a.m_a, &a.s_a);
  k_seed_grains<<<blocks_for(n_grains), kTexThreads, 0, (cudaStream_t)cuda_stream>>>(n_grains, a, z, u, seeds,
                                                                                      semi_axes);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gen_error(ELAS_ERR_CUDA, std::string("elas_seed_grains: ") + cudaGetErrorString(e));
  return ELAS_OK;
}

int elas_orientations(int n_grains, int texture, const double* crystal_axis, const double* sample_axis,
                      const double* draws, double* rho, void* cuda_stream) {
  if (n_grains < 0 || (n_grains > 0 && (!draws || !rho)))
    return gen_error(ELAS_ERR_INVALID_ARG, "elas_orientations: missing argument");
  if (texture != ELAS_TEXTURE_FIBER && texture != ELAS_TEXTURE_RANDOM)
    return gen_error(ELAS_ERR_INVALID_ARG, "elas_orientations: texture must be ELAS_TEXTURE_FIBER or _RANDOM");
  OrientArgs a{};
  a.texture = texture;
  for (int i = 0; i < 9; ++i) a.Rb[i] = (i % 4 == 0) ? 1.0 : 0.0;
  if (texture == ELAS_TEXTURE_FIBER) {
    const double c101[3] = {1.0, 0.0, 1.0}, x3[3] = {0.0, 0.0, 1.0};
    const double* cv = crystal_axis ? crystal_axis : c101;
    const double* sv = sample_axis ? sample_axis : x3;
    if (!finite3(cv) || !finite3(sv))
      return gen_error(ELAS_ERR_INVALID_ARG, "elas_orientations: axes must be finite");
    const double nc = std::sqrt(cv[0] * cv[0] + cv[1] * cv[1] + cv[2] * cv[2]);
    const double ns = std::sqrt(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
    if (!(nc > 0) || !(ns > 0)) return gen_error(ELAS_ERR_INVALID_ARG, "elas_orientations: zero axis");
    const double c[3] = {cv[0] / nc, cv[1] / nc, cv[2] / nc}, s[3] = {sv[0] / ns, sv[1] / ns, sv[2] / ns};
    // R_base = I + [v]x + [v]x^2 (1 - c.s) / |v|^2, v = c x s (identity when |v| < 1e-8)
    const double v[3] = {c[1] * s[2] - c[2] * s[1], c[2] * s[0] - c[0] * s[2], c[0] * s[1] - c[1] * s[0]};
    const double sn2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (std::sqrt(sn2) >= 1e-8) {
      const double cs = c[0] * s[0] + c[1] * s[1] + c[2] * s[2];
      const double K[9] = {0, -v[2], v[1], v[2], 0, -v[0], -v[1], v[0], 0};
      const double f = (1.0 - cs) / sn2;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double k2 = 0.0;
          for (int m = 0; m < 3; ++m) k2 += K[3 * i + m] * K[3 * m + j];
          a.Rb[3 * i + j] += K[3 * i + j] + k2 * f;
        }
    }
  }
  if (n_grains == 0) return ELAS_OK;
  k_orientations<<<blocks_for(n_grains), kTexThreads, 0, (cudaStream_t)cuda_stream>>>(n_grains, a, draws, rho);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gen_error(ELAS_ERR_CUDA, std::string("elas_orientations: ") + cudaGetErrorString(e));
  return ELAS_OK;
}

}  // extern "C"
