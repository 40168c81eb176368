/*
 * elas_oracle.c -- plain, slow, FP64 CPU oracle for the periodic voxel finite-element
 * elasticity solve of ELAS3D-Xtal (arXiv 2602.07354, Sec. 2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or helper with
 * the CUDA path: everything here is written out from the paper's definitions in the most
 * direct form (explicit 24x24 element matrices, element-loop scatter, 4-index tensor
 * rotation), so that a reader can check it against the paper line by line.
 *
 * Conventions (identical interface, independent code):
 *   grid       nx, ny, nz >= 2 voxels; node (i,j,k) is the low corner of voxel (i,j,k);
 *              index(i,j,k) = i + nx*(j + ny*k); periodic wrap as in Sec. 2.1.1, Eq. 1.
 *   vectors    component-major ("u(ns,3)" of Alg. 2): u[c*N + node], c = 0,1,2.
 *   phases     phase[e] in [0, n_phases) or -1 (pore, zero stiffness).
 *   Voigt      order 11,22,33,23,13,12; stress vector holds tensor shears, strain vector holds
 *              engineering shears inside C*eps.
 *   corners    local corner a = ax + 2*ay + 4*az, ax,ay,az in {0,1}; local dof 3*a + c.
 *   strain     applied macroscopic strain E (Sec. 2.1.2, Eq. 5) given as tensor components
 *              (E11,E22,E33,E23,E13,E12).
 *
 * Every function is pinned by tests in tests/test_oracle_pins.py against closed forms,
 * invariants, brute force and dense linear algebra.
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Constitutive law (Sec. 2.1.1)                                                         */
/* ------------------------------------------------------------------------------------ */

/* Voigt slot of the symmetric index pair (i,j): 11->0 22->1 33->2 23->3 13->4 12->5. */
static int voigt_slot(int i, int j) { return (i == j) ? i : 6 - (i + j); }

/* Eqs. 2-3: Lame constants from (E, nu) and C_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk),
 * written into the 6x6 Voigt matrix C6[v(ij)][v(kl)] = C_ijkl. */
void or_iso_stiffness(double E, double nu, double *C6) {
  double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double mu = E / (2.0 * (1.0 + nu));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          double dij = (i == j), dkl = (k == l), dik = (i == k), djl = (j == l), dil = (i == l),
                 djk = (j == k);
          C6[voigt_slot(i, j) * 6 + voigt_slot(k, l)] = lam * dij * dkl + mu * (dik * djl + dil * djk);
        }
}

/* Alg. 1, step 1: cubic crystal stiffness in the crystal frame. */
void or_cubic_stiffness(double c11, double c12, double c44, double *C6) {
  memset(C6, 0, 36 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C6[i * 6 + j] = (i == j) ? c11 : c12;
  for (int i = 3; i < 6; ++i) C6[i * 6 + i] = c44;
}

/* Rodrigues vector rho = tan(theta/2) n (Sec. 2.2.3) -> active rotation matrix R (row-major),
 * through the unit quaternion (1, rho)/sqrt(1 + rho.rho), which stays finite for huge rho. */
void or_rodrigues_to_R(const double *rho, double *R) {
  double s = 1.0 / sqrt(1.0 + rho[0] * rho[0] + rho[1] * rho[1] + rho[2] * rho[2]);
  double w = s, x = rho[0] * s, y = rho[1] * s, z = rho[2] * s;
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Eq. 4 / Alg. 1, written on the full fourth-rank tensor: crystal -> sample push-forward
 * C'_ijkl = R_ip R_jq R_kr R_ls C_pqrs (the Bond-matrix product is the same map in Voigt form). */
void or_rotate_stiffness(const double *C6_local, const double *R, double *C6_global) {
  double C4[3][3][3][3], D4[3][3][3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) C4[i][j][k][l] = C6_local[voigt_slot(i, j) * 6 + voigt_slot(k, l)];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          double acc = 0.0;
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q)
              for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s)
                  acc += R[i * 3 + p] * R[j * 3 + q] * R[k * 3 + r] * R[l * 3 + s] * C4[p][q][r][s];
          D4[i][j][k][l] = acc;
        }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) C6_global[voigt_slot(i, j) * 6 + voigt_slot(k, l)] = D4[i][j][k][l];
}

/* ------------------------------------------------------------------------------------ */
/* Trilinear hexahedral element on the unit voxel [0,1]^3 (Sec. 2.1.1)                   */
/* ------------------------------------------------------------------------------------ */

/* Derivatives dN_a/dx_d of the 8 trilinear shape functions at point p in [0,1]^3. */
static void shape_grad(const double *p, double dN[8][3]) {
  for (int a = 0; a < 8; ++a) {
    int c[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1};
    double f[3], df[3];
    for (int d = 0; d < 3; ++d) {
      f[d] = c[d] ? p[d] : 1.0 - p[d];
      df[d] = c[d] ? 1.0 : -1.0;
    }
    dN[a][0] = df[0] * f[1] * f[2];
    dN[a][1] = f[0] * df[1] * f[2];
    dN[a][2] = f[0] * f[1] * df[2];
  }
}

/* Strain-displacement matrix B (6 x 24, engineering shears) at point p. */
static void bmatrix(const double *p, double B[6][24]) {
  double dN[8][3];
  shape_grad(p, dN);
  memset(B, 0, 6 * 24 * sizeof(double));
  for (int a = 0; a < 8; ++a) {
    B[0][3 * a + 0] = dN[a][0];
    B[1][3 * a + 1] = dN[a][1];
    B[2][3 * a + 2] = dN[a][2];
    B[3][3 * a + 1] = dN[a][2];
    B[3][3 * a + 2] = dN[a][1];
    B[4][3 * a + 0] = dN[a][2];
    B[4][3 * a + 2] = dN[a][0];
    B[5][3 * a + 0] = dN[a][1];
    B[5][3 * a + 1] = dN[a][0];
  }
}

/* Element stiffness K_e = int_{[0,1]^3} B^T C B dV (24 x 24, row-major).
 * rule 0: 2x2x2 Gauss-Legendre; rule 1: 3x3x3 Simpson.  Both are exact for this integrand
 * (degree <= 2 in each coordinate), which is what makes them a cross-check of each other. */
void or_element_stiffness(const double *C6, int rule, double *Ke) {
  double pts[3], wts[3];
  int np;
  if (rule == 0) {
    double g = 0.5 / sqrt(3.0);
    pts[0] = 0.5 - g; pts[1] = 0.5 + g; wts[0] = wts[1] = 0.5; np = 2;
  } else {
    pts[0] = 0.0; pts[1] = 0.5; pts[2] = 1.0;
    wts[0] = 1.0 / 6.0; wts[1] = 4.0 / 6.0; wts[2] = 1.0 / 6.0; np = 3;
  }
  memset(Ke, 0, 576 * sizeof(double));
  for (int qx = 0; qx < np; ++qx)
    for (int qy = 0; qy < np; ++qy)
      for (int qz = 0; qz < np; ++qz) {
        double p[3] = {pts[qx], pts[qy], pts[qz]};
        double w = wts[qx] * wts[qy] * wts[qz];
        double B[6][24], CB[6][24];
        bmatrix(p, B);
        for (int r = 0; r < 6; ++r)
          for (int c = 0; c < 24; ++c) {
            double acc = 0.0;
            for (int s = 0; s < 6; ++s) acc += C6[r * 6 + s] * B[s][c];
            CB[r][c] = acc;
          }
        for (int r = 0; r < 24; ++r)
          for (int c = 0; c < 24; ++c) {
            double acc = 0.0;
            for (int s = 0; s < 6; ++s) acc += B[s][r] * CB[s][c];
            Ke[r * 24 + c] += w * acc;
          }
      }
}

/* Per-phase tables: C_global (n_phases x 36) and K_e (n_phases x 576) from the crystal-frame
 * C_local (n_phases x 36) and Rodrigues vectors (n_phases x 3, NULL = identity). */
void or_phase_tables(int n_phases, const double *C6_local, const double *rho, double *C6_global,
                     double *Ke_tab) {
  for (int p = 0; p < n_phases; ++p) {
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (rho) or_rodrigues_to_R(rho + 3 * p, R);
    or_rotate_stiffness(C6_local + 36 * p, R, C6_global + 36 * p);
    or_element_stiffness(C6_global + 36 * p, 0, Ke_tab + 576 * (size_t)p);
  }
}

/* ------------------------------------------------------------------------------------ */
/* Periodic grid (Sec. 2.1.1, Eq. 1)                                                      */
/* ------------------------------------------------------------------------------------ */

static int64_t wrap(int64_t i, int64_t n) { return ((i % n) + n) % n; }

/* Node of local corner a of voxel (i,j,k) after the periodic wrap. */
static int64_t corner_node(int nx, int ny, int nz, int64_t i, int64_t j, int64_t k, int a) {
  int64_t ii = wrap(i + (a & 1), nx), jj = wrap(j + ((a >> 1) & 1), ny), kk = wrap(k + ((a >> 2) & 1), nz);
  return ii + (int64_t)nx * (jj + (int64_t)ny * kk);
}

/* Applied strain E as a symmetric 3x3 tensor from (E11,E22,E33,E23,E13,E12). */
static void strain_tensor(const double *e6, double E[3][3]) {
  E[0][0] = e6[0]; E[1][1] = e6[1]; E[2][2] = e6[2];
  E[1][2] = E[2][1] = e6[3];
  E[0][2] = E[2][0] = e6[4];
  E[0][1] = E[1][0] = e6[5];
}

/* Affine element displacement Ebar_a = E . x_a at the 8 local corners x_a in {0,1}^3 (Eq. 5). */
static void affine_element(const double *e6, double *Ebar) {
  double E[3][3];
  strain_tensor(e6, E);
  for (int a = 0; a < 8; ++a) {
    double x[3] = {(double)(a & 1), (double)((a >> 1) & 1), (double)((a >> 2) & 1)};
    for (int i = 0; i < 3; ++i) Ebar[3 * a + i] = E[i][0] * x[0] + E[i][1] * x[1] + E[i][2] * x[2];
  }
}

/* ------------------------------------------------------------------------------------ */
/* Global operator, right-hand side, energy (Sec. 2.1.2, Eqs. 7-8)                        */
/* ------------------------------------------------------------------------------------ */

/* y = A u with A = sum_e P_e^T K_e P_e (element loop, scatter-add; aliasing on 2-wide grids
 * adds automatically).  Matrix-free product of Sec. 2.1.2 written in its plainest form. */
void or_apply(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, const double *u,
              double *y) {
  int64_t N = (int64_t)nx * ny * nz;
  memset(y, 0, 3 * N * sizeof(double));
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t e = i + nx * (j + ny * k);
        if (phase[e] < 0) continue;
        const double *Ke = Ke_tab + 576 * (size_t)phase[e];
        int64_t nodes[8];
        double ue[24], ye[24];
        for (int a = 0; a < 8; ++a) {
          nodes[a] = corner_node(nx, ny, nz, i, j, k, a);
          for (int c = 0; c < 3; ++c) ue[3 * a + c] = u[c * N + nodes[a]];
        }
        for (int r = 0; r < 24; ++r) {
          double acc = 0.0;
          for (int s = 0; s < 24; ++s) acc += Ke[r * 24 + s] * ue[s];
          ye[r] = acc;
        }
        for (int a = 0; a < 8; ++a)
          for (int c = 0; c < 3; ++c) y[c * N + nodes[a]] += ye[3 * a + c];
      }
}

/* Rows of A u for a list of nodes only (gather over the 8 voxels around each node).  Lets the
 * tests check very large grids at sampled nodes; pinned against or_apply on small grids. */
void or_apply_nodes(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, const double *u,
                    int64_t n_sel, const int64_t *sel, double *y_sel /* n_sel x 3 */) {
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t s = 0; s < n_sel; ++s) {
    int64_t m = sel[s];
    int64_t i = m % nx, j = (m / nx) % ny, k = m / ((int64_t)nx * ny);
    double acc[3] = {0, 0, 0};
    for (int a = 0; a < 8; ++a) {
      /* voxel whose corner a is node m */
      int64_t ei = wrap(i - (a & 1), nx), ej = wrap(j - ((a >> 1) & 1), ny), ek = wrap(k - ((a >> 2) & 1), nz);
      int64_t e = ei + nx * (ej + ny * ek);
      if (phase[e] < 0) continue;
      const double *Ke = Ke_tab + 576 * (size_t)phase[e];
      for (int b = 0; b < 8; ++b) {
        int64_t nb = corner_node(nx, ny, nz, ei, ej, ek, b);
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) acc[c] += Ke[(3 * a + c) * 24 + 3 * b + d] * u[d * N + nb];
      }
    }
    for (int c = 0; c < 3; ++c) y_sel[3 * s + c] = acc[c];
  }
}

/* Right-hand side b = sum_e P_e^T K_e Ebar (Eqs. 5-8 in fluctuation form u = E.X + w). */
void or_rhs(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, const double *e6, double *b) {
  int64_t N = (int64_t)nx * ny * nz;
  double Ebar[24];
  affine_element(e6, Ebar);
  memset(b, 0, 3 * N * sizeof(double));
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t e = i + nx * (j + ny * k);
        if (phase[e] < 0) continue;
        const double *Ke = Ke_tab + 576 * (size_t)phase[e];
        for (int a = 0; a < 8; ++a) {
          int64_t n = corner_node(nx, ny, nz, i, j, k, a);
          for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int s = 0; s < 24; ++s) acc += Ke[(3 * a + c) * 24 + s] * Ebar[s];
            b[c * N + n] += acc;
          }
        }
      }
}

/* Scale of the right-hand side without cancellation: sqrt(sum_e sum_a |(K_e Ebar)_a|^2), the norm
 * of the unassembled element forces.  A right-hand side with ||b|| <= 1e-12 of this is round-off
 * of an exactly zero load (homogeneous cell) and is treated as zero. */
double or_rhs_scale(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, const double *e6) {
  int64_t N = (int64_t)nx * ny * nz;
  double Ebar[24], acc = 0.0;
  affine_element(e6, Ebar);
  for (int64_t e = 0; e < N; ++e) {
    if (phase[e] < 0) continue;
    const double *Ke = Ke_tab + 576 * (size_t)phase[e];
    for (int r = 0; r < 24; ++r) {
      double t = 0.0;
      for (int s = 0; s < 24; ++s) t += Ke[r * 24 + s] * Ebar[s];
      acc += t * t;
    }
  }
  return sqrt(acc);
}

/* Total potential energy Pi(w) = sum_e 1/2 (w_e + Ebar)^T K_e (w_e + Ebar) (Eq. 7, with the
 * constant and linear terms of the affine start folded in). */
double or_energy(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, const double *e6,
                 const double *w) {
  int64_t N = (int64_t)nx * ny * nz;
  double Ebar[24], total = 0.0;
  affine_element(e6, Ebar);
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t e = i + nx * (j + ny * k);
        if (phase[e] < 0) continue;
        const double *Ke = Ke_tab + 576 * (size_t)phase[e];
        double ue[24];
        for (int a = 0; a < 8; ++a) {
          int64_t n = corner_node(nx, ny, nz, i, j, k, a);
          for (int c = 0; c < 3; ++c) ue[3 * a + c] = w[c * N + n] + Ebar[3 * a + c];
        }
        double q = 0.0;
        for (int r = 0; r < 24; ++r)
          for (int s = 0; s < 24; ++s) q += ue[r] * Ke[r * 24 + s] * ue[s];
        total += 0.5 * q;
      }
  return total;
}

/* Dense A (3N x 3N, row-major, dof index c*N + node) for grids of a few hundred nodes. */
void or_dense(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, double *A) {
  int64_t N = (int64_t)nx * ny * nz, D = 3 * N;
  memset(A, 0, D * D * sizeof(double));
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t e = i + nx * (j + ny * k);
        if (phase[e] < 0) continue;
        const double *Ke = Ke_tab + 576 * (size_t)phase[e];
        int64_t nodes[8];
        for (int a = 0; a < 8; ++a) nodes[a] = corner_node(nx, ny, nz, i, j, k, a);
        for (int a = 0; a < 8; ++a)
          for (int c = 0; c < 3; ++c)
            for (int b = 0; b < 8; ++b)
              for (int d = 0; d < 3; ++d)
                A[(c * N + nodes[a]) * D + d * N + nodes[b]] += Ke[(3 * a + c) * 24 + 3 * b + d];
      }
}

/* ------------------------------------------------------------------------------------ */
/* Point-block Jacobi preconditioner (Sec. 2.1.2, Eq. 9)                                   */
/* ------------------------------------------------------------------------------------ */

/* Minv: N x 9 (row-major 3x3 per node).  A_mm = sum over the 8 voxels around m of the
 * corner's 3x3 diagonal block of K_e, inverted by cofactors; identity where the block is
 * exactly zero (all 8 voxels are pores). */
void or_jacobi(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, double *Minv) {
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t m = 0; m < N; ++m) {
    int64_t i = m % nx, j = (m / nx) % ny, k = m / ((int64_t)nx * ny);
    double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < 8; ++a) {
      int64_t ei = wrap(i - (a & 1), nx), ej = wrap(j - ((a >> 1) & 1), ny), ek = wrap(k - ((a >> 2) & 1), nz);
      int64_t e = ei + nx * (ej + ny * ek);
      if (phase[e] < 0) continue;
      const double *Ke = Ke_tab + 576 * (size_t)phase[e];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] += Ke[(3 * a + r) * 24 + 3 * a + c];
    }
    int zero = 1;
    for (int t = 0; t < 9; ++t)
      if (M[t] != 0.0) zero = 0;
    double *Mi = Minv + 9 * m;
    if (zero) {
      for (int t = 0; t < 9; ++t) Mi[t] = (t % 4 == 0) ? 1.0 : 0.0;
      continue;
    }
    double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
    double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
    Mi[0] = c00 / det;
    Mi[1] = (M[2] * M[7] - M[1] * M[8]) / det;
    Mi[2] = (M[1] * M[5] - M[2] * M[4]) / det;
    Mi[3] = c01 / det;
    Mi[4] = (M[0] * M[8] - M[2] * M[6]) / det;
    Mi[5] = (M[2] * M[3] - M[0] * M[5]) / det;
    Mi[6] = c02 / det;
    Mi[7] = (M[1] * M[6] - M[0] * M[7]) / det;
    Mi[8] = (M[0] * M[4] - M[1] * M[3]) / det;
  }
}

/* ------------------------------------------------------------------------------------ */
/* PCG (Algorithm 2, dembx), in fluctuation form: solve A w = -b from w = 0                */
/* ------------------------------------------------------------------------------------ */

static double dot3n(int64_t n3, const double *a, const double *b) {
  double s = 0.0;
  for (int64_t t = 0; t < n3; ++t) s += a[t] * b[t];
  return s;
}

/* Scalar Jacobi: Dinv (3N, component-major) = 1 / the diagonal entries of the assembled
 * diagonal blocks A_mm (the same 8-voxel sum as or_jacobi), 1 where the entry is exactly zero. */
static void scalar_jacobi(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, double *Dinv) {
  int64_t N = (int64_t)nx * ny * nz;
  for (int64_t m = 0; m < N; ++m) {
    int64_t i = m % nx, j = (m / nx) % ny, k = m / ((int64_t)nx * ny);
    double d[3] = {0, 0, 0};
    for (int a = 0; a < 8; ++a) {
      int64_t ei = wrap(i - (a & 1), nx), ej = wrap(j - ((a >> 1) & 1), ny), ek = wrap(k - ((a >> 2) & 1), nz);
      int64_t e = ei + nx * (ej + ny * ek);
      if (phase[e] < 0) continue;
      const double *Ke = Ke_tab + 576 * (size_t)phase[e];
      for (int r = 0; r < 3; ++r) d[r] += Ke[(3 * a + r) * 24 + 3 * a + r];
    }
    for (int r = 0; r < 3; ++r) Dinv[r * N + m] = d[r] != 0.0 ? 1.0 / d[r] : 1.0;
  }
}

/* precond: 0 none (z = g), 1 point-block Jacobi (Minv, N x 9), 2 scalar Jacobi (Minv holds Dinv) */
static void precondition(int64_t N, const double *Minv, const double *g, double *z, int precond) {
  for (int64_t m = 0; m < N; ++m) {
    if (precond == 0) {
      for (int c = 0; c < 3; ++c) z[c * N + m] = g[c * N + m];
      continue;
    }
    if (precond == 2) {
      for (int c = 0; c < 3; ++c) z[c * N + m] = Minv[c * N + m] * g[c * N + m];
      continue;
    }
    const double *Mi = Minv + 9 * m;
    for (int r = 0; r < 3; ++r)
      z[r * N + m] = Mi[3 * r] * g[m] + Mi[3 * r + 1] * g[N + m] + Mi[3 * r + 2] * g[2 * N + m];
  }
}

/* Outcome codes shared in meaning (not in code) with the library's info.status. */
enum { OR_CONVERGED = 0, OR_MAX_ITER = 1, OR_BREAKDOWN = 2 };

/* Algorithm 2.  w (3N) is the output, started at zero (affine start of Eq. 5).  Stops when
 * sqrt(gg/gg0) < tol with gg = z.g and gg0 its value at w = 0.  A zero load (||b|| <= 1e-12 *
 * rhs_scale) returns w = 0 as converged after 0 iterations; a non-zero load with gg0 not positive
 * (a preconditioner that is not definite) is a breakdown.  The breakdown test follows the
 * reading that replaces the absolute |hAh| < 1e-14 by "hAh not positive and finite"
 * (paper_guard = 1 restores the absolute test).  precond = 1 is the paper's point-block Jacobi;
 * 0 gives plain CG (M = I), the unpreconditioned solver Table 4 compares against, and 2 scalar
 * (point) Jacobi, M = diag(A).
 * Returns the outcome; *iters the number of completed iterations; *gg_out the final gg/gg0.
 * hist (optional, max_iter+1 entries) receives sqrt(gg/gg0) after each iteration. */
int or_pcg(int nx, int ny, int nz, const int32_t *phase, const double *Ke_tab, const double *b,
           double rhs_scale, double tol, int max_iter, int precond, int paper_guard, double *w, int *iters,
           double *ratio_out, double *hist) {
  int64_t N = (int64_t)nx * ny * nz, n3 = 3 * N;
  double *Minv = (double *)malloc(9 * N * sizeof(double));
  double *g = (double *)malloc(n3 * sizeof(double));
  double *z = (double *)malloc(n3 * sizeof(double));
  double *h = (double *)malloc(n3 * sizeof(double));
  double *Ah = (double *)malloc(n3 * sizeof(double));
  if (precond == 2)
    scalar_jacobi(nx, ny, nz, phase, Ke_tab, Minv);
  else
    or_jacobi(nx, ny, nz, phase, Ke_tab, Minv);
  memset(w, 0, n3 * sizeof(double));
  memcpy(g, b, n3 * sizeof(double));
  precondition(N, Minv, g, z, precond);
  memcpy(h, z, n3 * sizeof(double));
  double gg = dot3n(n3, z, g), gg0 = gg;
  int outcome = OR_MAX_ITER, it = 0;
  double ratio = 0.0;
  if (hist) hist[0] = 1.0;
  double bnorm = sqrt(dot3n(n3, b, b));
  if (bnorm <= 1e-12 * rhs_scale) {
    outcome = OR_CONVERGED; /* zero right-hand side: w = 0 is the solution */
  } else if (!(gg0 > 0.0)) {
    outcome = OR_BREAKDOWN; /* z.g of a non-zero load is not positive: M is not definite */
  } else {
    for (it = 0; it < max_iter;) {
      or_apply(nx, ny, nz, phase, Ke_tab, h, Ah);
      double hAh = dot3n(n3, h, Ah);
      int bad = paper_guard ? (fabs(hAh) < 1e-14) : !(hAh > 0.0 && isfinite(hAh));
      if (bad) { outcome = OR_BREAKDOWN; break; }
      double lam = gg / hAh;
      for (int64_t t = 0; t < n3; ++t) {
        w[t] -= lam * h[t];
        g[t] -= lam * Ah[t];
      }
      precondition(N, Minv, g, z, precond);
      double gg_last = gg;
      gg = dot3n(n3, z, g);
      ++it;
      ratio = sqrt(gg / gg0);
      if (hist) hist[it] = ratio;
      if (ratio < tol) { outcome = OR_CONVERGED; break; }
      double gam = gg / gg_last;
      for (int64_t t = 0; t < n3; ++t) h[t] = z[t] + gam * h[t];
    }
  }
  *iters = it;
  *ratio_out = ratio;
  free(Minv); free(g); free(z); free(h); free(Ah);
  return outcome;
}

/* ------------------------------------------------------------------------------------ */
/* Stress (stress_OpenMP / stress_fullfield_OpenMP of Table 1)                            */
/* ------------------------------------------------------------------------------------ */

/* Voxel strain at the centroid (the exact voxel average for a trilinear field):
 * eps = E + B(1/2,1/2,1/2) w_e; stress = C eps (Voigt, tensor shears out); von Mises;
 * macro stress = mean over all voxels (pores contribute zero).  stress: 6N component-major.
 * C6_tab: per-phase sample-frame stiffness. */
void or_stress(int nx, int ny, int nz, const int32_t *phase, const double *C6_tab, const double *e6,
               const double *w, double *stress, double *vm, double *macro) {
  int64_t N = (int64_t)nx * ny * nz;
  double B[6][24], mid[3] = {0.5, 0.5, 0.5};
  bmatrix(mid, B);
  double Ev[6] = {e6[0], e6[1], e6[2], 2.0 * e6[3], 2.0 * e6[4], 2.0 * e6[5]};
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t e = i + nx * (j + ny * k);
        double s[6] = {0, 0, 0, 0, 0, 0};
        if (phase[e] >= 0) {
          double ue[24], eps[6];
          for (int a = 0; a < 8; ++a) {
            int64_t n = corner_node(nx, ny, nz, i, j, k, a);
            for (int c = 0; c < 3; ++c) ue[3 * a + c] = w[c * N + n];
          }
          for (int r = 0; r < 6; ++r) {
            double t = Ev[r];
            for (int c = 0; c < 24; ++c) t += B[r][c] * ue[c];
            eps[r] = t;
          }
          const double *C6 = C6_tab + 36 * (size_t)phase[e];
          for (int r = 0; r < 6; ++r) {
            double t = 0.0;
            for (int c = 0; c < 6; ++c) t += C6[r * 6 + c] * eps[c];
            s[r] = t;
          }
        }
        for (int r = 0; r < 6; ++r) {
          stress[r * N + e] = s[r];
          acc[r] += s[r];
        }
        if (vm) {
          double d1 = s[0] - s[1], d2 = s[1] - s[2], d3 = s[2] - s[0];
          vm[e] = sqrt(0.5 * (d1 * d1 + d2 * d2 + d3 * d3) + 3.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]));
        }
      }
  for (int r = 0; r < 6; ++r) macro[r] = acc[r] / (double)N;
}

/* Voxel strain field only (Voigt, tensor shears), for the strain-average and Eshelby pins. */
void or_strain(int nx, int ny, int nz, const int32_t *phase, const double *e6, const double *w, double *strain) {
  int64_t N = (int64_t)nx * ny * nz;
  double B[6][24], mid[3] = {0.5, 0.5, 0.5};
  bmatrix(mid, B);
  (void)phase;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t e = i + nx * (j + ny * k);
        double ue[24];
        for (int a = 0; a < 8; ++a) {
          int64_t n = corner_node(nx, ny, nz, i, j, k, a);
          for (int c = 0; c < 3; ++c) ue[3 * a + c] = w[c * N + n];
        }
        for (int r = 0; r < 6; ++r) {
          double t = 0.0;
          for (int c = 0; c < 24; ++c) t += B[r][c] * ue[c];
          strain[r * N + e] = e6[r] + (r >= 3 ? 0.5 * t : t);
        }
      }
}

/* ------------------------------------------------------------------------------------ */
/* Microstructure generator (Sec. 2.2): grain assignment (Algorithm 4) and pore overwrite  */
/* (Algorithm 5), brute force over all grains / pores                                      */
/* ------------------------------------------------------------------------------------ */

/* One periodic minimum-image wrap of a difference of two points of [0, L). */
static double min_image(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

/* Voxel (i,j,k), centre (i+1/2, j+1/2, k+1/2), takes the grain l minimising the weighted
 * ellipsoidal distance of Algorithm 4, D^2 = (dx^2 + dy^2) / rt^2 + dz^2 / rl^2, with d the
 * periodic minimum-image difference of the centre and the seed s_l; ties go to the lowest l.
 * seeds: n x 3; semi: n x 2 (rt, rl), NULL for rt = rl = 1 (plain Voronoi).  Evaluated in FP64
 * in exactly this order: dx*dx + dy*dy, / (rt*rt), dz*dz / (rl*rl), sum. */
void or_assign_grains(int nx, int ny, int nz, const double *seeds, const double *semi, int n, int32_t *phase) {
  const double L[3] = {(double)nx, (double)ny, (double)nz};
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const double x[3] = {(double)i + 0.5, (double)j + 0.5, (double)k + 0.5};
        double best = INFINITY;
        int32_t arg = -1;
        for (int l = 0; l < n; ++l) {
          const double dx = min_image(x[0] - seeds[3 * l], L[0]);
          const double dy = min_image(x[1] - seeds[3 * l + 1], L[1]);
          const double dz = min_image(x[2] - seeds[3 * l + 2], L[2]);
          const double rt = semi ? semi[2 * l] : 1.0, rl = semi ? semi[2 * l + 1] : 1.0;
          const double D2 = (dx * dx + dy * dy) / (rt * rt) + (dz * dz) / (rl * rl);
          if (D2 < best) { best = D2; arg = l; }
        }
        phase[i + (int64_t)nx * (j + (int64_t)ny * k)] = arg;
      }
}

/* The same assignment for the listed voxels only (linear ids), for sampled checks on large grids. */
void or_assign_voxels(int nx, int ny, int nz, const double *seeds, const double *semi, int n, const int64_t *vox,
                      int64_t m, int32_t *out) {
  const double L[3] = {(double)nx, (double)ny, (double)nz};
  for (int64_t t = 0; t < m; ++t) {
    const int64_t v = vox[t];
    const double x[3] = {(double)(v % nx) + 0.5, (double)((v / nx) % ny) + 0.5, (double)(v / ((int64_t)nx * ny)) + 0.5};
    double best = INFINITY;
    int32_t arg = -1;
    for (int l = 0; l < n; ++l) {
      const double dx = min_image(x[0] - seeds[3 * l], L[0]);
      const double dy = min_image(x[1] - seeds[3 * l + 1], L[1]);
      const double dz = min_image(x[2] - seeds[3 * l + 2], L[2]);
      const double rt = semi ? semi[2 * l] : 1.0, rl = semi ? semi[2 * l + 1] : 1.0;
      const double D2 = (dx * dx + dy * dy) / (rt * rt) + (dz * dz) / (rl * rl);
      if (D2 < best) { best = D2; arg = l; }
    }
    out[t] = arg;
  }
}

/* Algorithm 5 with general ellipsoids: pore p = (cx, cy, cz, a0, a1, a2, R00 ... R22) with R
 * row-major whose columns are the principal axes.  A voxel is overwritten with -1 when
 * (q0/a0)^2 + (q1/a1)^2 + (q2/a2)^2 <= 1, q_m = R_0m d0 + R_1m d1 + R_2m d2, d the periodic
 * minimum-image difference of the voxel centre and the pore centre (a sphere of radius r:
 * a = (r, r, r), R = I).  Returns the number of pore voxels afterwards. */
int64_t or_stamp_pores(int nx, int ny, int nz, const double *pores, int n, int32_t *phase) {
  const double L[3] = {(double)nx, (double)ny, (double)nz};
  int64_t count = 0;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t v = i + (int64_t)nx * (j + (int64_t)ny * k);
        const double x[3] = {(double)i + 0.5, (double)j + 0.5, (double)k + 0.5};
        for (int p = 0; p < n; ++p) {
          const double *P = pores + 15 * p;
          const double d0 = min_image(x[0] - P[0], L[0]), d1 = min_image(x[1] - P[1], L[1]),
                       d2 = min_image(x[2] - P[2], L[2]);
          double t = 0.0;
          for (int m = 0; m < 3; ++m) {
            const double q = P[6 + m] * d0 + P[9 + m] * d1 + P[12 + m] * d2;
            const double u = q / P[3 + m];
            t = t + u * u;
          }
          if (t <= 1.0) {
            phase[v] = -1;
            break;
          }
        }
        count += phase[v] < 0;
      }
  return count;
}

/* ------------------------------------------------------------------------------------ */
/* Grain seeding (Algorithm 3) and orientation assignment (Algorithm 6).  The random draws  */
/* of both algorithms are inputs (standard normal z, uniform u in [0,1), angles).           */
/* ------------------------------------------------------------------------------------ */

/* Algorithm 3, part 1: grain count N_g = ceil(V / V_mean) for a box lx x ly x lz, with the mean
 * grain volume that of a cylinder of diameter mu_d and height mu_alpha * mu_d:
 * V_mean = pi (mu_d / 2)^2 (mu_alpha mu_d). */
int64_t or_grain_count(double lx, double ly, double lz, double mu_d, double mu_alpha) {
  const double V = lx * ly * lz;
  const double Vg = M_PI * (mu_d / 2.0) * (mu_d / 2.0) * (mu_alpha * mu_d);
  return (int64_t)ceil(V / Vg);
}

/* Algorithm 3, part 1 (Eq. 10 and the semi-axes): grain i draws its diameter d_i and aspect ratio
 * alpha_i from lognormal distributions given by the mean (mu) and standard deviation (sd) of the
 * variate itself: log-space spread s = sqrt(log(1 + (sd/mu)^2)), log-space mean m = log(mu) - s^2/2,
 * so d_i = exp(m_d + s_d z[2i]), alpha_i = exp(m_a + s_a z[2i+1]).  Then rt_i = d_i / 2,
 * rl_i = alpha_i rt_i (semi[2i], semi[2i+1]) and the seed s_i = lo + u (hi - lo) per axis
 * (u[3i+a]).  z: n x 2 standard normal draws; u: n x 3 uniform draws. */
void or_seed_grains(int n, const double *lo, const double *hi, double mu_d, double sd_d, double mu_a, double sd_a,
                    const double *z, const double *u, double *seeds, double *semi) {
  const double s_d = sqrt(log(1.0 + (sd_d / mu_d) * (sd_d / mu_d))), m_d = log(mu_d) - 0.5 * s_d * s_d;
  const double s_a = sqrt(log(1.0 + (sd_a / mu_a) * (sd_a / mu_a))), m_a = log(mu_a) - 0.5 * s_a * s_a;
  for (int i = 0; i < n; ++i) {
    const double d = exp(m_d + s_d * z[2 * i]);
    const double alpha = exp(m_a + s_a * z[2 * i + 1]);
    semi[2 * i] = d / 2.0;
    semi[2 * i + 1] = alpha * (d / 2.0);
    for (int a = 0; a < 3; ++a) seeds[3 * i + a] = lo[a] + u[3 * i + a] * (hi[a] - lo[a]);
  }
}

static void matmul3(const double *A, const double *B, double *C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = acc;
    }
}

/* Rotation by angle t about the unit axis k (row-major): I + sin t [k]x + (1 - cos t) [k]x^2. */
static void axis_angle_R(const double *k, double t, double *R) {
  const double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
  double K2[9];
  matmul3(K, K, K2);
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + sin(t) * K[i] + (1.0 - cos(t)) * K2[i];
}

/* Rodrigues vector of a rotation matrix from its plain definition: rho = tan(theta/2) n equals the
 * axial vector of R - R^T divided by 1 + tr R (2 sin(theta) n / (2 (1 + cos theta))). */
static void R_to_rodrigues(const double *R, double *rho) {
  const double den = 1.0 + R[0] + R[4] + R[8];
  rho[0] = (R[7] - R[5]) / den;
  rho[1] = (R[2] - R[6]) / den;
  rho[2] = (R[3] - R[1]) / den;
}

/* Algorithm 6, textured branch.  R_base turns the unit crystal axis c onto the unit sample axis
 * s (v = c x s, sin = |v|, cos = c.s: I + [v]x + [v]x^2 (1 - cos) / sin^2, or I when sin < 1e-8);
 * grain k draws a spin phi about X3, a wobble axis angle alpha and a wobble angle theta
 * (draws[3k], [3k+1], [3k+2], radians; theta ~ N(0, sigma_spread^2)), and
 * R_total = R_spin(phi) R_wobble R_base with R_wobble the rotation by theta about
 * (cos alpha, sin alpha, 0).  rho[3k..3k+2]: the Rodrigues vector of R_total. */
void or_fiber_orientations(int n, const double *crystal, const double *sample, const double *draws, double *rho) {
  double c[3], s[3];
  const double nc = sqrt(crystal[0] * crystal[0] + crystal[1] * crystal[1] + crystal[2] * crystal[2]);
  const double ns = sqrt(sample[0] * sample[0] + sample[1] * sample[1] + sample[2] * sample[2]);
  for (int a = 0; a < 3; ++a) {
    c[a] = crystal[a] / nc;
    s[a] = sample[a] / ns;
  }
  const double v[3] = {c[1] * s[2] - c[2] * s[1], c[2] * s[0] - c[0] * s[2], c[0] * s[1] - c[1] * s[0]};
  const double sn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double cs = c[0] * s[0] + c[1] * s[1] + c[2] * s[2];
  double Rb[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (!(sn < 1e-8)) {
    const double V[9] = {0, -v[2], v[1], v[2], 0, -v[0], -v[1], v[0], 0};
    double V2[9];
    matmul3(V, V, V2);
    for (int i = 0; i < 9; ++i) Rb[i] += V[i] + V2[i] * (1.0 - cs) / (sn * sn);
  }
  for (int k = 0; k < n; ++k) {
    const double phi = draws[3 * k], alpha = draws[3 * k + 1], theta = draws[3 * k + 2];
    const double Rs[9] = {cos(phi), -sin(phi), 0, sin(phi), cos(phi), 0, 0, 0, 1};
    const double ax[3] = {cos(alpha), sin(alpha), 0.0};
    double Rw[9], T[9], R[9];
    axis_angle_R(ax, theta, Rw);
    matmul3(Rs, Rw, T);
    matmul3(T, Rb, R);
    R_to_rodrigues(R, rho + 3 * k);
  }
}

/* Algorithm 6, random branch: Shoemake's uniform quaternion from u = (u1, u2, u3) (u[3k..3k+2]),
 * q_w = sqrt(1-u1) sin(2 pi u2), q_x = sqrt(1-u1) cos(2 pi u2), q_y = sqrt(u1) sin(2 pi u3),
 * q_z = sqrt(u1) cos(2 pi u3); rho = (q_x, q_y, q_z) / q_w, or (q_x, q_y, q_z) 1e9 when
 * |q_w| < 1e-8. */
void or_random_orientations(int n, const double *u, double *rho) {
  for (int k = 0; k < n; ++k) {
    const double u1 = u[3 * k], u2 = u[3 * k + 1], u3 = u[3 * k + 2];
    const double qw = sqrt(1.0 - u1) * sin(2.0 * M_PI * u2), qx = sqrt(1.0 - u1) * cos(2.0 * M_PI * u2);
    const double qy = sqrt(u1) * sin(2.0 * M_PI * u3), qz = sqrt(u1) * cos(2.0 * M_PI * u3);
    if (fabs(qw) < 1e-8) {
      rho[3 * k] = qx * 1e9;
      rho[3 * k + 1] = qy * 1e9;
      rho[3 * k + 2] = qz * 1e9;
    } else {
      rho[3 * k] = qx / qw;
      rho[3 * k + 1] = qy / qw;
      rho[3 * k + 2] = qz / qw;
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Maximum-stress extraction (App. C): masked (normalised) Gaussian smoothing of the von   */
/* Mises field and the largest 26-neighbourhood local maximum in the solid                 */
/* ------------------------------------------------------------------------------------ */

/* w: 2r+1 one-dimensional weights exp(-x^2 / (2 s^2)), x = -r..r, normalised to sum 1. */
void or_gauss_weights(double s, int r, double *w) {
  double sum = 0.0;
  for (int x = -r; x <= r; ++x) {
    w[x + r] = exp(-(double)(x * x) / (2.0 * s * s));
    sum += w[x + r];
  }
  for (int x = -r; x <= r; ++x) w[x + r] /= sum;
}

/* smooth = (G * (vm M)) / (G * M) with M = 1 in solid voxels (phase >= 0), 0 in pores, G the
 * separable periodic Gaussian with weights w (2r+1 taps); 0 where G * M = 0.  Both sums run over
 * dz, dy, dx (outer to inner) with the weight (w[dz] * w[dy]) * w[dx].  Then a voxel is a hotspot
 * when it is solid and no 26-neighbour has a larger smoothed value (App. C's regional maxima in
 * the solid); with solid_only, pore neighbours are left out of that comparison.  Returns the
 * largest hotspot value (0 if none) and its voxel in *at (lowest id among equal values). */
double or_hotspot(int nx, int ny, int nz, const int32_t *phase, const double *vm, const double *w, int r,
                  int solid_only, double *smooth, int64_t *at) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        double num = 0.0, den = 0.0;
        for (int dz = -r; dz <= r; ++dz)
          for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
              const int64_t u = wrap(i + dx, nx) + nx * (wrap(j + dy, ny) + ny * wrap(k + dz, nz));
              const double wt = (w[dz + r] * w[dy + r]) * w[dx + r];
              if (phase[u] >= 0) {
                num = num + wt * vm[u];
                den = den + wt;
              }
            }
        smooth[i + nx * (j + ny * k)] = den > 0.0 ? num / den : 0.0;
      }
  double best = 0.0;
  int64_t arg = -1;
  for (int64_t v = 0; v < N; ++v) {
    if (phase[v] < 0) continue;
    const int64_t i = v % nx, j = (v / nx) % ny, k = v / ((int64_t)nx * ny);
    int is_max = 1;
    for (int dz = -1; dz <= 1 && is_max; ++dz)
      for (int dy = -1; dy <= 1 && is_max; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int64_t u = wrap(i + dx, nx) + nx * (wrap(j + dy, ny) + ny * wrap(k + dz, nz));
          if (solid_only && phase[u] < 0) continue;
          if (smooth[u] > smooth[v]) { is_max = 0; break; }
        }
    if (is_max && (arg < 0 || smooth[v] > best)) { best = smooth[v]; arg = v; }
  }
  if (at) *at = arg;
  return arg < 0 ? 0.0 : best;
}
