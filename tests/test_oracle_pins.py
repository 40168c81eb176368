"""Pins of the FP64 CPU oracle to the paper and to mathematics (no GPU).

Every check compares the oracle with something other than itself: closed forms, invariants,
an independent library routine (matrix exponential, dense eigen/least squares), brute force
on tiny grids, or values printed in ELAS3D-Xtal (arXiv 2602.07354).
"""
import os

import numpy as np
import pytest
from scipy.linalg import expm

from paper_2602_07354_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_C(rng):
    c12 = rng.uniform(80, 140)
    return c12 + rng.uniform(40, 120), c12, rng.uniform(40, 130)


def _skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


# ---------------------------------------------------------------- constitutive (Sec. 2.1.1)
def test_iso_stiffness_recovers_E_nu(oracle):
    # Eqs. 2-3: inverting C must give the compliance of an isotropic solid: 1/S11 = E, -S12/S11 = nu
    for E, nu in [(200.0, 0.3), (194.0, 0.2934), (400.0, 0.25), (1.0, 0.0)]:
        S = np.linalg.inv(oracle.iso_stiffness(E, nu))
        assert np.isclose(1 / S[0, 0], E, rtol=1e-13)
        assert np.isclose(-S[0, 1] / S[0, 0], nu, rtol=1e-12, atol=1e-15)
        assert np.isclose(1 / S[3, 3], E / (2 * (1 + nu)), rtol=1e-13)  # engineering shear compliance


def test_rodrigues_matches_matrix_exponential(oracle):
    # rho = tan(theta/2) n (Sec. 2.2.3) must be the rotation exp(theta [n]x)
    rng = np.random.default_rng(0)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        theta = rng.uniform(-3.0, 3.0)
        R = oracle.rodrigues_to_R(np.tan(theta / 2) * n)
        assert np.allclose(R, expm(theta * _skew(n)), atol=1e-13)
    R = oracle.rodrigues_to_R([0.0, 0.0, 1.0])  # 90 degrees about z
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    R = oracle.rodrigues_to_R([1e9, 0.0, 0.0])  # the |q_w| < 1e-8 guard of Algorithm 6: 180 deg
    assert np.allclose(R, np.diag([1, -1, -1]), atol=3e-9)  # theta = pi - 2e-9


def test_rotation_invariances(oracle):
    rng = np.random.default_rng(1)
    Ciso = oracle.iso_stiffness(210.0, 0.29)
    Ccub = oracle.cubic_stiffness(204.6, 137.7, 126.2)
    for _ in range(5):
        R = oracle.rodrigues_to_R(rng.normal(size=3))
        assert np.allclose(oracle.rotate_stiffness(Ciso, R), Ciso, atol=1e-11)
    for axis in np.eye(3):  # cubic symmetry: 90 degree turns about the cube axes
        R = oracle.rodrigues_to_R(np.tan(np.pi / 4) * axis)
        assert np.allclose(oracle.rotate_stiffness(Ccub, R), Ccub, atol=1e-11)
    # composition: rotate(rotate(C, R1), R2) == rotate(C, R2 R1)
    R1 = oracle.rodrigues_to_R(rng.normal(size=3))
    R2 = oracle.rodrigues_to_R(rng.normal(size=3))
    a = oracle.rotate_stiffness(oracle.rotate_stiffness(Ccub, R1), R2)
    assert np.allclose(a, oracle.rotate_stiffness(Ccub, R2 @ R1), atol=1e-10)
    # the two tensor invariants C_iijj and C_ijij
    Cr = oracle.rotate_stiffness(Ccub, R1)
    for C in (Ccub, Cr):
        pass
    inv1 = lambda C: C[:3, :3].sum()
    inv2 = lambda C: np.trace(C[:3, :3]) + 2 * np.trace(C[3:, 3:])
    assert np.isclose(inv1(Cr), inv1(Ccub), rtol=1e-13)
    assert np.isclose(inv2(Cr), inv2(Ccub), rtol=1e-13)


def test_rotation_direction_cubic_young_modulus(oracle):
    # Textbook cubic crystal: 1/E(n) = S11 - 2 (S11 - S12 - S44/2)(n1^2 n2^2 + n2^2 n3^2 + n3^2 n1^2).
    # With rho the crystal->sample active rotation, sample axis x is crystal direction R^T e_x.
    C = oracle.cubic_stiffness(204.6, 137.7, 126.2)
    S = np.linalg.inv(C)
    S11, S12, S44 = S[0, 0], S[0, 1], S[3, 3]
    rng = np.random.default_rng(2)
    for _ in range(10):
        R = oracle.rodrigues_to_R(rng.normal(size=3))
        Sg = np.linalg.inv(oracle.rotate_stiffness(C, R))
        n = R.T @ np.array([1.0, 0, 0])
        J = n[0] ** 2 * n[1] ** 2 + n[1] ** 2 * n[2] ** 2 + n[2] ** 2 * n[0] ** 2
        assert np.isclose(Sg[0, 0], S11 - 2 * (S11 - S12 - S44 / 2) * J, rtol=1e-12)


def _orientation_average(oracle, C):
    # exact-to-roundoff Haar average over SO(3): ZYZ Euler angles, trapezoid in alpha/gamma
    # (exact for the degree-4 trigonometric integrand) and Gauss-Legendre in beta.
    na = 8
    xs, ws = np.polynomial.legendre.leggauss(24)
    betas = (xs + 1) * np.pi / 2
    wb = ws * np.pi / 2 * np.sin(betas) / 2.0
    acc = np.zeros((6, 6))
    for al in np.arange(na) * 2 * np.pi / na:
        for ga in np.arange(na) * 2 * np.pi / na:
            for be, w in zip(betas, wb):
                Rz1 = expm(al * _skew([0, 0, 1]))
                Ry = expm(be * _skew([0, 1, 0]))
                Rz2 = expm(ga * _skew([0, 0, 1]))
                acc += w * oracle.rotate_stiffness(C, Rz1 @ Ry @ Rz2) / na ** 2
    return acc


def test_orientation_average_gives_table4_moduli(oracle):
    # Sec. 3.2 / table of material parameters: every row has K = (C11+2C12)/3 = 156.64 GPa and
    # its stated Zener ratio; the baseline row (case 3) has G = 75.08 GPa.  The Haar average of
    # the rotated tensor is the Voigt isotropic tensor (C11 = K + 4G/3, C12 = K - 2G/3, C44 = G).
    rows = np.loadtxt(os.path.join(GOLDEN, "table4_materials.txt"))
    for case, A, c11, c12, c44 in rows:
        avg = _orientation_average(oracle, oracle.cubic_stiffness(c11, c12, c44))
        K = avg[:3, :3].sum() / 9
        G = avg[3, 3]
        assert np.isclose(K, 156.64, atol=0.011), (case, K)
        assert np.isclose(2 * c44 / (c11 - c12), A, atol=2e-4)
        assert np.allclose(avg[:3, :3], (K - 2 * G / 3) + np.eye(3) * 2 * G, atol=1e-9)
        assert np.allclose(avg[3:, 3:], G * np.eye(3), atol=1e-9)
        if case == 3:
            assert np.isclose(G, 75.08, atol=0.005)


# ---------------------------------------------------------------- element stiffness
def _corner_signs():
    return np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1] for a in range(8)], float)


def test_element_stiffness_structure(oracle):
    rng = np.random.default_rng(3)
    C = oracle.rotate_stiffness(oracle.cubic_stiffness(*_rand_C(rng)), oracle.rodrigues_to_R(rng.normal(size=3)))
    K = oracle.element_stiffness(C, 0)
    assert np.allclose(K, K.T, atol=1e-12 * np.abs(K).max())
    ev = np.linalg.eigvalsh(K)
    assert ev.min() > -1e-12 * ev.max()
    assert (ev < 1e-10 * ev.max()).sum() == 6  # 3 translations + 3 infinitesimal rotations
    X = (_corner_signs() + 1) / 2
    for t in np.eye(3):  # translations
        assert np.abs(K @ np.tile(t, 8)).max() < 1e-12 * np.abs(K).max()
    for ax in np.eye(3):  # rotations u = ax x X
        u = np.cross(ax, X).ravel()
        assert np.abs(K @ u).max() < 1e-12 * np.abs(K).max()
    # both quadratures are exact for this integrand, so they agree to round-off
    assert np.allclose(K, oracle.element_stiffness(C, 1), atol=1e-12 * np.abs(K).max())


def test_element_stiffness_affine_closed_form(oracle):
    # (K_e Ebar)_a = sigma . n_a with sigma = C:E and n_a = int grad N_a dV = s_a / 4;
    # 1/2 Ebar^T K_e Ebar = 1/2 E:C:E (unit voxel volume).
    rng = np.random.default_rng(4)
    C = oracle.rotate_stiffness(oracle.cubic_stiffness(*_rand_C(rng)), oracle.rodrigues_to_R(rng.normal(size=3)))
    K = oracle.element_stiffness(C, 0)
    e6 = rng.normal(size=6) * 1e-3
    E = np.array([[e6[0], e6[5], e6[4]], [e6[5], e6[1], e6[3]], [e6[4], e6[3], e6[2]]])
    X = (_corner_signs() + 1) / 2
    Ebar = (X @ E.T).ravel()
    ev = np.array([e6[0], e6[1], e6[2], 2 * e6[3], 2 * e6[4], 2 * e6[5]])
    s6 = C @ ev
    sig = np.array([[s6[0], s6[5], s6[4]], [s6[5], s6[1], s6[3]], [s6[4], s6[3], s6[2]]])
    f = (K @ Ebar).reshape(8, 3)
    expect = (_corner_signs() / 4) @ sig.T
    assert np.allclose(f, expect, atol=1e-14 * np.abs(s6).max() * 10)
    assert np.isclose(0.5 * Ebar @ K @ Ebar, 0.5 * ev @ C @ ev, rtol=1e-12)


def test_element_stiffness_higher_mode_energies(oracle):
    # Closed-form energies of the non-affine trilinear modes, valid for any Voigt C:
    #   u_x = (x-1/2)(y-1/2):         u^T K u = (C11 + C66)/12
    #   u_x = (x-1/2)(y-1/2)(z-1/2):  u^T K u = (C11 + C55 + C66)/144
    # (a dropped or mis-signed bilinear term in B changes these)
    rng = np.random.default_rng(5)
    C = oracle.rotate_stiffness(oracle.cubic_stiffness(*_rand_C(rng)), oracle.rodrigues_to_R(rng.normal(size=3)))
    K = oracle.element_stiffness(C, 0)
    X = (_corner_signs() + 1) / 2
    u = np.zeros((8, 3))
    u[:, 0] = (X[:, 0] - 0.5) * (X[:, 1] - 0.5)
    assert np.isclose(u.ravel() @ K @ u.ravel(), (C[0, 0] + C[5, 5]) / 12, rtol=1e-12)
    u[:, 0] = (X[:, 0] - 0.5) * (X[:, 1] - 0.5) * (X[:, 2] - 0.5)
    assert np.isclose(u.ravel() @ K @ u.ravel(), (C[0, 0] + C[4, 4] + C[5, 5]) / 144, rtol=1e-12)
    u[:, 0] = 0
    u[:, 2] = (X[:, 1] - 0.5) * (X[:, 0] - 0.5)  # u_z = (x-1/2)(y-1/2): eps_zz = 0, g_yz = x-1/2, g_xz = y-1/2
    assert np.isclose(u.ravel() @ K @ u.ravel(), (C[3, 3] + C[4, 4]) / 12, rtol=1e-12)


# ---------------------------------------------------------------- global operator
def _problem(oracle, dims, n_phases=3, seed=0, pore_prob=0.15):
    ms = synth.random_problem(dims, n_phases, np.random.default_rng(seed), pore_prob=pore_prob)
    return oracle.Problem.from_micro(ms)


@pytest.mark.parametrize("dims", [(2, 2, 2), (3, 3, 3), (4, 3, 2), (4, 4, 4)])
def test_operator_dense_symmetric_psd(oracle, dims):
    p = _problem(oracle, dims, seed=sum(dims))
    A = p.dense()
    rng = np.random.default_rng(7)
    u = rng.normal(size=3 * p.N)
    assert np.allclose(p.apply(u), A @ u, atol=1e-12 * np.abs(A).max())
    assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-11 * ev.max()
    for c in range(3):  # rigid translations are in the null space (periodic cell)
        t = np.zeros((3, p.N))
        t[c] = 1
        assert np.abs(A @ t.ravel()).max() < 1e-11 * np.abs(A).max()
    # point-block Jacobi (Eq. 9): the stored inverse is the inverse of A's 3x3 diagonal block
    Minv = p.jacobi()
    N = p.N
    for m in range(N):
        blk = A[np.ix_([m, N + m, 2 * N + m], [m, N + m, 2 * N + m])]
        if np.all(blk == 0):
            assert np.allclose(Minv[m], np.eye(3))
        else:
            assert np.allclose(Minv[m] @ blk, np.eye(3), atol=1e-10)
    # sampled-node gather equals the scatter product
    sel = rng.choice(N, size=min(N, 11), replace=False)
    assert np.allclose(p.apply_nodes(u, sel), p.apply(u).reshape(3, N)[:, sel].T, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("dims", [(2, 2, 2), (3, 4, 5), (6, 5, 4)])
def test_operator_and_rhs_are_energy_derivatives(oracle, dims):
    # Eqs. 7-8: Pi(w) = C + 1/2 w^T A w + b^T w, with Pi evaluated element by element.
    # Central differences of a quadratic are exact, so A v and b come out of Pi alone.
    p = _problem(oracle, dims, seed=11 + sum(dims))
    rng = np.random.default_rng(8)
    e6 = rng.normal(size=6) * 1e-3
    w = rng.normal(size=3 * p.N) * 1e-3
    v = rng.normal(size=3 * p.N) * 1e-3
    b = p.rhs(e6)
    Pi = lambda x: p.energy(e6, x)
    dd = (Pi(w + v) - Pi(w - v)) / 2.0
    assert np.isclose(dd, v @ (p.apply(w) + b), rtol=1e-9, atol=1e-14)
    zero = np.zeros(6)
    assert np.isclose(p.energy(zero, w), 0.5 * w @ p.apply(w), rtol=1e-12)


def test_rhs_is_stress_flux_through_voxel_faces(oracle):
    # b_m = sum over the 8 voxels around m of sigma_e . n_a, with n_a = s_a/4 (affine closed form)
    p = _problem(oracle, (5, 4, 3), seed=3)
    e6 = np.array([1e-3, -2e-4, 3e-4, 1e-4, -5e-4, 2e-4])
    b = p.rhs(e6).reshape(3, p.N)
    ev = e6 * np.array([1, 1, 1, 2, 2, 2])
    nx, ny, nz = p.dims
    s = _corner_signs()
    expect = np.zeros((3, p.N))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = i + nx * (j + ny * k)
                if p.phase[e] < 0:
                    continue
                s6 = p.C_global[p.phase[e]] @ ev
                sig = np.array([[s6[0], s6[5], s6[4]], [s6[5], s6[1], s6[3]], [s6[4], s6[3], s6[2]]])
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
                    m = (i + ax) % nx + nx * (((j + ay) % ny) + ny * ((k + az) % nz))
                    expect[:, m] += sig @ (s[a] / 4)
    assert np.allclose(b, expect, atol=1e-16 + 1e-13 * np.abs(expect).max())


# ---------------------------------------------------------------- solve (Algorithm 2)
def _remove_translation(p, w, oracle):
    mask = oracle.solid_node_mask(p)
    W = w.reshape(3, p.N)
    return (W[:, mask] - W[:, mask].mean(axis=1, keepdims=True)).ravel()


@pytest.mark.parametrize("dims,seed", [((3, 3, 3), 1), ((4, 4, 4), 2), ((2, 3, 4), 3)])
def test_pcg_matches_dense_direct_solve(oracle, dims, seed):
    p = _problem(oracle, dims, seed=seed, pore_prob=0.1)
    e6 = np.array([2e-4, -1e-4, 1e-3, 3e-4, 0.0, -2e-4])
    r = p.pcg(e6, 1e-13, 500)
    assert r["outcome"] == oracle.CONVERGED
    A = p.dense()
    w_direct = np.linalg.lstsq(A, -r["b"], rcond=1e-13)[0]
    # solution is unique up to translations of solid islands: compare strains and stresses
    s1, _, m1 = p.stress(e6, r["w"])
    s2, _, m2 = p.stress(e6, w_direct)
    assert np.allclose(s1, s2, atol=1e-10 * np.abs(s2).max())
    assert np.allclose(m1, m2, atol=1e-10 * np.abs(m2).max())
    assert p.true_relres(e6, r["w"]) < 1e-11


def test_homogeneous_anisotropic_cube_is_affine(oracle):
    # a homogeneous cell under any applied strain has b = 0, w = 0 and uniform eps = E, sigma = C E
    rng = np.random.default_rng(9)
    ms = synth.Microstructure(6, 5, 4, np.zeros(120, np.int32), synth.cubic_mat(204.6, 137.7, 126.2)[None],
                              rng.normal(size=(1, 3)))
    p = oracle.Problem.from_micro(ms)
    e6 = rng.normal(size=6) * 1e-3
    b = p.rhs(e6)
    ev = e6 * np.array([1, 1, 1, 2, 2, 2])
    assert np.abs(b).max() < 1e-13 * np.abs(p.C_global[0] @ ev).max()
    r = p.pcg(e6, 1e-10, 100)
    assert r["iters"] <= 1
    eps = p.strain(e6, r["w"])
    assert np.allclose(eps, e6[:, None], atol=1e-15)
    s, vm, macro = p.stress(e6, r["w"])
    assert np.allclose(s, (p.C_global[0] @ ev)[:, None], rtol=1e-10, atol=1e-14)


def test_mean_strain_equals_applied_strain(oracle):
    # the periodic fluctuation averages to zero: <eps> = E for ANY periodic w
    p = _problem(oracle, (5, 6, 7), seed=4)
    rng = np.random.default_rng(10)
    e6 = rng.normal(size=6) * 1e-3
    eps = p.strain(e6, rng.normal(size=3 * p.N))
    assert np.allclose(eps.mean(axis=1), e6, atol=1e-15)


def test_energy_monotone_hill_mandel_and_bounds(oracle):
    ms = synth.polycrystal(10, 8, pore_frac=0.0, seed=3)
    p = oracle.Problem.from_micro(ms)
    e6 = np.array([0.0, 0.0, 1e-3, 0.0, 0.0, 0.0])
    energies = [p.energy(e6, p.pcg(e6, 0.0, k)["w"]) for k in range(0, 12)]
    assert all(b <= a * (1 + 1e-13) for a, b in zip(energies, energies[1:]))
    r = p.pcg(e6, 1e-12, 1000)
    assert r["outcome"] == oracle.CONVERGED
    _, _, macro = p.stress(e6, r["w"])
    ev = e6 * np.array([1, 1, 1, 2, 2, 2])
    # Hill-Mandel: Pi(w*) = 1/2 V E:sigma_bar (V = number of unit voxels)
    assert np.isclose(p.energy(e6, r["w"]), 0.5 * p.N * ev @ macro, rtol=1e-10)
    # Voigt (affine trial field) and Reuss (uniform stress) bounds on E:C_eff:E
    Cs = p.C_global[p.phase]
    voigt = np.mean(np.einsum("i,nij,j->n", ev, Cs, ev))
    S_mean = np.linalg.inv(Cs).mean(axis=0)
    reuss = ev @ np.linalg.inv(S_mean) @ ev
    eff = ev @ macro
    assert reuss * (1 - 1e-9) <= eff <= voigt * (1 + 1e-12)
    assert eff < voigt * (1 - 1e-4)  # a polycrystal is strictly softer than its Voigt bound


@pytest.mark.parametrize("precond", ["none", "scalar"])
def test_preconditioner_variants_match_dense_direct_solve(oracle, precond):
    # the Table 4 comparison solvers (plain CG, and point Jacobi) reach the dense solution too
    p = _problem(oracle, (4, 3, 4), seed=21, pore_prob=0.1)
    e6 = np.array([1e-3, 2e-4, -3e-4, 0.0, 1e-4, 5e-4])
    r = p.pcg(e6, 1e-13, 4000, precond=precond)
    assert r["outcome"] == oracle.CONVERGED
    w_direct = np.linalg.lstsq(p.dense(), -r["b"], rcond=1e-13)[0]
    s1 = p.stress(e6, r["w"])[0]
    s2 = p.stress(e6, w_direct)[0]
    assert np.allclose(s1, s2, atol=1e-10 * np.abs(s2).max())


def test_scalar_jacobi_is_the_diagonal_of_the_block_preconditioner(oracle):
    # M = diag(A): z = g / A_ii, with A_ii the diagonal of the dense operator
    p = _problem(oracle, (3, 4, 3), seed=22, pore_prob=0.15)
    e6 = np.array([0.0, 0.0, 1e-3, 0.0, 0.0, 0.0])
    A = p.dense()
    b = p.rhs(e6)
    d = np.diag(A).copy()
    d[d == 0.0] = 1.0
    # one iteration of Algorithm 2 from w = 0 with M = diag(A): lambda = (z.g)/(z.A z), w = -lambda z
    z = b / d
    lam = (z @ b) / (z @ (A @ z))
    r = p.pcg(e6, 0.0, 1, precond="scalar")
    assert np.allclose(r["w"], -lam * z, rtol=1e-12, atol=1e-14 * np.abs(lam * z).max())


def test_unpreconditioned_cg_reaches_same_solution(oracle):
    p = _problem(oracle, (4, 4, 4), seed=12, pore_prob=0.05)
    e6 = np.array([0.0, 1e-3, 0.0, 0.0, 2e-4, 0.0])
    r1 = p.pcg(e6, 1e-12, 2000)
    r2 = p.pcg(e6, 1e-12, 4000, precond=False)
    s1 = p.stress(e6, r1["w"])[0]
    s2 = p.stress(e6, r2["w"])[0]
    assert np.allclose(s1, s2, atol=1e-9 * np.abs(s1).max())
    assert r1["iters"] < r2["iters"]


def test_zero_rhs_and_paper_guard(oracle):
    p = _problem(oracle, (3, 3, 3), seed=5)
    r = p.pcg(np.zeros(6), 1e-8, 50)
    assert r["iters"] == 0 and r["outcome"] == oracle.CONVERGED and not r["w"].any()
    # the paper's absolute |hAh| < 1e-14 stops a GPa-unit solve long before tol 1e-10
    ms = synth.eshelby_inclusion(12, 3.0)
    q = oracle.Problem.from_micro(ms)
    e6 = np.array([1e-3, 0, 0, 0, 0, 0])
    r_paper = q.pcg(e6, 1e-10, 500, paper_guard=True)
    r_rel = q.pcg(e6, 1e-10, 500)
    assert r_rel["outcome"] == oracle.CONVERGED
    assert r_paper["outcome"] == oracle.BREAKDOWN and r_paper["iters"] < r_rel["iters"]


def test_jacobi_identity_for_void_nodes(oracle):
    phase = np.full(27, -1, np.int32)
    phase[0] = 0
    ms = synth.Microstructure(3, 3, 3, phase, synth.iso_mat(200.0, 0.3)[None], None)
    p = oracle.Problem.from_micro(ms)
    M = p.jacobi()
    mask = oracle.solid_node_mask(p)
    assert mask.sum() == 8
    assert np.allclose(M[~mask], np.eye(3))


# ---------------------------------------------------------------- stress
def test_stress_von_mises_and_pores(oracle):
    p = _problem(oracle, (4, 4, 4), seed=6, pore_prob=0.3)
    rng = np.random.default_rng(11)
    e6 = rng.normal(size=6) * 1e-3
    w = rng.normal(size=3 * p.N) * 1e-4
    s, vm, macro = p.stress(e6, w)
    eps = p.strain(e6, w)
    pores = p.phase < 0
    assert np.all(s[:, pores] == 0) and np.all(vm[pores] == 0)
    for e in np.flatnonzero(~pores)[:10]:
        ev = eps[:, e] * np.array([1, 1, 1, 2, 2, 2])
        assert np.allclose(s[:, e], p.C_global[p.phase[e]] @ ev, rtol=1e-12, atol=1e-15)
        sig = np.array([[s[0, e], s[5, e], s[4, e]], [s[5, e], s[1, e], s[3, e]], [s[4, e], s[3, e], s[2, e]]])
        dev = sig - np.trace(sig) / 3 * np.eye(3)
        assert np.isclose(vm[e], np.sqrt(1.5 * (dev * dev).sum()), rtol=1e-12)
    assert np.allclose(macro, s.mean(axis=1), rtol=1e-13, atol=1e-18)


# ---------------------------------------------------------------- Eshelby (approximate physics pin)
def test_eshelby_inclusion_mori_tanaka(oracle):
    # 20^3 cell, isotropic matrix E=200 nu=0.3, centred sphere r=5 of E=400 nu=0.25, E11 = 1e-3.
    # Eshelby's interior strain of a spherical inclusion, Mori-Tanaka-corrected for the
    # voxelised volume fraction, must match the voxel mean inclusion strain within a few percent
    # (staircase boundary, simple-cubic periodic arrangement and finite fraction make this
    # approximate: the voxel mean sits 5.3% above Mori-Tanaka at 20^3, 4.2% at 30^3, 3.6% at 40^3).
    ms = synth.eshelby_inclusion()
    p = oracle.Problem.from_micro(ms)
    e6 = np.array([1e-3, 0, 0, 0, 0, 0])
    r = p.pcg(e6, 1e-10, 2000)
    assert r["outcome"] == oracle.CONVERGED
    eps = p.strain(e6, r["w"])
    inc = p.phase == 1
    f = inc.mean()
    E0, nu0, E1, nu1 = 200.0, 0.3, 400.0, 0.25
    K0, G0 = E0 / (3 * (1 - 2 * nu0)), E0 / (2 * (1 + nu0))
    K1, G1 = E1 / (3 * (1 - 2 * nu1)), E1 / (2 * (1 + nu1))
    al = (1 + nu0) / (3 * (1 - nu0))
    be = 2 * (4 - 5 * nu0) / (15 * (1 - nu0))
    Tv = 1 / (1 + al * (K1 / K0 - 1))
    Td = 1 / (1 + be * (G1 / G0 - 1))
    vol, dev_xx, dev_yy = 1e-3 / 3, 1e-3 - 1e-3 / 3, -1e-3 / 3
    cv = Tv / ((1 - f) + f * Tv)
    cd = Td / ((1 - f) + f * Td)
    exx = cv * vol + cd * dev_xx
    eyy = cv * vol + cd * dev_yy
    mean_xx = eps[0, inc].mean()
    mean_yy = eps[1, inc].mean()
    assert abs(mean_xx - exx) < 0.08 * abs(exx), (mean_xx, exx)
    assert 0 < mean_yy < 2 * eyy, (mean_yy, eyy)  # small lateral difference of two ~2.4e-4 terms
    # inclusion is stiffer: its axial strain is below the applied one, the matrix's above
    assert mean_xx < 1e-3 < eps[0, ~inc].mean()


# ---- microstructure generator (Sec. 2.2, Algorithms 4 and 5) ---------------------------------
def test_grain_assignment_is_the_periodic_nearest_seed(oracle):
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(31)
    dims = (12, 10, 9)
    seeds = rng.random((15, 3)) * np.array(dims)
    phase = oracle.assign_grains(dims, seeds)
    k, j, i = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], 1) + 0.5
    _, ref = cKDTree(seeds, boxsize=dims).query(X)
    assert np.array_equal(phase, ref.astype(np.int32))


def test_sampled_grain_assignment_matches_the_k_d_tree(oracle):
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(34)
    dims = (40, 30, 50)
    seeds = rng.random((200, 3)) * np.array(dims)
    vox = rng.choice(np.prod(dims), size=500, replace=False)
    X = np.stack([vox % 40, (vox // 40) % 30, vox // 1200], 1) + 0.5
    _, ref = cKDTree(seeds, boxsize=dims).query(X)
    assert np.array_equal(oracle.assign_voxels(dims, seeds, vox), ref.astype(np.int32))


def test_uniform_grain_weights_stretch_the_tessellation(oracle):
    # equal (rt, rl) for every grain: the assignment is the plain Voronoi diagram of the grid
    # with z scaled by rt/rl (a stretched, still periodic, nearest-seed problem)
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(32)
    dims = (9, 8, 12)
    seeds = rng.random((11, 3)) * np.array(dims)
    rt, rl = 1.0, 2.5
    phase = oracle.assign_grains(dims, seeds, np.tile([rt, rl], (11, 1)))
    s = np.array([1.0, 1.0, rt / rl])
    k, j, i = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    X = (np.stack([i.ravel(), j.ravel(), k.ravel()], 1) + 0.5) * s
    _, ref = cKDTree(seeds * s, boxsize=np.array(dims) * s).query(X)
    assert np.array_equal(phase, ref.astype(np.int32))
    # and scaling every weight by 2 (exact in binary) changes nothing
    assert np.array_equal(oracle.assign_grains(dims, seeds, np.tile([2 * rt, 2 * rl], (11, 1))), phase)


def _pore(c, axes, R=np.eye(3)):
    return np.concatenate([np.asarray(c, float), np.asarray(axes, float), np.asarray(R, float).ravel()])


@pytest.mark.parametrize("r,count", [(2.0, 33), (2.5, 81), (3.0, 123)])
def test_sphere_pores_hold_the_lattice_points_of_the_ball(oracle, r, count):
    # voxel centres within radius r of a voxel centre: the integer points of a ball (1 + 6 + 12 +
    # 8 + 6 = 33 for r = 2, 81 for r^2 = 6.25, 123 for r = 3), also when the ball wraps around
    dims = (11, 12, 13)
    for c in ([5.5, 6.5, 6.5], [0.5, 11.5, 0.5]):
        phase = np.zeros(np.prod(dims), np.int32)
        assert oracle.stamp_pores(dims, _pore(c, [r, r, r])[None], phase) == count


def test_pore_rotations(oracle):
    dims = (16, 16, 16)
    c = [8.5, 8.5, 8.5]
    # a sphere is the same under any rotation (radius 2.5: no lattice point on the surface)
    rng = np.random.default_rng(33)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    a = np.zeros(16 ** 3, np.int32)
    b = np.zeros(16 ** 3, np.int32)
    oracle.stamp_pores(dims, _pore(c, [2.5] * 3)[None], a)
    oracle.stamp_pores(dims, _pore(c, [2.5] * 3, R)[None], b)
    assert np.array_equal(a, b)
    # an ellipsoid turned by 90 degrees about z is the one with its x and y semi-axes swapped
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    a[:] = 0
    b[:] = 0
    na = oracle.stamp_pores(dims, _pore(c, [4.3, 2.2, 1.7], Rz)[None], a)
    nb = oracle.stamp_pores(dims, _pore(c, [2.2, 4.3, 1.7])[None], b)
    assert na == nb and np.array_equal(a, b) and na > 0


# ---- maximum-stress extraction (App. C) --------------------------------------------------------
def test_gaussian_weights(oracle):
    w = oracle.gauss_weights(0.4, 1)
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs(w[0] / w[1] - np.exp(-1.0 / (2 * 0.16))) < 1e-15 and w[0] == w[2]


def test_normalised_convolution_keeps_a_constant_field(oracle):
    # a constant stress in the solid stays constant at every voxel that sees solid, pores or not
    rng = np.random.default_rng(41)
    dims = (9, 8, 7)
    phase = np.where(rng.random(9 * 8 * 7) < 0.3, -1, 0).astype(np.int32)
    vm = np.where(phase >= 0, 0.37, 0.0)
    best, at, sm = oracle.hotspot(dims, phase, vm)
    assert np.allclose(sm[sm != 0], 0.37, rtol=1e-14, atol=0)
    assert abs(best - 0.37) < 1e-14 and phase[at] >= 0


def test_smoothed_impulse_is_the_product_of_gaussians(oracle):
    dims = (7, 7, 7)
    phase = np.zeros(343, np.int32)
    vm = np.zeros(343)
    vm[3 + 7 * (3 + 7 * 3)] = 2.0
    best, at, sm = oracle.hotspot(dims, phase, vm, s=0.7, r=2)
    g = np.exp(-np.arange(-2, 3) ** 2 / (2 * 0.49))
    g /= g.sum()
    ref = 2.0 * g[:, None, None] * g[None, :, None] * g[None, None, :]  # (dz, dy, dx) around the centre
    assert np.allclose(sm.reshape(7, 7, 7)[1:6, 1:6, 1:6], ref, rtol=1e-13, atol=0)
    assert at == 3 + 7 * (3 + 7 * 3) and abs(best - 2.0 * g[2] ** 3) < 1e-15


def test_pore_neighbours_can_outrank_the_solid_surface(oracle):
    # a pore voxel whose six face neighbours carry a high stress: its smoothed value (an average of
    # those six) exceeds theirs (each averaged with its low-stress surroundings), so with every
    # neighbour competing none of the six is a hotspot; with solid neighbours only, the largest
    # hotspot is the largest smoothed value in the solid
    n = 5
    phase = np.zeros(n ** 3, np.int32)
    vm = np.full(n ** 3, 0.1)
    lin = lambda i, j, k: i + n * (j + n * k)
    phase[lin(2, 2, 2)] = -1
    vm[lin(2, 2, 2)] = 0.0
    faces = [lin(1, 2, 2), lin(3, 2, 2), lin(2, 1, 2), lin(2, 3, 2), lin(2, 2, 1), lin(2, 2, 3)]
    vm[faces] = 1.0
    best_all, at_all, sm = oracle.hotspot((n, n, n), phase, vm)
    best_sol, at_sol, sm2 = oracle.hotspot((n, n, n), phase, vm, solid_only=True)
    assert np.array_equal(sm, sm2)
    assert sm[lin(2, 2, 2)] > sm[faces].max()
    assert at_all not in faces and best_all < 0.2
    assert at_sol == min(faces) and best_sol == sm[phase >= 0].max()


def test_solid_only_hotspot_is_the_solid_maximum(oracle):
    rng = np.random.default_rng(43)
    for dims in ((9, 8, 7), (6, 11, 5)):
        N = int(np.prod(dims))
        phase = np.where(rng.random(N) < 0.25, -1, rng.integers(0, 3, N)).astype(np.int32)
        vm = np.where(phase >= 0, rng.random(N), 0.0)
        b_all, _, sm = oracle.hotspot(dims, phase, vm)
        b_sol, at, _ = oracle.hotspot(dims, phase, vm, solid_only=True)
        assert b_sol == sm[phase >= 0].max() and at == np.flatnonzero((sm == b_sol) & (phase >= 0))[0]
        assert b_all <= b_sol


# ---- grain seeding (Algorithm 3) and orientations (Algorithm 6) --------------------------------
def test_grain_count_fills_the_box_with_mean_cylinders(oracle):
    # N_g is the least count of cylinders of diameter mu_d and height mu_alpha mu_d whose volume
    # reaches the box; the cylinder's volume here comes from integrating its disc's chord length
    from scipy import integrate

    for lengths, mu_d, mu_a in (((100, 100, 100), 10.0, 2.0), ((64, 48, 80), 7.5, 3.18), ((200, 200, 200), 9.1, 1.0)):
        r = mu_d / 2.0
        disc, _ = integrate.quad(lambda x: 2.0 * np.sqrt(r * r - x * x), -r, r, epsabs=1e-13, epsrel=1e-13)
        vcyl = disc * mu_a * mu_d
        V = float(np.prod(lengths))
        n = oracle.grain_count(lengths, mu_d, mu_a)
        assert n * vcyl >= V * (1 - 1e-12) and (n - 1) * vcyl < V


def test_seed_grains_lognormal_moments_and_semi_axes(oracle):
    # the lognormal draws have the requested mean and standard deviation of the variate itself:
    # Gauss-Hermite quadrature over z ~ N(0, 1) of d(z) and d(z)^2 (exact for these smooth
    # integrands to far below the tolerance)
    from numpy.polynomial.hermite_e import hermegauss

    zq, wq = hermegauss(80)
    wq = wq / wq.sum()
    mu_d, sd_d, mu_a, sd_a = 55.0, 12.0, 3.18, 0.9
    z = np.stack([zq, zq], axis=1)
    u = np.zeros((zq.size, 3))
    seeds, semi = oracle.seed_grains([0, 0, 0], [10, 20, 30], mu_d, sd_d, mu_a, sd_a, z, u)
    d = 2.0 * semi[:, 0]
    alpha = semi[:, 1] / semi[:, 0]
    for v, mu, sd in ((d, mu_d, sd_d), (alpha, mu_a, sd_a)):
        m1 = float(wq @ v)
        m2 = float(wq @ (v * v))
        assert abs(m1 - mu) <= 1e-9 * mu
        assert abs(np.sqrt(m2 - m1 * m1) - sd) <= 1e-7 * sd
    assert np.all(seeds == 0.0)
    # seeds: the unit cube's corners and centre map onto the box's
    u = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5], [0.25, 0.75, 0.125]])
    seeds, _ = oracle.seed_grains([1.0, -2.0, 4.0], [11.0, 18.0, 36.0], 10, 1, 2, 0.5, np.zeros((3, 2)), u)
    assert np.array_equal(seeds, [[1.0, -2.0, 4.0], [6.0, 8.0, 20.0], [3.5, 13.0, 8.0]])


def _rho_of(rot):
    v = rot.as_rotvec()
    t = np.linalg.norm(v, axis=-1, keepdims=True)
    return np.where(t > 0, np.tan(t / 2) * v / np.where(t > 0, t, 1.0), 0.0)


def test_fibre_orientations_compose_spin_wobble_and_base(oracle):
    # R_total = R_spin R_wobble R_base rebuilt from scipy rotations (rotation vectors), its
    # Rodrigues vector tan(theta/2) n from scipy's rotation vector
    from scipy.spatial.transform import Rotation

    rng = np.random.default_rng(53)
    n = 300
    draws = np.stack([rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n), rng.normal(0, np.radians(12.5), n)], 1)
    for crystal in ((1.0, 0.0, 1.0), (1.0, 1.0, 1.0), (0.0, 0.0, 2.0)):
        rho = oracle.fiber_orientations(draws, crystal)
        c = np.asarray(crystal) / np.linalg.norm(crystal)
        v = np.cross(c, [0, 0, 1.0])
        base = Rotation.from_rotvec(np.arcsin(min(np.linalg.norm(v), 1.0)) * v / np.linalg.norm(v)) \
            if np.linalg.norm(v) > 1e-12 else Rotation.identity()
        spin = Rotation.from_rotvec(np.stack([np.zeros(n), np.zeros(n), draws[:, 0]], 1))
        axis = np.stack([np.cos(draws[:, 1]), np.sin(draws[:, 1]), np.zeros(n)], 1)
        wob = Rotation.from_rotvec(axis * draws[:, 2:3])
        ref = _rho_of(spin * wob * base)
        ok = np.abs((spin * wob * base).magnitude()) < np.radians(170)  # away from the half turn
        assert ok.sum() > n // 2
        assert np.max(np.abs(rho[ok] - ref[ok]) / (1 + np.abs(ref[ok]))) <= 1e-12
    # without spread the crystal axis lands exactly on X3, and the angle to X3 is |theta|
    rho = oracle.fiber_orientations(np.stack([draws[:, 0], draws[:, 1], np.zeros(n)], 1))
    c = np.array([1.0, 0.0, 1.0]) / np.sqrt(2.0)
    for r in rho[:40]:
        R = oracle.rodrigues_to_R(r)
        assert np.allclose(R @ c, [0, 0, 1], atol=1e-12)
    rho = oracle.fiber_orientations(draws)
    ang = np.array([np.arccos(np.clip((oracle.rodrigues_to_R(r) @ c)[2], -1, 1)) for r in rho])
    assert np.allclose(ang, np.abs(draws[:, 2]), atol=1e-7)


def test_random_orientations_are_shoemake_quaternions(oracle):
    from scipy.spatial.transform import Rotation

    rng = np.random.default_rng(54)
    u = rng.random((500, 3))
    rho = oracle.random_orientations(u)
    qw = np.sqrt(1 - u[:, 0]) * np.sin(2 * np.pi * u[:, 1])
    qv = np.stack([np.sqrt(1 - u[:, 0]) * np.cos(2 * np.pi * u[:, 1]), np.sqrt(u[:, 0]) * np.sin(2 * np.pi * u[:, 2]),
                   np.sqrt(u[:, 0]) * np.cos(2 * np.pi * u[:, 2])], 1)
    rot = Rotation.from_quat(np.concatenate([qv, qw[:, None]], 1))  # scalar-last
    ok = rot.magnitude() < np.radians(170)
    ref = _rho_of(rot)
    assert np.max(np.abs(rho[ok] - ref[ok]) / (1 + np.abs(ref[ok]))) <= 1e-12
    # the guard of a vanishing scalar part (a half turn): q_w = 0 exactly at u2 = 0
    g = oracle.random_orientations(np.array([[0.36, 0.0, 0.2]]))[0]
    assert np.array_equal(g, np.array([0.8, np.sqrt(0.36) * np.sin(0.4 * np.pi), np.sqrt(0.36) * np.cos(0.4 * np.pi)]) * 1e9)
    # Haar measure: the rotated crystal axes are uniform on the sphere (first and second moments)
    e = np.array([oracle.rodrigues_to_R(r) @ [0, 0, 1.0] for r in oracle.random_orientations(rng.random((4000, 3)))])
    assert np.all(np.abs(e.mean(0)) < 0.05)
    assert np.allclose(e.T @ e / len(e), np.eye(3) / 3, atol=0.03)
