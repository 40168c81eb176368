"""Pins of the analytic spherical-cavity field (tests/cavity.py) that the Eshelby-void GPU test
compares with: it must satisfy equilibrium, leave the cavity surface traction-free, tend to the
remote field, and reproduce the classical stress concentrations of a spherical cavity under
uniaxial tension (Timoshenko and Goodier: (27 - 15 nu) / (2 (7 - 5 nu)) at the equator,
-(3 + 15 nu) / (2 (7 - 5 nu)) at the pole) and of one under hydrostatic tension (1.5)."""
import numpy as np
import pytest

import cavity

MU, NU, A = 75.08, 0.2934, 1.3


def _rand_strain(rng):
    M = rng.normal(size=(3, 3))
    return 1e-3 * (M + M.T)


def _exterior_points(rng, n, rmin=1.05, rmax=4.0):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * (A * rng.uniform(rmin, rmax, size=(n, 1)))


def test_gradient_is_the_derivative_of_the_displacement():
    rng = np.random.default_rng(1)
    E = _rand_strain(rng)
    x = _exterior_points(rng, 50)
    h = 1e-6
    G = cavity.gradient(x, E, NU, A)
    for k in range(3):
        dx = np.zeros(3)
        dx[k] = h
        fd = (cavity.displacement(x + dx, E, NU, A) - cavity.displacement(x - dx, E, NU, A)) / (2 * h)
        assert np.allclose(G[:, :, k], fd, rtol=0, atol=1e-9 * np.abs(E).max())


def test_equilibrium():
    rng = np.random.default_rng(2)
    E = _rand_strain(rng)
    x = _exterior_points(rng, 50)
    h = 1e-5
    div = np.zeros((50, 3))
    for k in range(3):
        dx = np.zeros(3)
        dx[k] = h
        ds = (cavity.stress(x + dx, E, MU, NU, A) - cavity.stress(x - dx, E, MU, NU, A)) / (2 * h)
        div += ds[:, :, k]
    scale = np.abs(cavity.stress(x, E, MU, NU, A)).max() / A
    assert np.abs(div).max() < 1e-6 * scale


def test_cavity_surface_is_traction_free():
    rng = np.random.default_rng(3)
    for _ in range(3):
        E = _rand_strain(rng)
        n = _exterior_points(rng, 200, 1.0, 1.0) / A
        t = np.einsum("pij,pj->pi", cavity.stress(A * n, E, MU, NU, A), n)
        assert np.abs(t).max() < 1e-12 * np.abs(cavity.stress(A * n, E, MU, NU, A)).max()


def test_remote_field_is_the_applied_one():
    rng = np.random.default_rng(4)
    E = _rand_strain(rng)
    lam = 2 * MU * NU / (1 - 2 * NU)
    s_inf = lam * np.trace(E) * np.eye(3) + 2 * MU * E
    x = _exterior_points(rng, 20, 1e4, 2e4)
    assert np.allclose(cavity.stress(x, E, MU, NU, A), s_inf, rtol=0, atol=1e-10 * np.abs(s_inf).max())


@pytest.mark.parametrize("nu", [0.0, 0.25, 0.2934, 0.45])
def test_uniaxial_tension_concentrations_are_the_classical_ones(nu):
    S, mu = 1.0, 80.0
    Y = 2 * mu * (1 + nu)
    E = S / Y * np.diag([-nu, -nu, 1.0])  # remote uniaxial stress S along x3
    s_eq = cavity.stress(np.array([A, 0.0, 0.0]), E, mu, nu, A)
    s_pole = cavity.stress(np.array([0.0, 0.0, A]), E, mu, nu, A)
    assert s_eq[2, 2] == pytest.approx(S * (27 - 15 * nu) / (2 * (7 - 5 * nu)), rel=1e-12)
    assert s_pole[0, 0] == pytest.approx(-S * (3 + 15 * nu) / (2 * (7 - 5 * nu)), rel=1e-12)
    assert s_pole[1, 1] == pytest.approx(s_pole[0, 0], rel=1e-12)


def test_hydrostatic_tension_doubles_half_again_at_the_surface():
    E = 1e-3 * np.eye(3)
    lam = 2 * MU * NU / (1 - 2 * NU)
    p = (3 * lam + 2 * MU) * 1e-3
    s = cavity.stress(np.array([0.0, A, 0.0]), E, MU, NU, A)
    assert s[0, 0] == pytest.approx(1.5 * p, rel=1e-12) and s[2, 2] == pytest.approx(1.5 * p, rel=1e-12)
    assert abs(s[1, 1]) < 1e-12 * p
