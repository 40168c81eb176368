"""Analytic displacement and stress around a traction-free spherical cavity of radius a in an
infinite isotropic matrix (shear modulus mu, Poisson ratio nu) under a uniform remote strain E —
the closed-form field the paper compares its Eshelby-void solutions with (Sec. 3.1, App. A).

With e = tr(E)/3, D = E - e I and q = x.D.x, the field is
    u = E x + a^3 [ (A1/r^3 + A2 a^2/r^5) D x + (B1/r^5 + B2 a^2/r^7) q x + C1 e x / r^3 ]
    A1 = 5(1-2nu)/(7-5nu),  A2 = 3/(7-5nu),  B1 = -B2 = 15/(2(7-5nu)),  C1 = (1+nu)/(2(1-2nu)).
The five coefficients are the unique ones for which this isotropic ansatz (the decaying harmonic
and biharmonic terms linear in E) satisfies Navier's equation and leaves r = a traction-free;
the pins in test_cavity_pins.py check equilibrium, the free surface, the remote limit and the
classical concentration factors of a cavity under uniaxial stress, so none of this is taken on
trust.  Test infrastructure only."""
import numpy as np


def coefficients(nu):
    d = 7.0 - 5.0 * nu
    return 5.0 * (1.0 - 2.0 * nu) / d, 3.0 / d, 7.5 / d, -7.5 / d, (1.0 + nu) / (2.0 * (1.0 - 2.0 * nu))


def _parts(E):
    E = np.asarray(E, dtype=np.float64)
    e = np.trace(E) / 3.0
    return E, e, E - e * np.eye(3)


def displacement(x, E, nu, a):
    """u at points x (..., 3) outside the cavity (|x| >= a), cavity centred at the origin."""
    A1, A2, B1, B2, C1 = coefficients(nu)
    E, e, D = _parts(E)
    x = np.asarray(x, dtype=np.float64)
    r = np.linalg.norm(x, axis=-1)[..., None]
    Dx = x @ D.T
    q = np.sum(x * Dx, axis=-1)[..., None]
    a3 = a ** 3
    return x @ E.T + a3 * ((A1 / r ** 3 + A2 * a * a / r ** 5) * Dx + (B1 / r ** 5 + B2 * a * a / r ** 7) * q * x
                           + C1 * e * x / r ** 3)


def gradient(x, E, nu, a):
    """du_i/dx_k at points x (..., 3), shape (..., 3, 3), from the derivative of each term."""
    A1, A2, B1, B2, C1 = coefficients(nu)
    E, e, D = _parts(E)
    x = np.asarray(x, dtype=np.float64)
    r = np.linalg.norm(x, axis=-1)[..., None, None]
    xi = x[..., :, None]
    xk = x[..., None, :]
    Dx = (x @ D.T)[..., :, None]
    q = np.sum(x * (x @ D.T), axis=-1)[..., None, None]
    a2 = a * a
    f = A1 / r ** 3 + A2 * a2 / r ** 5
    df = -3.0 * A1 / r ** 4 - 5.0 * A2 * a2 / r ** 6
    g = B1 / r ** 5 + B2 * a2 / r ** 7
    dg = -5.0 * B1 / r ** 6 - 7.0 * B2 * a2 / r ** 8
    I = np.eye(3)
    pert = (df * Dx * xk / r + f * D + dg * q * xi * xk / r + 2.0 * g * xi * Dx.swapaxes(-1, -2) + g * q * I
            + C1 * e * (I / r ** 3 - 3.0 * xi * xk / r ** 5))
    return E + a ** 3 * pert


def stress(x, E, mu, nu, a):
    """sigma (..., 3, 3) at points x outside the cavity."""
    G = gradient(x, E, nu, a)
    eps = 0.5 * (G + G.swapaxes(-1, -2))
    lam = 2.0 * mu * nu / (1.0 - 2.0 * nu)
    tr = np.trace(eps, axis1=-2, axis2=-1)[..., None, None]
    return lam * tr * np.eye(3) + 2.0 * mu * eps


def von_mises(s):
    d = s - np.trace(s, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3.0
    return np.sqrt(1.5 * np.sum(d * d, axis=(-2, -1)))


def surface_peak_von_mises(E, mu, nu, n_theta=2001, n_phi=73):
    """Largest von Mises stress on the cavity surface (a = 1), sampled over the sphere."""
    th = np.linspace(0.0, np.pi, n_theta)[:, None]
    ph = np.linspace(0.0, 2.0 * np.pi, n_phi)[None, :]
    n = np.stack(np.broadcast_arrays(np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)), -1)
    return float(von_mises(stress(n, E, mu, nu, 1.0)).max())
