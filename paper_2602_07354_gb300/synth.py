"""Seeded synthetic microstructures: the inputs of the solve, shaped like the paper's workloads.

This module holds input generation only (grain tessellation, pore insertion, orientation
sampling, material constants).  It contains none of the solver's arithmetic and is shared by
the CUDA path's tests and benchmark and by the oracle's tests.

Readings (ELAS3D-Xtal, arXiv 2602.07354):
  * Voxel centres sit at (i+1/2, j+1/2, k+1/2); a voxel is inside a sphere of centre c and
    radius r when |x - c|^2 <= r^2 (Algorithm 5), measured with the periodic minimum image.
  * Grains: plain periodic Voronoi cells of seeds uniform in the box (the equiaxed,
    aspect-ratio-1 limit of the ellipsoidal assignment of Algorithm 4).
  * Random texture: Shoemake's uniform quaternions converted to Rodrigues vectors
    (Algorithm 6, random branch), including its |q_w| < 1e-8 guard.
  * Pores get phase id -1 (zero stiffness) instead of N_g + 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

try:  # periodic nearest-seed queries; fall back to chunked brute force without scipy
    from scipy.spatial import cKDTree
except Exception:  # pragma: no cover
    cKDTree = None


@dataclass
class Microstructure:
    nx: int
    ny: int
    nz: int
    phase: np.ndarray            # int32, N, x fastest; -1 = pore
    materials: np.ndarray        # n_phases x 4: (ISO, E, nu, 0) or (CUBIC, C11, C12, C44), GPa
    rho: np.ndarray | None       # n_phases x 3 Rodrigues vectors (None = identity)
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_phases(self) -> int:
        return int(self.materials.shape[0])


# Material rows carry constants only; each consumer builds its own 6x6 stiffness from them.
ISO, CUBIC = 0.0, 1.0


def iso_mat(E: float, nu: float) -> np.ndarray:
    return np.array([ISO, E, nu, 0.0])


def cubic_mat(c11: float, c12: float, c44: float) -> np.ndarray:
    return np.array([CUBIC, c11, c12, c44])


def shoemake_rodrigues(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform SO(3) orientations as Rodrigues vectors (Algorithm 6, random branch)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    qw = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2)
    qx = np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
    qy = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    qz = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    q = np.stack([qx, qy, qz], axis=1)
    small = np.abs(qw) < 1e-8
    rho = np.where(small[:, None], q * 1e9, q / np.where(small, 1.0, qw)[:, None])
    return rho


def fibre_draws(rng: np.random.Generator, n: int, spread_deg: float) -> np.ndarray:
    """The random draws of the fibre texture (Algorithm 6, textured branch), n x 3: a uniform spin
    phi about the build direction, a uniform wobble-axis angle alpha and a Gaussian wobble angle
    theta of standard deviation spread_deg, all in radians (the orientations themselves come from
    the library's elas_orientations)."""
    return np.stack([rng.uniform(0.0, 2.0 * np.pi, n), rng.uniform(0.0, 2.0 * np.pi, n),
                     rng.normal(0.0, np.deg2rad(spread_deg), n)], axis=1)


def _centres(nx, ny, nz, k0=0, k1=None):
    k1 = nz if k1 is None else k1
    k, j, i = np.meshgrid(np.arange(k0, k1), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([i.ravel() + 0.5, j.ravel() + 0.5, k.ravel() + 0.5], axis=1)


def periodic_voronoi(nx, ny, nz, seeds: np.ndarray) -> np.ndarray:
    """Nearest seed (periodic minimum image) for every voxel centre; int32 ids, x fastest."""
    box = np.array([nx, ny, nz], float)
    out = np.empty(nx * ny * nz, np.int32)
    per_layer = nx * ny
    chunk = max(1, (1 << 22) // per_layer)
    tree = cKDTree(np.mod(seeds, box), boxsize=box) if cKDTree is not None else None
    for k0 in range(0, nz, chunk):
        k1 = min(nz, k0 + chunk)
        X = _centres(nx, ny, nz, k0, k1)
        if tree is not None:
            try:
                _, idx = tree.query(X, k=1, workers=-1)
            except TypeError:  # older scipy
                _, idx = tree.query(X, k=1)
        else:
            best = np.full(X.shape[0], np.inf)
            idx = np.zeros(X.shape[0], np.int64)
            for s, c in enumerate(seeds):
                d = X - c
                d -= box * np.round(d / box)
                d2 = (d * d).sum(1)
                upd = d2 < best
                best[upd] = d2[upd]
                idx[upd] = s
        out[k0 * per_layer:k1 * per_layer] = idx
    return out


def _stamp(phase3, centre, semi, Rm=None, value=-1):
    """Overwrite voxels whose centre lies in the (possibly rotated) ellipsoid, periodic."""
    nz, ny, nx = phase3.shape
    rmax = float(np.max(semi))
    lo = np.floor(centre - rmax - 1).astype(int)
    hi = np.ceil(centre + rmax + 1).astype(int)
    ii = np.arange(lo[0], hi[0] + 1)
    jj = np.arange(lo[1], hi[1] + 1)
    kk = np.arange(lo[2], hi[2] + 1)
    K, J, I = np.meshgrid(kk, jj, ii, indexing="ij")
    d = np.stack([I + 0.5 - centre[0], J + 0.5 - centre[1], K + 0.5 - centre[2]], -1)
    if Rm is not None:
        d = d @ Rm  # coordinates in the ellipsoid frame
    inside = ((d / np.asarray(semi, float)) ** 2).sum(-1) <= 1.0
    kk_, jj_, ii_ = np.mod(K[inside], nz), np.mod(J[inside], ny), np.mod(I[inside], nx)
    # count each newly carved voxel once (periodic images of a large pore may repeat an index)
    flat = np.unique((kk_ * ny + jj_) * nx + ii_)
    view = phase3.reshape(-1)
    fresh = int((view[flat] != value).sum())
    view[flat] = value
    return fresh


def add_spherical_pores(phase, nx, ny, nz, rng, frac, rmin, rmax):
    """Spheres with radius ~ U[rmin, rmax] and uniform centres until the pore fraction >= frac."""
    ph = phase.reshape(nz, ny, nx)
    n_pores = 0
    carved, target = int((ph < 0).sum()), frac * ph.size
    while frac > 0 and carved < target:
        c = rng.random(3) * np.array([nx, ny, nz])
        r = rng.uniform(rmin, rmax)
        carved += _stamp(ph, c, (r, r, r))
        n_pores += 1
    return n_pores


def _rand_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def add_mixed_pores(phase, nx, ny, nz, rng, frac):
    """Half spheres r ~ U[2,8], half randomly oriented ellipsoids with a ~ U[2,3],
    b/a ~ U[1,2], c/a ~ U[3,6] (gas / lack-of-fusion / keyhole-like shapes)."""
    ph = phase.reshape(nz, ny, nx)
    n = 0
    carved, target = int((ph < 0).sum()), frac * ph.size
    while carved < target:
        c = rng.random(3) * np.array([nx, ny, nz])
        if n % 2 == 0:
            r = rng.uniform(2, 8)
            carved += _stamp(ph, c, (r, r, r))
        else:
            a = rng.uniform(2, 3)
            carved += _stamp(ph, c, (a, a * rng.uniform(1, 2), a * rng.uniform(3, 6)), _rand_rotation(rng))
        n += 1
    return n


def mixed_pore_draws(rng, n, k):
    """k pore records (15 numbers each: centre, semi-axes, row-major axes) of the large-solve
    recipe on an n^3 cell: alternately a sphere r ~ U[2,8] and a randomly oriented ellipsoid with
    a ~ U[2,3], b/a ~ U[1,2], c/a ~ U[3,6]."""
    out = np.zeros((k, 15))
    for i in range(k):
        c = rng.random(3) * n
        if i % 2 == 0:
            r = rng.uniform(2, 8)
            out[i] = np.concatenate([c, [r, r, r], np.eye(3).ravel()])
        else:
            a = rng.uniform(2, 3)
            out[i] = np.concatenate([c, [a, a * rng.uniform(1, 2), a * rng.uniform(3, 6)], _rand_rotation(rng).ravel()])
    return out


# --- the workloads ---------------------------------------------------------------------------
def eshelby_inclusion(n: int = 20, radius: float = 5.0, E0=200.0, nu0=0.3, E1=400.0, nu1=0.25) -> Microstructure:
    """Isotropic matrix with a centred spherical isotropic inclusion (20^3, r = 5 by default)."""
    phase = np.zeros(n ** 3, np.int32)
    X = _centres(n, n, n)
    c = np.array([n / 2, n / 2, n / 2])
    phase[((X - c) ** 2).sum(1) <= radius ** 2] = 1
    mats = np.stack([iso_mat(E0, nu0), iso_mat(E1, nu1)])
    return Microstructure(n, n, n, phase, mats, None, dict(kind="eshelby", radius=radius))


def eshelby_void(n: int = 100, radius_frac: float = 2.0 / 50.0, E=194.0, nu=0.2934) -> Microstructure:
    """Sec. 3.1's benchmark geometry: spherical void of radius 2/50 of the box in an isotropic matrix."""
    phase = np.zeros(n ** 3, np.int32)
    X = _centres(n, n, n)
    c = np.array([n / 2, n / 2, n / 2])
    phase[((X - c) ** 2).sum(1) <= (radius_frac * n) ** 2] = -1
    return Microstructure(n, n, n, phase, iso_mat(E, nu)[None], None, dict(kind="eshelby_void"))


def polycrystal(n, n_grains, pore_frac=0.01, seed=1, c=(204.6, 137.7, 126.2), pore_r=(2.0, 6.0),
                pore_mix=False, dims=None) -> Microstructure:
    """Periodic Voronoi polycrystal with cubic grains, random texture and zero-stiffness pores."""
    nx, ny, nz = dims if dims is not None else (n, n, n)
    rng = np.random.Generator(np.random.PCG64(seed))
    seeds = rng.random((n_grains, 3)) * np.array([nx, ny, nz])
    phase = periodic_voronoi(nx, ny, nz, seeds)
    if pore_mix:
        n_pores = add_mixed_pores(phase, nx, ny, nz, rng, pore_frac)
    else:
        n_pores = add_spherical_pores(phase, nx, ny, nz, rng, pore_frac, *pore_r)
    rho = shoemake_rodrigues(rng, n_grains)
    mats = np.broadcast_to(cubic_mat(*c), (n_grains, 4)).copy()
    return Microstructure(nx, ny, nz, phase, mats, rho,
                          dict(kind="polycrystal", n_grains=n_grains, seed=seed, n_pores=n_pores,
                               pore_frac=float(np.count_nonzero(phase < 0)) / phase.size))


def random_problem(dims, n_phases, rng, pore_prob=0.1, anisotropic=True) -> Microstructure:
    """Small random problem for parity tests: random phases, random cubic/iso constants."""
    nx, ny, nz = dims
    N = nx * ny * nz
    phase = rng.integers(0, n_phases, N).astype(np.int32)
    phase[rng.random(N) < pore_prob] = -1
    mats = []
    for p in range(n_phases):
        if anisotropic and p % 2 == 0:
            c12 = rng.uniform(80, 140)
            mats.append(cubic_mat(c12 + rng.uniform(40, 120), c12, rng.uniform(40, 130)))
        else:
            mats.append(iso_mat(rng.uniform(50, 400), rng.uniform(0.1, 0.4)))
    rho = rng.normal(size=(n_phases, 3)) if anisotropic else None
    return Microstructure(nx, ny, nz, phase, np.stack(mats), rho, dict(kind="random"))


def random_symmetric_strain(rng, norm=1e-3) -> np.ndarray:
    """Random symmetric strain tensor (E11,E22,E33,E23,E13,E12) of Frobenius norm `norm`."""
    e = rng.normal(size=6)
    E = np.array([[e[0], e[5], e[4]], [e[5], e[1], e[3]], [e[4], e[3], e[2]]])
    e = e * norm / np.linalg.norm(E)
    return e


UNIT_LOAD_CASES = 1e-3 * np.eye(6)  # e11, e22, e33, e23, e13, e12 (tensor components)

SS316L = (206.0, 133.0, 119.0)  # cubic C11, C12, C44 (GPa) of the LPBF SS316L study (Sec. 3.3)

# The anisotropy sensitivity study of Sec. 3.2 (its material table): Zener ratio A and cubic
# C11, C12, C44 (GPa) at fixed Voigt K = 156.64 and baseline G = 75.08 GPa.
ANISOTROPY_CASES = [(0.50, 300.04, 84.95, 53.77), (0.75, 274.65, 97.64, 66.38), (1.00, 256.75, 106.59, 75.08),
                    (1.50, 232.07, 118.93, 84.85), (2.00, 216.52, 126.70, 89.82), (3.00, 198.66, 135.64, 94.53),
                    (4.00, 188.74, 140.60, 96.28), (5.00, 182.38, 143.78, 96.50)]


def void_polycrystal_seeds(n: int, n_grains: int = 81488, seed: int = 11):
    """Seeds, semi-axes and orientations of Sec. 3.2's anisotropy cell scaled to n^3 voxels: the
    grain count of the 200 um cube (81,488 equiaxed grains, size spread 10%, aspect ratio 1 +- 0.1)
    with uniform seeds, and one central spherical void of radius n/40 (5 um of 200 um) as a pore
    record for the pore overwrite."""
    rng = np.random.Generator(np.random.PCG64(seed))
    seeds = rng.random((n_grains, 3)) * n
    rt = rng.lognormal(0.0, 0.1, n_grains)
    rl = rt * np.clip(rng.normal(1.0, 0.1, n_grains), 0.5, 1.5)
    rho = shoemake_rodrigues(rng, n_grains)
    r = n / 40.0
    void = np.concatenate([[n / 2.0, n / 2.0, n / 2.0], [r, r, r], np.eye(3).ravel()])
    return seeds, np.stack([rt, rl], 1), rho, void[None]


def batch_rves(n_rve=64, seed0=1000, edges=(32, 48, 64, 80, 96), voxels_per_grain=2000, pores=(0.0, 0.03)):
    """Uneven RVEs: edge uniform in `edges`, one grain per `voxels_per_grain` voxels, random
    texture, spherical pores with a volume fraction uniform in `pores`."""
    out = []
    for i in range(n_rve):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        n = int(rng.choice(edges))
        frac = float(rng.uniform(*pores))
        out.append(polycrystal(n, max(1, n ** 3 // voxels_per_grain), pore_frac=frac, seed=seed0 + i))
    return out


def request_stream(n_requests=2000, rate=20.0, seed=7, edges=(48, 64, 96, 128, 160), tols=(1e-6, 1e-8),
                   pores=(0.0, 0.03), voxels_per_grain=2000):
    """A Poisson stream of solve requests, each with its own seeded polycrystal recipe: arrival time
    (s), grid edge, grain count (one grain per `voxels_per_grain` voxels), pore fraction, strain
    (random symmetric, Frobenius norm 1e-3), tolerance and the seed of its microstructure draws
    (request j: 10000 + j)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_requests))
    reqs = []
    for j in range(n_requests):
        r = np.random.Generator(np.random.PCG64(10000 + j))
        n = int(r.choice(edges))
        reqs.append(dict(arrival=float(arrivals[j]), edge=n, n_grains=max(1, n ** 3 // voxels_per_grain),
                         pore_frac=float(r.uniform(*pores)), strain=random_symmetric_strain(r), tol=float(r.choice(tols)),
                         seed=10000 + j))
    return reqs


def polycrystal_draws(n, n_grains, pore_frac, seed, pore_r=(2.0, 6.0)):
    """The random draws of one seeded polycrystal recipe on an n^3 periodic cell, for generation on
    the device: seeds uniform in the box (n_grains x 3), the Shoemake draws of the random texture
    (n_grains x 3, Algorithm 6) and a generator of pore batches (15 numbers per spherical pore:
    centre, semi-axes r, r, r, identity axes; r ~ U[pore_r]); the caller stamps batches until the
    pore fraction is reached."""
    rng = np.random.Generator(np.random.PCG64(seed))
    seeds = rng.random((n_grains, 3)) * n
    u = rng.random((n_grains, 3))
    mean_vol = np.pi * (pore_r[1] ** 4 - pore_r[0] ** 4) / (3.0 * (pore_r[1] - pore_r[0]))  # E[4/3 pi r^3]

    def pore_batch(missing_voxels):
        # about 70% of the missing pore volume per batch, so that the last batch overshoots little
        k = max(1, int(0.7 * missing_voxels / mean_vol))
        c = rng.random((k, 3)) * n
        r = rng.uniform(pore_r[0], pore_r[1], k)
        return np.concatenate([c, np.repeat(r[:, None], 3, 1), np.tile(np.eye(3).ravel(), (k, 1))], axis=1)

    return seeds, u, pore_batch
