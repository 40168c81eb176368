"""ctypes wrapper around the FP64 CPU oracle (``elas_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The library product never imports this module.

The oracle follows ELAS3D-Xtal (arXiv 2602.07354) Sec. 2.1: Eqs. 1-9, Algorithm 1
(stiffness rotation) and Algorithm 2 (point-block Jacobi PCG).  See ``elas_oracle.c`` for the
conventions (component-major vectors, Voigt order 11,22,33,23,13,12, corner numbering).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "elas_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")

CONVERGED, MAX_ITER, BREAKDOWN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 (plain C, no vectorisation pragmas, no FMA contraction, so
    that every host rounds each operation as written)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i, d, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        L.or_iso_stiffness.argtypes = [d, d, _dp]
        L.or_cubic_stiffness.argtypes = [d, d, d, _dp]
        L.or_rodrigues_to_R.argtypes = [_dp, _dp]
        L.or_rotate_stiffness.argtypes = [_dp, _dp, _dp]
        L.or_element_stiffness.argtypes = [_dp, i, _dp]
        L.or_phase_tables.argtypes = [i, _dp, ctypes.c_void_p, _dp, _dp]
        L.or_apply.argtypes = [i, i, i, _ip, _dp, _dp, _dp]
        L.or_apply_nodes.argtypes = [i, i, i, _ip, _dp, _dp, i64, _lp, _dp]
        L.or_rhs.argtypes = [i, i, i, _ip, _dp, _dp, _dp]
        L.or_energy.argtypes = [i, i, i, _ip, _dp, _dp, _dp]
        L.or_energy.restype = d
        L.or_dense.argtypes = [i, i, i, _ip, _dp, _dp]
        L.or_jacobi.argtypes = [i, i, i, _ip, _dp, _dp]
        L.or_rhs_scale.argtypes = [i, i, i, _ip, _dp, _dp]
        L.or_rhs_scale.restype = d
        L.or_pcg.argtypes = [i, i, i, _ip, _dp, _dp, d, d, i, i, i, _dp,
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        L.or_pcg.restype = i
        L.or_stress.argtypes = [i, i, i, _ip, _dp, _dp, _dp, _dp, ctypes.c_void_p, _dp]
        L.or_strain.argtypes = [i, i, i, _ip, _dp, _dp, _dp]
        L.or_assign_grains.argtypes = [i, i, i, _dp, ctypes.c_void_p, i, _ip]
        L.or_assign_voxels.argtypes = [i, i, i, _dp, ctypes.c_void_p, i, _lp, i64, _ip]
        L.or_stamp_pores.argtypes = [i, i, i, _dp, i, _ip]
        L.or_stamp_pores.restype = i64
        L.or_grain_count.argtypes = [d, d, d, d, d]
        L.or_grain_count.restype = i64
        L.or_seed_grains.argtypes = [i, _dp, _dp, d, d, d, d, _dp, _dp, _dp, _dp]
        L.or_fiber_orientations.argtypes = [i, _dp, _dp, _dp, _dp]
        L.or_random_orientations.argtypes = [i, _dp, _dp]
        L.or_gauss_weights.argtypes = [d, i, _dp]
        L.or_hotspot.argtypes = [i, i, i, _ip, _dp, _dp, i, i, _dp, ctypes.POINTER(ctypes.c_int64)]
        L.or_hotspot.restype = d
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --- constitutive (Sec. 2.1.1) ---------------------------------------------------------
def iso_stiffness(E: float, nu: float) -> np.ndarray:
    C = np.zeros(36)
    lib().or_iso_stiffness(E, nu, C)
    return C.reshape(6, 6)


def cubic_stiffness(c11: float, c12: float, c44: float) -> np.ndarray:
    C = np.zeros(36)
    lib().or_cubic_stiffness(c11, c12, c44, C)
    return C.reshape(6, 6)


def rodrigues_to_R(rho) -> np.ndarray:
    R = np.zeros(9)
    lib().or_rodrigues_to_R(_f64(rho), R)
    return R.reshape(3, 3)


def rotate_stiffness(C6, R) -> np.ndarray:
    out = np.zeros(36)
    lib().or_rotate_stiffness(_f64(C6).ravel(), _f64(R).ravel(), out)
    return out.reshape(6, 6)


def element_stiffness(C6, rule: int = 0) -> np.ndarray:
    K = np.zeros(576)
    lib().or_element_stiffness(_f64(C6).ravel(), rule, K)
    return K.reshape(24, 24)


def materials_to_C(materials) -> np.ndarray:
    """Material rows (kind, p1, p2, p3) -> crystal-frame 6x6 stiffness, with the oracle's own
    Eqs. 2-3 (kind 0: E, nu) and cubic fill of Algorithm 1 (kind 1: C11, C12, C44)."""
    mats = np.asarray(materials, dtype=np.float64).reshape(-1, 4)
    out = np.zeros((mats.shape[0], 6, 6))
    for p, (kind, a, b, c) in enumerate(mats):
        out[p] = iso_stiffness(a, b) if kind == 0 else cubic_stiffness(a, b, c)
    return out


# --- problem object ----------------------------------------------------------------------
@dataclass
class Problem:
    """A periodic voxel problem: grid dims, per-voxel phase ids (-1 = pore), per-phase
    crystal-frame stiffness (n_phases x 6 x 6) and Rodrigues vectors (n_phases x 3 or None)."""

    nx: int
    ny: int
    nz: int
    phase: np.ndarray
    C_local: np.ndarray
    rho: np.ndarray | None = None

    def __post_init__(self):
        self.phase = np.ascontiguousarray(self.phase, dtype=np.int32).ravel()
        self.C_local = _f64(self.C_local).reshape(-1, 6, 6)
        if self.rho is not None:
            self.rho = _f64(self.rho).reshape(-1, 3)
        assert self.phase.size == self.N
        P = self.C_local.shape[0]
        C6g = np.zeros(P * 36)
        Ke = np.zeros(P * 576)
        rho_ptr = None if self.rho is None else self.rho.ctypes.data_as(ctypes.c_void_p)
        lib().or_phase_tables(P, self.C_local.ravel().copy(), rho_ptr, C6g, Ke)
        self.C_global = C6g.reshape(P, 6, 6)
        self.Ke = Ke

    @classmethod
    def from_micro(cls, ms) -> "Problem":
        """From a synthetic microstructure (phase ids, material rows, Rodrigues vectors)."""
        return cls(ms.nx, ms.ny, ms.nz, ms.phase, materials_to_C(ms.materials), ms.rho)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dims(self):
        return (self.nx, self.ny, self.nz)

    # operator and right-hand side (Eqs. 7-8)
    def apply(self, u) -> np.ndarray:
        y = np.zeros(3 * self.N)
        lib().or_apply(*self.dims, self.phase, self.Ke, _f64(u).ravel(), y)
        return y

    def apply_nodes(self, u, nodes) -> np.ndarray:
        sel = np.ascontiguousarray(nodes, dtype=np.int64)
        y = np.zeros(3 * sel.size)
        lib().or_apply_nodes(*self.dims, self.phase, self.Ke, _f64(u).ravel(), sel.size, sel, y)
        return y.reshape(-1, 3)

    def rhs(self, strain6) -> np.ndarray:
        b = np.zeros(3 * self.N)
        lib().or_rhs(*self.dims, self.phase, self.Ke, _f64(strain6), b)
        return b

    def rhs_scale(self, strain6) -> float:
        return lib().or_rhs_scale(*self.dims, self.phase, self.Ke, _f64(strain6))

    def energy(self, strain6, w) -> float:
        return lib().or_energy(*self.dims, self.phase, self.Ke, _f64(strain6), _f64(w).ravel())

    def dense(self) -> np.ndarray:
        D = 3 * self.N
        A = np.zeros(D * D)
        lib().or_dense(*self.dims, self.phase, self.Ke, A)
        return A.reshape(D, D)

    def jacobi(self) -> np.ndarray:
        M = np.zeros(9 * self.N)
        lib().or_jacobi(*self.dims, self.phase, self.Ke, M)
        return M.reshape(self.N, 3, 3)

    # Algorithm 2
    def pcg(self, strain6, tol: float, max_iter: int, precond=True, paper_guard: bool = False,
            history: bool = False):
        """Algorithm 2.  precond: True / "block" point-block Jacobi (the paper's), False / "none"
        plain CG, "scalar" point Jacobi M = diag(A)."""
        precond = {True: 1, False: 0, "block": 1, "none": 0, "scalar": 2}[precond]
        b = self.rhs(strain6)
        w = np.zeros(3 * self.N)
        it = ctypes.c_int(0)
        ratio = ctypes.c_double(0.0)
        hist = np.zeros(max_iter + 1) if history else None
        hp = None if hist is None else hist.ctypes.data_as(ctypes.c_void_p)
        out = lib().or_pcg(*self.dims, self.phase, self.Ke, b, self.rhs_scale(strain6), tol, max_iter, int(precond),
                           int(paper_guard),
                           w, ctypes.byref(it), ctypes.byref(ratio), hp)
        res = dict(w=w, b=b, iters=it.value, outcome=out, ratio=ratio.value)
        if history:
            res["history"] = hist[: it.value + 1]
        return res

    def stress(self, strain6, w):
        s = np.zeros(6 * self.N)
        vm = np.zeros(self.N)
        macro = np.zeros(6)
        lib().or_stress(*self.dims, self.phase, self.C_global.ravel().copy(), _f64(strain6), _f64(w).ravel(), s,
                        vm.ctypes.data_as(ctypes.c_void_p), macro)
        return s.reshape(6, self.N), vm, macro

    def strain(self, strain6, w) -> np.ndarray:
        e = np.zeros(6 * self.N)
        lib().or_strain(*self.dims, self.phase, _f64(strain6), _f64(w).ravel(), e)
        return e.reshape(6, self.N)

    def true_relres(self, strain6, w) -> float:
        b = self.rhs(strain6)
        r = b + self.apply(w)
        nb = np.linalg.norm(b)
        return float(np.linalg.norm(r) / nb) if nb > 0 else float(np.linalg.norm(r))


def assign_grains(dims, seeds, semi=None) -> np.ndarray:
    """Algorithm 4 by brute force: nearest grain under the weighted ellipsoidal distance with the
    periodic minimum image (ties to the lowest index); int32, x fastest."""
    nx, ny, nz = dims
    phase = np.zeros(nx * ny * nz, np.int32)
    sem = None if semi is None else _f64(semi).ravel()
    lib().or_assign_grains(nx, ny, nz, _f64(seeds).ravel(), None if sem is None else sem.ctypes.data_as(ctypes.c_void_p),
                           len(seeds), phase)
    return phase


def assign_voxels(dims, seeds, voxels, semi=None) -> np.ndarray:
    """Algorithm 4 by brute force for the listed voxel ids only."""
    nx, ny, nz = dims
    vox = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.zeros(len(vox), np.int32)
    sem = None if semi is None else _f64(semi).ravel()
    lib().or_assign_voxels(nx, ny, nz, _f64(seeds).ravel(), None if sem is None else sem.ctypes.data_as(ctypes.c_void_p),
                           len(seeds), vox, len(vox), out)
    return out


def stamp_pores(dims, pores, phase) -> int:
    """Algorithm 5 with rotated ellipsoids (15 numbers per pore), in place; returns the pore voxels."""
    nx, ny, nz = dims
    return int(lib().or_stamp_pores(nx, ny, nz, _f64(pores).ravel(), len(pores), phase))


def grain_count(lengths, mu_d: float, mu_alpha: float) -> int:
    """Algorithm 3: N_g = ceil(V / (pi (mu_d/2)^2 mu_alpha mu_d))."""
    lx, ly, lz = (float(v) for v in lengths)
    return int(lib().or_grain_count(lx, ly, lz, float(mu_d), float(mu_alpha)))


def seed_grains(lo, hi, mu_d, sd_d, mu_a, sd_a, z, u):
    """Algorithm 3: lognormal diameters and aspect ratios from normal draws z (n x 2), semi-axes
    (rt, rl) and uniform seeds from u (n x 3).  Returns seeds (n x 3), semi (n x 2)."""
    z = _f64(z).reshape(-1, 2)
    u = _f64(u).reshape(-1, 3)
    n = z.shape[0]
    seeds, semi = np.zeros((n, 3)), np.zeros((n, 2))
    lib().or_seed_grains(n, _f64(lo), _f64(hi), mu_d, sd_d, mu_a, sd_a, z, u, seeds, semi)
    return seeds, semi


def fiber_orientations(draws, crystal=(1.0, 0.0, 1.0), sample=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Algorithm 6, textured branch: draws (n x 3) = spin phi, wobble axis angle alpha, wobble
    angle theta (radians).  Returns Rodrigues vectors (n x 3)."""
    d = _f64(draws).reshape(-1, 3)
    rho = np.zeros_like(d)
    lib().or_fiber_orientations(d.shape[0], _f64(crystal), _f64(sample), d, rho)
    return rho


def random_orientations(u) -> np.ndarray:
    """Algorithm 6, random branch: Shoemake quaternions from u (n x 3) -> Rodrigues vectors."""
    u = _f64(u).reshape(-1, 3)
    rho = np.zeros_like(u)
    lib().or_random_orientations(u.shape[0], u, rho)
    return rho


def gauss_weights(s: float, r: int) -> np.ndarray:
    w = np.zeros(2 * r + 1)
    lib().or_gauss_weights(s, r, w)
    return w


def hotspot(dims, phase, vm, s: float = 0.4, r: int = 1, solid_only: bool = False):
    """App. C: masked Gaussian smoothing (normalised convolution, periodic) of the von Mises field
    and the largest 26-neighbourhood local maximum in the solid (with solid_only, pore voxels do
    not take part in the neighbour comparison).  Returns (max, voxel, smoothed)."""
    nx, ny, nz = dims
    sm = np.zeros(nx * ny * nz)
    at = ctypes.c_int64(-1)
    best = lib().or_hotspot(nx, ny, nz, np.ascontiguousarray(phase, np.int32), _f64(vm).ravel(), gauss_weights(s, r), r,
                            int(solid_only), sm, ctypes.byref(at))
    return best, at.value, sm


def solid_node_mask(p: Problem) -> np.ndarray:
    """Nodes touching at least one voxel with a nonzero stiffness (where w is determined)."""
    solid_vox = np.zeros(p.N, bool)
    ok = p.phase >= 0
    nz_phase = np.abs(p.C_global).reshape(p.C_global.shape[0], -1).max(axis=1) > 0
    solid_vox[ok] = nz_phase[p.phase[ok]]
    sv = solid_vox.reshape(p.nz, p.ny, p.nx)
    m = np.zeros_like(sv)
    for az in (0, 1):
        for ay in (0, 1):
            for ax in (0, 1):
                # node (i,j,k) is corner a of voxel (i-ax, j-ay, k-az)
                m |= np.roll(sv, shift=(az, ay, ax), axis=(0, 1, 2))
    return m.ravel()
