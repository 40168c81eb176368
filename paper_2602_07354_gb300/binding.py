"""Thin Python binding of the libelas C ABI (``include/elas.h``).

Every function here marshals arguments and calls the entry point of the same name; all
computation runs in the library's CUDA kernels.  PyTorch supplies device memory (the context
workspace and the vectors) and the CUDA stream.  There is no fallback: if ``libelas.so`` is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libelas.so")

ELAS_OK = 0
ELAS_ERR = {-1: "INVALID_ARG", -2: "WORKSPACE", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT", -6: "ADMISSION",
            -7: "STATE"}
CONVERGED, MAX_ITER, BREAKDOWN, NONFINITE, CANCELLED = 0, 1, 2, 3, 4
PREC_FP64, PREC_MIXED = 0, 1
STOP_PRECOND, STOP_TRUE = 0, 1
PRECOND_BLOCK, PRECOND_SCALAR, PRECOND_NONE = 0, 1, 2
HOTSPOT_ALL, HOTSPOT_SOLID = 0, 1
FP64_OP_PAIRED, FP64_OP_NATIVE = 0, 1
TEXTURE_FIBER, TEXTURE_RANDOM = 0, 1


class ElasError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ELAS_ERR.get(code, code)}: {msg}")
        self.code = code


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("relres_precond", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("n_replacements", ctypes.c_int), ("launches", ctypes.c_int),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveOpts(ctypes.Structure):
    _fields_ = [("stop_rule", ctypes.c_int), ("replace_every", ctypes.c_int), ("check_every", ctypes.c_int),
                ("replace_drop", ctypes.c_int), ("precond", ctypes.c_int)]


_lib = None


def lib():
    """Load libelas.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2602_07354_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        L.elas_isotropic_stiffness.argtypes = [d, d, vp]
        L.elas_cubic_stiffness.argtypes = [d, d, d, vp]
        L.elas_rotated_stiffness.argtypes = [vp, vp, vp]
        L.elas_workspace_bytes.argtypes = [i, i, i, i, i, ctypes.POINTER(sz)]
        L.elas_create.argtypes = [ctypes.POINTER(vp), i, i, i, vp, i, vp, vp, i, vp, sz, vp]
        L.elas_destroy.argtypes = [vp]
        L.elas_destroy.restype = None
        L.elas_last_error.argtypes = [vp]
        L.elas_last_error.restype = ctypes.c_char_p
        L.elas_apply.argtypes = [vp, vp, vp]
        L.elas_apply_f32.argtypes = [vp, vp, vp]
        L.elas_rhs.argtypes = [vp, vp, vp]
        L.elas_residual.argtypes = [vp, vp, vp, vp, vp]
        L.elas_jacobi.argtypes = [vp, vp]
        L.elas_set_fp64_operator.argtypes = [vp, i]
        L.elas_batch_set_fp64_operator.argtypes = [vp, i]
        L.elas_pcg_solve.argtypes = [vp, vp, d, i, vp, vp, vp]
        L.elas_stress.argtypes = [vp, vp, vp, vp, vp, vp]
        L.elas_autotune.argtypes = [vp, i, ctypes.POINTER(d)]
        L.elas_hotspot.argtypes = [vp, vp, d, i, vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]
        L.elas_tuning_export.argtypes = [ctypes.c_char_p, sz, ctypes.POINTER(sz)]
        L.elas_tuning_import.argtypes = [ctypes.c_char_p]
        L.elas_batch_workspace_bytes.argtypes = [i, vp, i, i, ctypes.POINTER(sz)]
        L.elas_batch_create.argtypes = [ctypes.POINTER(vp), i, vp, i, i, vp, sz, vp]
        L.elas_batch_autotune.argtypes = [vp, i]
        L.elas_batch_solve.argtypes = [vp, vp, d, i, vp, vp]
        L.elas_batch_fluctuation.argtypes = [vp, i, i, vp]
        L.elas_batch_stress.argtypes = [vp, i, i, vp, vp, vp, vp]
        L.elas_batch_destroy.argtypes = [vp]
        L.elas_batch_destroy.restype = None
        L.elas_batch_last_error.argtypes = [vp]
        L.elas_batch_last_error.restype = ctypes.c_char_p
        L.elas_server_workspace_bytes.argtypes = [sz, i, ctypes.POINTER(sz)]
        L.elas_server_create.argtypes = [ctypes.POINTER(vp), sz, i, i, i, vp, sz, vp]
        L.elas_server_submit.argtypes = [vp, vp, vp, d, i, ctypes.POINTER(ctypes.c_longlong)]
        L.elas_server_step.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        L.elas_server_poll.argtypes = [vp, ctypes.c_longlong, vp, vp, ctypes.POINTER(d), ctypes.POINTER(i)]
        L.elas_server_stats.argtypes = [vp, ctypes.POINTER(sz), ctypes.POINTER(i), ctypes.POINTER(i),
                                        ctypes.POINTER(ctypes.c_longlong)]
        L.elas_server_set_replacement.argtypes = [vp, i, i]
        L.elas_server_cancel.argtypes = [vp, ctypes.c_longlong]
        L.elas_server_destroy.argtypes = [vp]
        L.elas_server_destroy.restype = None
        L.elas_server_last_error.argtypes = [vp]
        L.elas_server_last_error.restype = ctypes.c_char_p
        L.elas_generate_workspace_bytes.argtypes = [i, i, i, i, i, ctypes.POINTER(sz)]
        L.elas_assign_grains.argtypes = [i, i, i, vp, vp, i, vp, vp, sz, vp]
        L.elas_stamp_pores.argtypes = [i, i, i, vp, i, vp, ctypes.POINTER(ctypes.c_longlong), vp, sz, vp]
        L.elas_grain_count.argtypes = [d, d, d, d, d, ctypes.POINTER(ctypes.c_longlong)]
        L.elas_seed_grains.argtypes = [i, vp, vp, d, d, d, d, vp, vp, vp, vp, vp]
        L.elas_orientations.argtypes = [i, i, vp, vp, vp, vp, vp]
        L.elas_generate_last_error.argtypes = []
        L.elas_generate_last_error.restype = ctypes.c_char_p
        for name in ("elas_isotropic_stiffness", "elas_cubic_stiffness", "elas_rotated_stiffness",
                     "elas_workspace_bytes", "elas_create", "elas_apply", "elas_apply_f32", "elas_rhs",
                     "elas_residual", "elas_jacobi", "elas_pcg_solve", "elas_stress", "elas_autotune", "elas_hotspot",
                     "elas_set_fp64_operator", "elas_batch_set_fp64_operator",
                     "elas_tuning_export", "elas_tuning_import",
                     "elas_batch_workspace_bytes", "elas_batch_create", "elas_batch_autotune", "elas_batch_solve",
                     "elas_batch_fluctuation", "elas_batch_stress", "elas_server_workspace_bytes",
                     "elas_server_create", "elas_server_submit", "elas_server_step", "elas_server_poll",
                     "elas_server_stats", "elas_server_set_replacement", "elas_server_cancel", "elas_generate_workspace_bytes",
                     "elas_assign_grains", "elas_stamp_pores", "elas_grain_count", "elas_seed_grains",
                     "elas_orientations"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(code: int, ctx=None):
    if code != ELAS_OK:
        msg = lib().elas_last_error(ctx)
        raise ElasError(code, msg.decode() if msg else "")


def _f64_host(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# --- constitutive helpers (host) -----------------------------------------------------------------
def elas_isotropic_stiffness(E: float, nu: float) -> np.ndarray:
    C = np.zeros(36)
    _check(lib().elas_isotropic_stiffness(E, nu, C.ctypes.data))
    return C.reshape(6, 6)


def elas_cubic_stiffness(c11: float, c12: float, c44: float) -> np.ndarray:
    C = np.zeros(36)
    _check(lib().elas_cubic_stiffness(c11, c12, c44, C.ctypes.data))
    return C.reshape(6, 6)


def elas_rotated_stiffness(C6_local, rho) -> np.ndarray:
    Cl = _f64_host(C6_local, 36)
    r = _f64_host(rho, 3)
    out = np.zeros(36)
    _check(lib().elas_rotated_stiffness(Cl.ctypes.data, r.ctypes.data, out.ctypes.data))
    return out.reshape(6, 6)


def materials_to_C(materials) -> np.ndarray:
    """Material rows (kind, p1, p2, p3) -> crystal-frame stiffness via the library's helpers."""
    mats = np.asarray(materials, dtype=np.float64).reshape(-1, 4)
    return np.stack([elas_isotropic_stiffness(a, b) if k == 0 else elas_cubic_stiffness(a, b, c)
                     for k, a, b, c in mats]) if len(mats) else np.zeros((0, 6, 6))


def elas_workspace_bytes(nx: int, ny: int, nz: int, n_phases: int, precision: int) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().elas_workspace_bytes(nx, ny, nz, n_phases, precision, ctypes.byref(n)))
    return n.value


# --- context -------------------------------------------------------------------------------------
@dataclass
class Context:
    """An elas_ctx plus the torch-owned workspace it lives in."""

    handle: ctypes.c_void_p
    workspace: object
    nx: int
    ny: int
    nz: int
    precision: int
    stream: object

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def close(self):
        if self.handle:
            lib().elas_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def elas_create(nx, ny, nz, phase_id, C_local, rodrigues=None, precision=PREC_FP64, device="cuda",
                stream=None) -> Context:
    import torch

    phase = np.ascontiguousarray(phase_id, dtype=np.int32).ravel()
    C = np.ascontiguousarray(C_local, dtype=np.float64).reshape(-1, 36)
    n_phases = C.shape[0]
    rho = None if rodrigues is None else _f64_host(rodrigues, 3 * n_phases)
    nbytes = elas_workspace_bytes(nx, ny, nz, n_phases, precision)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    if stream is None:
        stream = torch.cuda.current_stream(ws.device)
    h = ctypes.c_void_p(0)
    _check(lib().elas_create(ctypes.byref(h), nx, ny, nz, phase.ctypes.data, n_phases, C.ctypes.data,
                             None if rho is None else rho.ctypes.data, precision, ctypes.c_void_p(aligned), nbytes,
                             ctypes.c_void_p(stream.cuda_stream)))
    return Context(h, ws, nx, ny, nz, precision, stream)


def create_from_micro(ms, precision=PREC_FP64, device="cuda", stream=None) -> Context:
    """Context for a synthetic microstructure (phase ids, material rows, Rodrigues vectors)."""
    return elas_create(ms.nx, ms.ny, ms.nz, ms.phase, materials_to_C(ms.materials), ms.rho, precision, device, stream)


def elas_set_fp64_operator(ctx: Context, form: int):
    _check(lib().elas_set_fp64_operator(ctx.handle, form), ctx.handle)


def elas_apply(ctx: Context, u, y):
    _check(lib().elas_apply(ctx.handle, _ptr(u), _ptr(y)), ctx.handle)


def elas_apply_f32(ctx: Context, u, y):
    _check(lib().elas_apply_f32(ctx.handle, _ptr(u), _ptr(y)), ctx.handle)


def elas_rhs(ctx: Context, strain, b):
    e = _f64_host(strain, 6)
    _check(lib().elas_rhs(ctx.handle, e.ctypes.data, _ptr(b)), ctx.handle)


def elas_residual(ctx: Context, strain, w, g, want_norm=True):
    e = _f64_host(strain, 6)
    rn = ctypes.c_double(0.0)
    _check(lib().elas_residual(ctx.handle, e.ctypes.data, _ptr(w), _ptr(g), ctypes.byref(rn) if want_norm else None),
           ctx.handle)
    return rn.value if want_norm else None


def elas_jacobi(ctx: Context, Minv):
    _check(lib().elas_jacobi(ctx.handle, _ptr(Minv)), ctx.handle)


def elas_pcg_solve(ctx: Context, strain, tol: float, max_iter: int, w_out=None, stop_rule=None, replace_every=0,
                   check_every=0, replace_drop=0, precond=0) -> dict:
    e = _f64_host(strain, 6)
    opts = SolveOpts(-1 if stop_rule is None else stop_rule, replace_every, check_every, replace_drop, precond)
    info = SolveInfo()
    code = lib().elas_pcg_solve(ctx.handle, e.ctypes.data, tol, max_iter, ctypes.byref(opts), _ptr(w_out),
                                ctypes.byref(info))
    if code not in (ELAS_OK, -4):
        _check(code, ctx.handle)
    out = info.as_dict()
    out["code"] = code
    return out


def elas_stress(ctx: Context, strain, w=None, stress=None, von_mises=None, want_macro=True):
    e = _f64_host(strain, 6)
    macro = np.zeros(6)
    _check(lib().elas_stress(ctx.handle, e.ctypes.data, _ptr(w), _ptr(stress), _ptr(von_mises),
                             macro.ctypes.data if want_macro else None), ctx.handle)
    return macro if want_macro else None


def elas_autotune(ctx: Context, max_candidates: int = 12) -> float:
    best = ctypes.c_double(0.0)
    _check(lib().elas_autotune(ctx.handle, max_candidates, ctypes.byref(best)), ctx.handle)
    return best.value


# --- batches ---------------------------------------------------------------------------------------
class ElasRve(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("phase_id", ctypes.c_void_p),
                ("n_phases", ctypes.c_int), ("C_local", ctypes.c_void_p), ("rodrigues", ctypes.c_void_p)]


def _bcheck(code: int, b=None):
    if code != ELAS_OK:
        msg = lib().elas_batch_last_error(b)
        raise ElasError(code, msg.decode() if msg else "")


@dataclass
class Batch:
    """An elas_batch plus its torch-owned workspace."""

    handle: ctypes.c_void_p
    workspace: object
    dims: list
    n_rhs: int
    precision: int
    stream: object

    @property
    def n_rve(self) -> int:
        return len(self.dims)

    def close(self):
        if self.handle:
            lib().elas_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rve_array(micros):
    keep, arr = [], (ElasRve * len(micros))()
    for k, ms in enumerate(micros):
        ph = np.ascontiguousarray(ms.phase, dtype=np.int32).ravel()
        C = np.ascontiguousarray(materials_to_C(ms.materials), dtype=np.float64).reshape(-1)
        rho = None if ms.rho is None else np.ascontiguousarray(ms.rho, dtype=np.float64).reshape(-1)
        keep += [ph, C, rho]
        arr[k] = ElasRve(ms.nx, ms.ny, ms.nz, ph.ctypes.data, ms.n_phases, C.ctypes.data,
                         None if rho is None else rho.ctypes.data)
    return arr, keep


def elas_batch_workspace_bytes(micros, n_rhs: int, precision: int) -> int:
    arr, _keep = _rve_array(micros)
    n = ctypes.c_size_t(0)
    _bcheck(lib().elas_batch_workspace_bytes(len(micros), ctypes.byref(arr), n_rhs, precision, ctypes.byref(n)))
    return n.value


def elas_batch_create(micros, n_rhs: int, precision=PREC_MIXED, device="cuda", stream=None) -> Batch:
    import torch

    arr, _keep = _rve_array(micros)
    n = ctypes.c_size_t(0)
    _bcheck(lib().elas_batch_workspace_bytes(len(micros), ctypes.byref(arr), n_rhs, precision, ctypes.byref(n)))
    ws = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
    aligned = (ws.data_ptr() + 255) // 256 * 256
    if stream is None:
        stream = torch.cuda.current_stream(ws.device)
    h = ctypes.c_void_p(0)
    _bcheck(lib().elas_batch_create(ctypes.byref(h), len(micros), ctypes.byref(arr), n_rhs, precision,
                                    ctypes.c_void_p(aligned), n.value, ctypes.c_void_p(stream.cuda_stream)))
    return Batch(h, ws, [(m.nx, m.ny, m.nz) for m in micros], n_rhs, precision, stream)


def elas_batch_set_fp64_operator(b: Batch, form: int):
    _bcheck(lib().elas_batch_set_fp64_operator(b.handle, form), b.handle)


def elas_batch_autotune(b: Batch, max_candidates: int = 12):
    _bcheck(lib().elas_batch_autotune(b.handle, max_candidates), b.handle)


def elas_batch_solve(b: Batch, strains, tol: float, max_iter: int, stop_rule=None, replace_every=0, check_every=0,
                     replace_drop=0):
    e = np.ascontiguousarray(strains, dtype=np.float64).reshape(-1)
    if e.size != 6 * b.n_rve * b.n_rhs:
        raise ValueError("strains must hold n_rve * n_rhs * 6 values")
    opts = SolveOpts(-1 if stop_rule is None else stop_rule, replace_every, check_every, replace_drop, 0)
    infos = (SolveInfo * (b.n_rve * b.n_rhs))()
    code = lib().elas_batch_solve(b.handle, e.ctypes.data, tol, max_iter, ctypes.byref(opts), ctypes.byref(infos))
    if code not in (ELAS_OK, -4):
        _bcheck(code, b.handle)
    return [x.as_dict() for x in infos]


def elas_batch_fluctuation(b: Batch, rve: int, rhs: int, w_out):
    _bcheck(lib().elas_batch_fluctuation(b.handle, rve, rhs, _ptr(w_out)), b.handle)


def elas_batch_stress(b: Batch, rve: int, rhs: int, strain, stress=None, von_mises=None, want_macro=True):
    e = _f64_host(strain, 6)
    macro = np.zeros(6)
    _bcheck(lib().elas_batch_stress(b.handle, rve, rhs, e.ctypes.data, _ptr(stress), _ptr(von_mises),
                                    macro.ctypes.data if want_macro else None), b.handle)
    return macro if want_macro else None


# --- solve server ------------------------------------------------------------------------------------
def _scheck(code: int, srv=None):
    if code != ELAS_OK:
        msg = lib().elas_server_last_error(srv)
        raise ElasError(code, msg.decode() if msg else "")


@dataclass
class Server:
    """An elas_server plus its torch-owned workspace (request budget + tables)."""

    handle: ctypes.c_void_p
    workspace: object
    stream: object
    sizes: dict

    def close(self):
        if self.handle:
            lib().elas_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def elas_server_create(budget_bytes: int, max_active: int, precision=PREC_MIXED, iters_per_step=0, device="cuda",
                       stream=None) -> Server:
    import torch

    n = ctypes.c_size_t(0)
    _scheck(lib().elas_server_workspace_bytes(budget_bytes, max_active, ctypes.byref(n)))
    ws = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
    aligned = (ws.data_ptr() + 255) // 256 * 256
    if stream is None:
        stream = torch.cuda.current_stream(ws.device)
    h = ctypes.c_void_p(0)
    _scheck(lib().elas_server_create(ctypes.byref(h), budget_bytes, max_active, precision, iters_per_step,
                                     ctypes.c_void_p(aligned), n.value, ctypes.c_void_p(stream.cuda_stream)))
    return Server(h, ws, stream, {})


def elas_server_submit(srv: Server, ms, strain, tol: float, max_iter: int) -> int:
    arr, _keep = _rve_array([ms])
    e = _f64_host(strain, 6)
    rid = ctypes.c_longlong(0)
    _scheck(lib().elas_server_submit(srv.handle, ctypes.byref(arr), e.ctypes.data, tol, max_iter, ctypes.byref(rid)),
            srv.handle)
    srv.sizes[rid.value] = ms.N
    return rid.value


def elas_server_step(srv: Server):
    a, q, f = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _scheck(lib().elas_server_step(srv.handle, ctypes.byref(a), ctypes.byref(q), ctypes.byref(f)), srv.handle)
    return a.value, q.value, f.value


def elas_server_poll(srv: Server, rid: int, w_out=None):
    info = SolveInfo()
    lat = ctypes.c_double(0.0)
    done = ctypes.c_int(0)
    _scheck(lib().elas_server_poll(srv.handle, rid, ctypes.byref(info), _ptr(w_out), ctypes.byref(lat),
                                   ctypes.byref(done)), srv.handle)
    if not done.value:
        return None
    out = info.as_dict()
    out["latency_s"] = lat.value
    return out


def elas_server_cancel(srv: Server, rid: int) -> None:
    _scheck(lib().elas_server_cancel(srv.handle, rid), srv.handle)


def elas_server_set_replacement(srv: Server, replace_every=0, replace_drop=0):
    _scheck(lib().elas_server_set_replacement(srv.handle, replace_every, replace_drop), srv.handle)


def elas_server_stats(srv: Server):
    b, a, q, d = ctypes.c_size_t(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_longlong(0)
    _scheck(lib().elas_server_stats(srv.handle, ctypes.byref(b), ctypes.byref(a), ctypes.byref(q), ctypes.byref(d)),
            srv.handle)
    return dict(bytes_in_use=b.value, active=a.value, queued=q.value, done=d.value)


# ---- microstructure generator (Sec. 2.2) ------------------------------------------------------
def _gcheck(code: int):
    if code != ELAS_OK:
        raise ElasError(code, lib().elas_generate_last_error().decode())


def _gen_workspace(dims, n_grains, n_pores, device):
    import torch

    n = ctypes.c_size_t(0)
    _gcheck(lib().elas_generate_workspace_bytes(*dims, n_grains, n_pores, ctypes.byref(n)))
    ws = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
    return ws, (ws.data_ptr() + 255) // 256 * 256, n.value


def elas_assign_grains(dims, seeds, semi_axes=None, phase=None, device="cuda", stream=None):
    """Algorithm 4 on the device: int32 grain ids (torch tensor, x fastest) of the nearest seed
    under the weighted ellipsoidal distance, periodic cell."""
    import torch

    nx, ny, nz = dims
    seeds = np.ascontiguousarray(seeds, dtype=np.float64)
    semi = None if semi_axes is None else np.ascontiguousarray(semi_axes, dtype=np.float64)
    if phase is None:
        phase = torch.empty(nx * ny * nz, dtype=torch.int32, device=device)
    ws, base, nb = _gen_workspace(dims, len(seeds), 0, phase.device)
    if stream is None:
        stream = torch.cuda.current_stream(phase.device)
    _gcheck(lib().elas_assign_grains(nx, ny, nz, seeds.ctypes.data_as(ctypes.c_void_p),
                                     None if semi is None else semi.ctypes.data_as(ctypes.c_void_p), len(seeds),
                                     ctypes.c_void_p(phase.data_ptr()), ctypes.c_void_p(base), nb,
                                     ctypes.c_void_p(stream.cuda_stream)))
    del ws
    return phase


def elas_grain_count(lengths, mean_d: float, mean_alpha: float) -> int:
    """Algorithm 3: grains of mean diameter and aspect ratio that fill the box."""
    n = ctypes.c_longlong(0)
    lx, ly, lz = (float(v) for v in lengths)
    _gcheck(lib().elas_grain_count(lx, ly, lz, float(mean_d), float(mean_alpha), ctypes.byref(n)))
    return n.value


def elas_seed_grains(lo, hi, mean_d, sd_d, mean_alpha, sd_alpha, z, u, seeds=None, semi_axes=None, stream=None):
    """Algorithm 3 on the device: seeds (n x 3) and semi-axes (rt, rl) (n x 2) from normal draws z
    (n x 2) and uniform draws u (n x 3), all float64 torch tensors on the device."""
    import torch

    n = int(z.shape[0])
    if seeds is None:
        seeds = torch.empty((n, 3), dtype=torch.float64, device=z.device)
    if semi_axes is None:
        semi_axes = torch.empty((n, 2), dtype=torch.float64, device=z.device)
    lo = _f64_host(lo, 3)
    hi = _f64_host(hi, 3)
    if stream is None:
        stream = torch.cuda.current_stream(z.device)
    _gcheck(lib().elas_seed_grains(n, lo.ctypes.data, hi.ctypes.data, float(mean_d), float(sd_d), float(mean_alpha),
                                   float(sd_alpha), _ptr(z), _ptr(u), _ptr(seeds), _ptr(semi_axes),
                                   ctypes.c_void_p(stream.cuda_stream)))
    return seeds, semi_axes


def elas_orientations(texture: int, draws, rho=None, crystal_axis=None, sample_axis=None, stream=None):
    """Algorithm 6 on the device: Rodrigues vectors (n x 3) from draws (n x 3, float64 on the
    device): (phi, alpha, theta) for TEXTURE_FIBER, (u1, u2, u3) for TEXTURE_RANDOM."""
    import torch

    n = int(draws.shape[0])
    if rho is None:
        rho = torch.empty((n, 3), dtype=torch.float64, device=draws.device)
    ca = None if crystal_axis is None else _f64_host(crystal_axis, 3)
    sa = None if sample_axis is None else _f64_host(sample_axis, 3)
    if stream is None:
        stream = torch.cuda.current_stream(draws.device)
    _gcheck(lib().elas_orientations(n, texture, None if ca is None else ca.ctypes.data,
                                    None if sa is None else sa.ctypes.data, _ptr(draws), _ptr(rho),
                                    ctypes.c_void_p(stream.cuda_stream)))
    return rho


def elas_stamp_pores(dims, pores, phase, stream=None) -> int:
    """Algorithm 5 (rotated ellipsoids, 15 numbers per pore) on the device, in place; returns the
    number of voxels with a negative id afterwards."""
    import torch

    nx, ny, nz = dims
    pores = np.ascontiguousarray(pores, dtype=np.float64).reshape(-1, 15)
    ws, base, nb = _gen_workspace(dims, 0, len(pores), phase.device)
    if stream is None:
        stream = torch.cuda.current_stream(phase.device)
    cnt = ctypes.c_longlong(0)
    _gcheck(lib().elas_stamp_pores(nx, ny, nz, pores.ctypes.data_as(ctypes.c_void_p), len(pores),
                                   ctypes.c_void_p(phase.data_ptr()), ctypes.byref(cnt), ctypes.c_void_p(base), nb,
                                   ctypes.c_void_p(stream.cuda_stream)))
    del ws
    return cnt.value


def elas_hotspot(ctx: Context, von_mises, s_kernel: float = 0.4, smoothed=None, neighbours=HOTSPOT_ALL):
    """App. C: (sigma_max, voxel id, smoothed field) of the masked Gaussian-smoothed von Mises field;
    neighbours: HOTSPOT_ALL (pores compete in the 26-neighbour test) or HOTSPOT_SOLID."""
    import torch

    if smoothed is None:
        smoothed = torch.empty_like(von_mises)
    sm = ctypes.c_double(0.0)
    at = ctypes.c_longlong(-1)
    _check(lib().elas_hotspot(ctx.handle, ctypes.c_void_p(von_mises.data_ptr()), s_kernel, neighbours,
                              ctypes.c_void_p(smoothed.data_ptr()), ctypes.byref(sm), ctypes.byref(at)), ctx.handle)
    return sm.value, at.value, smoothed


def elas_tuning_export() -> str:
    """The autotuner's per-size tilings of this process as text (one line per grid size)."""
    n = ctypes.c_size_t(0)
    _check(lib().elas_tuning_export(None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(lib().elas_tuning_export(buf, n.value + 1, ctypes.byref(n)))
    return buf.value.decode()


def elas_tuning_import(text: str) -> None:
    _check(lib().elas_tuning_import(text.encode()))


def save_tuning(path: str) -> None:
    with open(path, "w") as f:
        f.write(elas_tuning_export())


def load_tuning(path: str) -> None:
    with open(path) as f:
        elas_tuning_import(f.read())
