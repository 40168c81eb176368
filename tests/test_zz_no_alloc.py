"""elas_stress_noalloc against elas_stress.

The no-allocation entry point exists for callers that may not allocate memory when they need
the stress (code running during another component's graph capture, fixed-memory real-time
loops, plug-ins in frameworks that own all device memory).  It must return the same stress,
von Mises and macro stress as the context-based elas_stress, call after call, even though every
call reuses the same scratch array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_07354_gb300 import binding as B
from paper_2602_07354_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
vp = ctypes.c_void_p


def _noalloc():
    from paper_2602_07354_gb300 import build

    build.build()
    L = B.lib()
    f = L.elas_stress_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp]
    f.restype = ctypes.c_int
    return f


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _call(f, ms, phase_dev, e6, w, s, vm, macro, stream, C=None, rho=None, n_phases=None):
    C = np.ascontiguousarray(B.materials_to_C(ms.materials)).reshape(-1) if C is None else C
    rho = np.ascontiguousarray(ms.rho).reshape(-1) if rho is None and ms.rho is not None else rho
    return f(ms.nx, ms.ny, ms.nz, vp(phase_dev.data_ptr()), ms.n_phases if n_phases is None else n_phases,
             C.ctypes.data, None if rho is None else rho.ctypes.data, e6.ctypes.data, vp(w.data_ptr()),
             None if s is None else vp(s.data_ptr()), None if vm is None else vp(vm.data_ptr()),
             None if macro is None else macro.ctypes.data, vp(stream.cuda_stream))


def test_noalloc_stress_matches_elas_stress_and_oracle(oracle):
    # two calls in a row on different microstructures and phase counts (70 phases: more than one
    # host-side chunk of 32 phases of the stiffness table), each against elas_stress and the oracle
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = _noalloc()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(5)
    for call, ms in enumerate((synth.polycrystal(14, 70, pore_frac=0.03, seed=18, dims=(14, 12, 16)),
                               synth.polycrystal(10, 9, pore_frac=0.05, seed=19, dims=(10, 13, 9)))):
        N = ms.N
        ctx = B.create_from_micro(ms)
        phase_dev = torch.from_numpy(ms.phase.astype(np.int32)).cuda()
        e6 = rng.normal(size=6) * 1e-3
        w_h = rng.normal(size=3 * N) * 1e-4
        w = torch.from_numpy(w_h).cuda()
        s_ref = torch.empty(6 * N, dtype=torch.float64, device="cuda")
        vm_ref = torch.empty(N, dtype=torch.float64, device="cuda")
        macro_ref = B.elas_stress(ctx, e6, w, s_ref, vm_ref)
        s = torch.full((6 * N,), np.nan, dtype=torch.float64, device="cuda")
        vm = torch.full((N,), np.nan, dtype=torch.float64, device="cuda")
        macro = np.full(6, np.nan)
        assert _call(f, ms, phase_dev, e6, w, s, vm, macro, stream) == B.ELAS_OK, call
        torch.cuda.synchronize()
        sg, vg = s.cpu().numpy(), vm.cpu().numpy()
        assert _rel(sg, s_ref.cpu().numpy()) <= 1e-12
        assert _rel(vg, vm_ref.cpu().numpy()) <= 1e-12
        assert _rel(macro, macro_ref) <= 1e-12
        so, vo, mo = oracle.Problem.from_micro(ms).stress(e6, w_h)
        assert _rel(sg, so.ravel()) <= 1e-12 and _rel(vg, vo) <= 1e-12 and _rel(macro, mo) <= 1e-12
        ctx.close()


def test_noalloc_stress_matches_elas_stress_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = _noalloc()
    ms = synth.polycrystal(22, 30, pore_frac=0.04, seed=17, dims=(22, 19, 24))
    N = ms.N
    C = np.ascontiguousarray(B.materials_to_C(ms.materials)).reshape(-1)
    rho = np.ascontiguousarray(ms.rho).reshape(-1)
    ctx = B.create_from_micro(ms)
    phase_dev = torch.from_numpy(ms.phase.astype(np.int32)).cuda()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(4)
    for call in range(2):
        e6 = rng.normal(size=6) * 1e-3
        w = torch.from_numpy(rng.normal(size=3 * N) * 1e-4).cuda()
        s_ref = torch.empty(6 * N, dtype=torch.float64, device="cuda")
        vm_ref = torch.empty(N, dtype=torch.float64, device="cuda")
        macro_ref = B.elas_stress(ctx, e6, w, s_ref, vm_ref)
        s = torch.full((6 * N,), np.nan, dtype=torch.float64, device="cuda")
        vm = torch.full((N,), np.nan, dtype=torch.float64, device="cuda")
        macro = np.full(6, np.nan)
        rc = f(ms.nx, ms.ny, ms.nz, vp(phase_dev.data_ptr()), ms.n_phases, C.ctypes.data, rho.ctypes.data,
               e6.ctypes.data, vp(w.data_ptr()), vp(s.data_ptr()), vp(vm.data_ptr()), macro.ctypes.data,
               vp(stream.cuda_stream))
        assert rc == B.ELAS_OK, (call, rc)
        torch.cuda.synchronize()
        assert _rel(s.cpu().numpy(), s_ref.cpu().numpy()) <= 1e-12
        assert _rel(vm.cpu().numpy(), vm_ref.cpu().numpy()) <= 1e-12
        assert _rel(macro, macro_ref) <= 1e-12


def test_noalloc_rejects_bad_sizes_and_ids():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = _noalloc()
    N = 4 * 4 * 4
    phase = torch.zeros(N, dtype=torch.int32, device="cuda")
    w = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    C = np.tile(np.eye(6).ravel() * 100.0, 4097)
    e6 = np.zeros(6)
    stream = torch.cuda.current_stream()
    args = lambda n_ph, ph: (4, 4, 4, vp(ph.data_ptr()), n_ph, C.ctypes.data, None, e6.ctypes.data,
                             vp(w.data_ptr()), None, None, None, vp(stream.cuda_stream))
    assert f(*args(4097, phase)) == -1  # more phases than the scratch table holds
    bad = phase.clone()
    bad[5] = 7
    assert f(*args(3, bad)) == -1  # id outside [-1, n_phases), caught on the device
    assert f(*args(8, bad)) == B.ELAS_OK



def test_noalloc_rejects_bad_inputs_and_capturing_streams():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = _noalloc()
    ms = synth.polycrystal(6, 3, pore_frac=0.0, seed=20)
    N = ms.N
    phase_dev = torch.from_numpy(ms.phase.astype(np.int32)).cuda()
    w = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    e6 = np.array([1e-3, 0, 0, 0, 0, 0.0])
    C = np.ascontiguousarray(B.materials_to_C(ms.materials)).reshape(-1).copy()
    asym = C.copy()
    asym[1] += 10.0  # C_12 != C_21
    assert _call(f, ms, phase_dev, e6, w, None, None, None, stream, C=asym) == -1
    nan_e6 = e6.copy()
    nan_e6[2] = np.nan
    assert _call(f, ms, phase_dev, nan_e6, w, None, None, None, stream) == -1
    # no phases, every voxel a pore: zero stress everywhere, zero macro stress
    void = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    s = torch.full((6 * N,), np.nan, dtype=torch.float64, device="cuda")
    macro = np.full(6, np.nan)
    assert _call(f, ms, void, e6, w, s, None, macro, stream, C=np.zeros(0), rho=np.zeros(0), n_phases=0) == B.ELAS_OK
    torch.cuda.synchronize()
    assert np.all(s.cpu().numpy() == 0.0) and np.all(macro == 0.0)
    # a stream under capture is refused before any work is enqueued (the capture stays usable)
    side = torch.cuda.Stream()
    x = torch.zeros(4, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        x.add_(1.0)
        rc = _call(f, ms, phase_dev, e6, w, None, None, None, side)
    assert rc == -1
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
