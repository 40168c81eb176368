"""Batched solves (many RVEs x load cases in shared persistent launches) and the autotuner.

A problem's iterates depend only on its own grid, tiling and load, so a batch problem must give
exactly the single-context result, and an RVE the same result alone and in any mix.
"""
import numpy as np
import pytest

from paper_2602_07354_gb300 import binding as B
from paper_2602_07354_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LOADS = 1e-3 * np.array([[0, 0, 1, 0, 0, 0], [1, 0, 0, 0, 0, 0], [0, 0, 0, 1, 0, 0]], float)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_07354_gb300 import build

    build.build()


def micros():
    return [synth.polycrystal(16, 8, pore_frac=0.02, seed=3),
            synth.polycrystal(20, 10, pore_frac=0.02, seed=4, dims=(20, 18, 22)),
            synth.polycrystal(24, 12, pore_frac=0.03, seed=5)]


@pytest.mark.parametrize("prec", [B.PREC_FP64, B.PREC_MIXED])
def test_batch_equals_single_context_bitwise(prec):
    ms = micros()
    n_rhs = len(LOADS)
    strains = np.stack([LOADS for _ in ms])  # (n_rve, n_rhs, 6)
    b = B.elas_batch_create(ms, n_rhs, prec)
    infos = B.elas_batch_solve(b, strains, 1e-8, 5000, stop_rule=B.STOP_TRUE, check_every=25)
    assert all(i["status"] == B.CONVERGED for i in infos)
    for i, m in enumerate(ms):
        ctx = B.create_from_micro(m, precision=prec)
        for r in range(n_rhs):
            w_single = torch.empty(3 * m.N, dtype=torch.float64, device="cuda")
            info = B.elas_pcg_solve(ctx, LOADS[r], 1e-8, 5000, w_out=w_single, stop_rule=B.STOP_TRUE,
                                    check_every=25)
            w_batch = torch.empty_like(w_single)
            B.elas_batch_fluctuation(b, i, r, w_batch)
            assert info["iters"] == infos[i * n_rhs + r]["iters"]
            assert np.array_equal(host(w_single), host(w_batch)), (i, r)


def test_alone_and_in_the_mix_bitwise():
    ms = micros()
    alone = B.elas_batch_create([ms[1]], 1, B.PREC_MIXED)
    B.elas_batch_solve(alone, LOADS[:1][None], 1e-8, 5000)
    mix = B.elas_batch_create(ms, 1, B.PREC_MIXED)
    B.elas_batch_solve(mix, np.stack([LOADS[:1] for _ in ms]), 1e-8, 5000)
    wa = torch.empty(3 * ms[1].N, dtype=torch.float64, device="cuda")
    wm = torch.empty_like(wa)
    B.elas_batch_fluctuation(alone, 0, 0, wa)
    B.elas_batch_fluctuation(mix, 1, 0, wm)
    assert np.array_equal(host(wa), host(wm))


def test_batch_against_oracle_and_effective_stiffness(oracle):
    # six unit load cases of one RVE (the columns of the effective stiffness) plus a second RVE
    ms = [synth.polycrystal(18, 9, pore_frac=0.02, seed=8), synth.polycrystal(14, 5, pore_frac=0.0, seed=9)]
    loads = synth.UNIT_LOAD_CASES
    b = B.elas_batch_create(ms, 6, B.PREC_MIXED)
    infos = B.elas_batch_solve(b, np.stack([loads for _ in ms]), 1e-8, 5000)
    assert all(i["status"] == B.CONVERGED and i["relres_true"] <= 1e-8 for i in infos)
    for i, m in enumerate(ms):
        p = oracle.Problem.from_micro(m)
        Ceff = np.zeros((6, 6))
        for r in range(6):
            macro = B.elas_batch_stress(b, i, r, loads[r])
            Ceff[:, r] = macro / 1e-3 * np.array([1, 1, 1, 1, 1, 1]) / np.array([1, 1, 1, 2, 2, 2])[r]
            if r in (2, 4):
                ref = p.pcg(loads[r], 1e-12, 5000)
                s_ref, _, macro_ref = p.stress(loads[r], ref["w"])
                s = torch.empty(6 * m.N, dtype=torch.float64, device="cuda")
                B.elas_batch_stress(b, i, r, loads[r], s, None, want_macro=False)
                assert rel(host(s), s_ref) <= 1e-5
                assert rel(macro, macro_ref) <= 1e-7
        # the effective stiffness of a periodic cell is symmetric (Hill-Mandel)
        assert np.abs(Ceff - Ceff.T).max() <= 1e-5 * np.abs(Ceff).max()


def test_autotune_keeps_parity(oracle):
    m = synth.polycrystal(30, 15, pore_frac=0.02, seed=11, dims=(30, 26, 34))
    p = oracle.Problem.from_micro(m)
    for prec, dt, tol in ((B.PREC_FP64, torch.float64, 1e-12), (B.PREC_MIXED, torch.float32, 2e-6)):
        ctx = B.create_from_micro(m, precision=prec)
        best = B.elas_autotune(ctx, 6)
        assert best > 0
        u = np.random.default_rng(1).normal(size=3 * m.N)
        ut = torch.from_numpy(u).to(device="cuda", dtype=dt)
        y = torch.empty_like(ut)
        (B.elas_apply if prec == B.PREC_FP64 else B.elas_apply_f32)(ctx, ut, y)
        assert rel(host(y), p.apply(ut.double().cpu().numpy())) <= tol
    b = B.elas_batch_create([m], 1, B.PREC_MIXED)
    B.elas_batch_autotune(b, 4)
    infos = B.elas_batch_solve(b, LOADS[:1][None], 1e-8, 5000)
    assert infos[0]["status"] == B.CONVERGED
    w = torch.empty(3 * m.N, dtype=torch.float64, device="cuda")
    B.elas_batch_fluctuation(b, 0, 0, w)
    assert p.true_relres(LOADS[0], host(w)) <= 1.0001e-8
