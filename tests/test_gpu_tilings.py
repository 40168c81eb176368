"""The operator product and the solve against the oracle under tilings forced through the tuning
cache, not only under the tile model's or the autotuner's choice: tiles of a few nodes with
one-layer chunks, one tile holding the whole grid, and ragged edges in x, y and z.  The grid size
is used by no other test, so the forced entries cannot leak into them."""
import numpy as np
import pytest

from paper_2602_07354_gb300 import binding as B
from paper_2602_07354_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS = (19, 14, 9)
# (bytes per element, tx, ty, kc): 8 = the FP64 operator (<= 384 threads), 4 = FP32 (<= 256)
CASES = [(8, 4, 2, 1), (8, 5, 3, 4), (8, 19, 14, 9), (8, 6, 13, 2), (4, 4, 2, 1), (4, 15, 14, 3), (4, 7, 6, 9)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_07354_gb300 import build

    build.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _force(eb, tx, ty, kc):
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    line = f"{DIMS[0]} {DIMS[1]} {DIMS[2]} {eb} {sm} {tx} {ty} {kc}"
    B.elas_tuning_import(line + "\n")
    assert line in B.elas_tuning_export().splitlines()


@pytest.mark.parametrize("eb,tx,ty,kc", CASES)
def test_forced_tilings_match_the_oracle(oracle, eb, tx, ty, kc):
    _force(eb, tx, ty, kc)
    ms = synth.random_problem(DIMS, 4, np.random.default_rng(tx + 10 * ty + 100 * kc), pore_prob=0.12)
    p = oracle.Problem.from_micro(ms)
    rng = np.random.default_rng(5)
    e6 = np.array([0.0, 4e-4, 1e-3, 0.0, 2e-4, 0.0])
    if eb == 8:
        ctx = B.create_from_micro(ms, precision=B.PREC_FP64)
        u = rng.normal(size=3 * p.N)
        y = torch.empty(3 * p.N, dtype=torch.float64, device="cuda")
        B.elas_apply(ctx, torch.from_numpy(u).cuda(), y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), p.apply(u)) <= 1e-12
        # Algorithm 2's iterates: same stopping rule, same count, same w
        ref = p.pcg(e6, 1e-10, 3000)
        w = torch.empty(3 * p.N, dtype=torch.float64, device="cuda")
        info = B.elas_pcg_solve(ctx, e6, 1e-10, 3000, w_out=w, stop_rule=B.STOP_PRECOND)
        torch.cuda.synchronize()
        assert info["status"] == B.CONVERGED and abs(info["iters"] - ref["iters"]) <= 1
        assert rel(w.cpu().numpy(), ref["w"]) <= 1e-7
    else:
        ctx = B.create_from_micro(ms, precision=B.PREC_MIXED)
        u = rng.normal(size=3 * p.N).astype(np.float32)
        y = torch.empty(3 * p.N, dtype=torch.float32, device="cuda")
        B.elas_apply_f32(ctx, torch.from_numpy(u).cuda(), y)
        torch.cuda.synchronize()
        assert rel(y.cpu().numpy(), p.apply(u.astype(np.float64))) <= 2e-6
        w = torch.empty(3 * p.N, dtype=torch.float64, device="cuda")
        info = B.elas_pcg_solve(ctx, e6, 1e-8, 3000, w_out=w)
        torch.cuda.synchronize()
        assert info["status"] == B.CONVERGED
        assert p.true_relres(e6, w.cpu().numpy()) <= 1.0001e-8  # recomputed by the oracle
    ctx.close()


@pytest.mark.parametrize("dims", [(2, 3, 200), (300, 2, 2), (2, 150, 2), (64, 2, 7)])
def test_extreme_aspect_ratios_match_the_oracle(oracle, dims):
    # the default tiling of needle and plate grids (tiles far wider than the grid in some
    # direction, wrap onto the tile's own nodes) for both operator precisions and an FP64 solve
    ms = synth.random_problem(dims, 3, np.random.default_rng(sum(dims)), pore_prob=0.1)
    p = oracle.Problem.from_micro(ms)
    rng = np.random.default_rng(9)
    u = rng.normal(size=3 * p.N)
    ctx = B.create_from_micro(ms, precision=B.PREC_FP64)
    y = torch.empty(3 * p.N, dtype=torch.float64, device="cuda")
    B.elas_apply(ctx, torch.from_numpy(u).cuda(), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), p.apply(u)) <= 1e-12
    e6 = np.array([3e-4, 0.0, 1e-3, 0.0, 0.0, -2e-4])
    ref = p.pcg(e6, 1e-10, 20000)
    w = torch.empty(3 * p.N, dtype=torch.float64, device="cuda")
    info = B.elas_pcg_solve(ctx, e6, 1e-10, 20000, w_out=w, stop_rule=B.STOP_PRECOND)
    torch.cuda.synchronize()
    assert info["status"] == B.CONVERGED and abs(info["iters"] - ref["iters"]) <= 1
    assert rel(w.cpu().numpy(), ref["w"]) <= 1e-7
    ctx.close()
    ctx = B.create_from_micro(ms, precision=B.PREC_MIXED)
    u32 = u.astype(np.float32)
    y32 = torch.empty(3 * p.N, dtype=torch.float32, device="cuda")
    B.elas_apply_f32(ctx, torch.from_numpy(u32).cuda(), y32)
    torch.cuda.synchronize()
    assert rel(y32.cpu().numpy(), p.apply(u32.astype(np.float64))) <= 2e-6
    ctx.close()
