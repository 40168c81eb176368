"""Solve server: continuous batching under a memory budget, results independent of the mix."""
import numpy as np
import pytest

from paper_2602_07354_gb300 import binding as B
from paper_2602_07354_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_ZZ = np.array([0, 0, 1e-3, 0, 0, 0.0])


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_07354_gb300 import build

    build.build()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def drain(srv, ids, sizes, max_steps=10000):
    out = {}
    for _ in range(max_steps):
        B.elas_server_step(srv)
        for rid in list(ids):
            if rid in out:
                continue
            w = torch.empty(3 * sizes[rid], dtype=torch.float64, device="cuda")
            r = B.elas_server_poll(srv, rid, w)
            if r is not None:
                out[rid] = (r, host(w))
        if len(out) == len(ids):
            return out
    raise AssertionError("server did not finish")


def test_result_same_alone_in_mix_and_in_a_plain_solve(oracle):
    target = synth.polycrystal(20, 10, pore_frac=0.02, seed=21, dims=(20, 18, 22))
    others = [synth.polycrystal(n, max(2, n ** 3 // 2000), pore_frac=0.02, seed=30 + n) for n in (16, 24, 28)]
    strain = synth.random_symmetric_strain(np.random.default_rng(5))
    # alone
    srv = B.elas_server_create(1 << 30, 8)
    rid = B.elas_server_submit(srv, target, strain, 1e-8, 5000)
    alone = drain(srv, [rid], {rid: target.N})[rid]
    srv.close()
    # in a mix: two requests first, the target arrives while they run, one more after it
    srv = B.elas_server_create(1 << 30, 8)
    sizes = {}
    ids = [B.elas_server_submit(srv, others[0], E_ZZ, 1e-8, 5000), B.elas_server_submit(srv, others[1], E_ZZ, 1e-6, 5000)]
    for i in ids:
        sizes[i] = srv.sizes[i]
    B.elas_server_step(srv)
    t = B.elas_server_submit(srv, target, strain, 1e-8, 5000)
    B.elas_server_step(srv)
    last = B.elas_server_submit(srv, others[2], strain, 1e-8, 5000)
    sizes.update({t: target.N, last: others[2].N})
    res = drain(srv, ids + [t, last], sizes)
    assert res[t][0]["iters"] == alone[0]["iters"]
    assert np.array_equal(res[t][1], alone[1])
    assert all(r[0]["status"] == B.CONVERGED for r in res.values())
    # the same problem through a plain context (same kernels, same schedule)
    ctx = B.create_from_micro(target, precision=B.PREC_MIXED)
    w = torch.empty(3 * target.N, dtype=torch.float64, device="cuda")
    B.elas_pcg_solve(ctx, strain, 1e-8, 5000, w_out=w)
    assert np.array_equal(host(w), alone[1])
    # and against the oracle's FP64 residual
    p = oracle.Problem.from_micro(target)
    assert p.true_relres(strain, alone[1]) <= 1.0001e-8


def test_replacement_policy_matches_plain_solve_options(oracle):
    # residual-drop replacement (every 1000 iterations at most, or after 3 decades of residual
    # reduction): the same iterates as a plain solve given the same options
    target = synth.polycrystal(24, 8, pore_frac=0.02, seed=41)
    strain = synth.random_symmetric_strain(np.random.default_rng(6))
    srv = B.elas_server_create(1 << 30, 4)
    B.elas_server_set_replacement(srv, 1000, 3)
    rid = B.elas_server_submit(srv, target, strain, 1e-8, 5000)
    r, w_srv = drain(srv, [rid], {rid: target.N})[rid]
    srv.close()
    assert r["status"] == B.CONVERGED and 1 <= r["n_replacements"] <= 4
    ctx = B.create_from_micro(target, precision=B.PREC_MIXED)
    w = torch.empty(3 * target.N, dtype=torch.float64, device="cuda")
    info = B.elas_pcg_solve(ctx, strain, 1e-8, 5000, w_out=w, replace_every=1000, replace_drop=3)
    assert info["iters"] == r["iters"] and info["n_replacements"] == r["n_replacements"]
    assert np.array_equal(host(w), w_srv)
    assert oracle.Problem.from_micro(target).true_relres(strain, w_srv) <= 1.0001e-8


def test_budget_limits_admission_and_memory_returns():
    ms = [synth.polycrystal(24, 7, pore_frac=0.01, seed=40 + k) for k in range(5)]
    per = B.elas_workspace_bytes(24, 24, 24, 7, B.PREC_MIXED)  # a context's footprint ~ a request's
    budget = int(per * 2.2)
    srv = B.elas_server_create(budget, 8)
    ids = [B.elas_server_submit(srv, m, E_ZZ, 1e-6, 5000) for m in ms]
    sizes = {i: m.N for i, m in zip(ids, ms)}
    active, queued, _ = B.elas_server_step(srv)
    assert active <= 2 and active + queued <= 5
    st = B.elas_server_stats(srv)
    assert 0 < st["bytes_in_use"] <= budget
    res = drain(srv, ids, sizes)
    assert all(r[0]["status"] == B.CONVERGED for r in res.values())
    st = B.elas_server_stats(srv)
    assert st["bytes_in_use"] == 0 and st["done"] == 5 and st["active"] == 0


def test_oversized_request_is_refused():
    srv = B.elas_server_create(1 << 21, 4)
    big = synth.polycrystal(40, 8, pore_frac=0.0, seed=1)
    with pytest.raises(B.ElasError) as ei:
        B.elas_server_submit(srv, big, E_ZZ, 1e-6, 100)
    assert ei.value.code == -6


def test_cancel_queued_and_running_requests():
    ms = [synth.polycrystal(n, max(2, n ** 3 // 2000), pore_frac=0.02, seed=60 + n) for n in (20, 24, 28)]
    srv = B.elas_server_create(1 << 30, 1)  # one slot: the later requests wait in the queue
    ids = [B.elas_server_submit(srv, m, E_ZZ, 1e-8, 5000) for m in ms]
    B.elas_server_step(srv)  # admits the first request and runs K iterations of it
    B.elas_server_cancel(srv, ids[0])  # running: stops at the next step
    B.elas_server_cancel(srv, ids[1])  # queued: withdrawn at once
    with pytest.raises(B.ElasError):
        B.elas_server_cancel(srv, 10 ** 9)
    res = drain(srv, ids, {i: m.N for i, m in zip(ids, ms)})
    r0, r1, r2 = (res[i][0] for i in ids)
    assert r0["status"] == B.CANCELLED and 0 < r0["iters"] < 5000 and r0["relres_true"] > 1e-8
    assert r1["status"] == B.CANCELLED and r1["iters"] == 0
    assert r2["status"] == B.CONVERGED
    assert B.elas_server_stats(srv)["bytes_in_use"] == 0
    srv.close()
