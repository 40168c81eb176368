"""Independent contexts used from several host threads at once, each on its own CUDA stream (the
binding releases the interpreter lock inside every library call): every solve must give exactly
the iterations and the fluctuation it gives when the solves run one after another."""
import threading

import numpy as np
import pytest

from paper_2602_07354_gb300 import binding as B
from paper_2602_07354_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E6 = np.array([0.0, 0.0, 1e-3, 0.0, 0.0, 0.0])


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_07354_gb300 import build

    build.build()


def _solve(ms, prec, stream):
    with torch.cuda.stream(stream):
        ctx = B.create_from_micro(ms, precision=prec, stream=stream)
        w = torch.empty(3 * ms.N, dtype=torch.float64, device="cuda")
        info = B.elas_pcg_solve(ctx, E6, 1e-8, 5000, w_out=w)
        macro = B.elas_stress(ctx, E6)
        stream.synchronize()
        out = (info["status"], info["iters"], w.cpu().numpy(), macro)
        ctx.close()
    return out


def test_threads_on_separate_streams_match_sequential_solves():
    problems = [(synth.polycrystal(40, 60, pore_frac=0.02, seed=31), B.PREC_FP64),
                (synth.polycrystal(48, 80, pore_frac=0.02, seed=32), B.PREC_MIXED),
                (synth.polycrystal(36, 50, pore_frac=0.03, seed=33, dims=(36, 44, 28)), B.PREC_MIXED),
                (synth.eshelby_inclusion(24, 6.0), B.PREC_FP64)]
    seq = [_solve(ms, prec, torch.cuda.Stream()) for ms, prec in problems]
    got = [None] * len(problems)
    errors = []

    def worker(i):
        try:
            got[i] = _solve(problems[i][0], problems[i][1], torch.cuda.Stream())
        except Exception as exc:  # reported below, in the main thread
            errors.append(exc)

    for _ in range(2):
        threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(problems))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for (st, it, w, m), (st0, it0, w0, m0) in zip(got, seq):
            assert st == st0 == B.CONVERGED and it == it0
            assert np.array_equal(w, w0) and np.array_equal(m, m0)
