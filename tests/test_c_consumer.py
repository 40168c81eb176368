"""The boundary from plain C: tests/c_consumer.c uses only include/elas.h and the CUDA runtime.
On the CPU the header must compile as strict C99 and the program must link against the in-tree
library; on the GPU the program's solve of the Eshelby inclusion cell must agree with the
binding's solve and with the oracle (Algorithm 2's iterates, the macroscopic stress)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2602_07354_gb300 import binding as B
from paper_2602_07354_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
N_EDGE, RADIUS = 12, 3.0


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime_api.h")):
        pytest.skip("no C compiler or CUDA headers")
    return cc


def _build_consumer(tmp_path):
    from paper_2602_07354_gb300 import build

    lib = build.build()
    exe = str(tmp_path / "c_consumer")
    cmd = [_cc(), "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-O1",
           "-I", os.path.join(ROOT, "include"), "-isystem", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "c_consumer.c"), "-o", exe,
           "-L", os.path.dirname(lib), "-lelas", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_header_is_c99_and_the_program_links(tmp_path):
    exe = _build_consumer(tmp_path)
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_c_program_solves_like_the_binding_and_the_oracle(tmp_path, oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _build_consumer(tmp_path)
    env = dict(os.environ, LD_LIBRARY_PATH=os.pathsep.join(
        [os.path.join(CUDA, "lib64"), os.environ.get("LD_LIBRARY_PATH", "")]))
    r = subprocess.run([exe, str(N_EDGE), str(RADIUS)], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    status, iters, relres, m11, m22 = r.stdout.split()
    assert int(status) == B.CONVERGED and float(relres) <= 1e-9
    ms = synth.eshelby_inclusion(N_EDGE, RADIUS)
    e6 = np.array([1e-3, 0, 0, 0, 0, 0])
    ctx = B.create_from_micro(ms)
    info = B.elas_pcg_solve(ctx, e6, 1e-10, 5000, stop_rule=B.STOP_PRECOND)
    macro = B.elas_stress(ctx, e6)
    assert info["iters"] == int(iters)
    assert abs(macro[0] - float(m11)) <= 1e-12 * abs(macro[0])
    assert abs(macro[1] - float(m22)) <= 1e-12 * abs(macro[0])
    p = oracle.Problem.from_micro(ms)
    ref = p.pcg(e6, 1e-10, 5000)
    assert abs(ref["iters"] - int(iters)) <= 1
    s_or = p.stress(e6, ref["w"])[0].reshape(6, -1).mean(axis=1)
    assert abs(s_or[0] - float(m11)) <= 1e-8 * abs(s_or[0])
    assert abs(s_or[1] - float(m22)) <= 1e-8 * abs(s_or[0])
