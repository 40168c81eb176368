"""Sec. 3.1's Eshelby-void benchmark against the analytic cavity field: an isotropic matrix
(E = 194 GPa, nu = 0.2934) with a central spherical void of radius 2/50 of the edge under the
macroscopic strain eps_33 = 1e-3, solved on the GPU; the voxel stresses on the three central
planes (the planes of the paper's Fig. 5) are compared with the closed-form field of tests/cavity.py,
and the App. C peak with the analytic surface maximum."""
import numpy as np
import pytest

import cavity
from paper_2602_07354_gb300 import binding as B
from paper_2602_07354_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_M, NU_M = 194.0, 0.2934
MU_M = E_M / (2 * (1 + NU_M))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_07354_gb300 import build

    build.build()


def _central_planes(n):
    """Voxel indices of the three central planes and their centres relative to the void centre."""
    i = np.arange(n)
    h = n // 2
    idx = []
    for ax in range(3):
        a, b = np.meshgrid(i, i, indexing="ij")
        ijk = [a.ravel(), b.ravel()]
        ijk.insert(ax, np.full(a.size, h))
        idx.append(np.stack(ijk, 1))
    ijk = np.unique(np.concatenate(idx), axis=0)
    lin = ijk[:, 0] + n * (ijk[:, 1] + n * ijk[:, 2])
    return lin, ijk + 0.5 - n / 2.0


@pytest.mark.parametrize("n", [200])
def test_void_field_matches_the_analytic_cavity(n):
    ms = synth.eshelby_void(n)
    a = 2.0 / 50.0 * n
    E = np.diag([0.0, 0.0, 1e-3])
    e6 = np.array([0, 0, 1e-3, 0, 0, 0.0])
    ctx = B.create_from_micro(ms, precision=B.PREC_MIXED)
    info = B.elas_pcg_solve(ctx, e6, 1e-8, 20000, stop_rule=B.STOP_TRUE)
    assert info["status"] == B.CONVERGED
    s6 = torch.empty(6 * ms.N, dtype=torch.float64, device="cuda")
    vm = torch.empty(ms.N, dtype=torch.float64, device="cuda")
    B.elas_stress(ctx, e6, None, s6, vm)
    lin, x = _central_planes(n)
    s = s6.view(6, ms.N)[:, torch.from_numpy(lin).to("cuda")].cpu().numpy().T
    v = vm[torch.from_numpy(lin).to("cuda")].cpu().numpy()
    r = np.linalg.norm(x, axis=1)
    sa = cavity.stress(x, E, MU_M, NU_M, a)
    sa6 = np.stack([sa[:, 0, 0], sa[:, 1, 1], sa[:, 2, 2], sa[:, 1, 2], sa[:, 0, 2], sa[:, 0, 1]], 1)
    lam = 2 * MU_M * NU_M / (1 - 2 * NU_M)
    s_inf = np.array([lam, lam, lam + 2 * MU_M, 0, 0, 0]) * 1e-3
    out = {}
    for lo, hi in ((a + 2, 1.5 * a), (1.5 * a, 3 * a), (3 * a, np.inf)):
        m = (r >= lo) & (r < hi)
        err = np.linalg.norm(s[m] - sa6[m]) / np.linalg.norm(sa6[m])
        perr = np.linalg.norm(s[m] - sa6[m]) / np.linalg.norm(sa6[m] - s_inf)
        vme = np.abs(v[m] - cavity.von_mises(sa[m])).max() / cavity.von_mises(sa[m]).max()
        out[(lo, hi)] = (err, perr, vme)
        print(f"\nr/a in [{lo / a:.2f}, {hi / a:.2f}): stress rel L2 {err:.2e}, of the perturbation {perr:.2e},"
              f" max von Mises error {vme:.2e}")
    near, mid, far = out.values()
    assert near[0] < 0.06 and mid[0] < 0.03 and far[0] < 0.02
    assert mid[1] < 0.15
    # App. C peak (smoothed, s = 0.4 voxels) against the analytic surface maximum
    smax, at, _ = B.elas_hotspot(ctx, vm, 0.4)
    peak = cavity.surface_peak_von_mises(E, MU_M, NU_M)
    print(f"smoothed FE peak {smax * 1e3:.1f} MPa, analytic surface peak {peak * 1e3:.1f} MPa "
          f"(ratio {smax / peak:.3f})")
    assert 0.9 < smax / peak < 1.05
