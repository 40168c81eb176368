"""Microstructure generator on the GPU (Sec. 2.2, Algorithms 4 and 5) against the brute-force
oracle: grain ids and pore voxels must be identical (integer results, bit-exact)."""
import numpy as np
import pytest

from paper_2602_07354_gb300 import binding as B
from paper_2602_07354_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_07354_gb300 import build

    build.build()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("dims,n,seed", [((23, 17, 19), 40, 1), ((48, 48, 48), 300, 2), ((8, 6, 50), 5, 3),
                                         ((2, 3, 2), 2, 4), ((33, 31, 29), 1, 5)])
def test_grain_ids_equal_the_oracle(oracle, dims, n, seed):
    rng = np.random.default_rng(seed)
    seeds = rng.random((n, 3)) * np.array(dims)
    ph = host(B.elas_assign_grains(dims, seeds))
    assert np.array_equal(ph, oracle.assign_grains(dims, seeds))


def test_weighted_grains_equal_the_oracle(oracle):
    rng = np.random.default_rng(6)
    dims = (30, 26, 34)
    seeds = rng.random((60, 3)) * np.array(dims)
    semi = np.stack([rng.uniform(0.5, 2.0, 60), rng.uniform(1.0, 4.0, 60)], 1)  # prolate grains along z
    ph = host(B.elas_assign_grains(dims, seeds, semi))
    assert np.array_equal(ph, oracle.assign_grains(dims, seeds, semi))


def test_exact_ties_go_to_the_lowest_index(oracle):
    # seeds 0 and 1 straddle the plane x = 5.5 at equal distance (exact in binary): that plane of
    # voxel centres belongs to grain 0; swapping the seeds' order hands it to the other seed
    dims = (11, 7, 5)
    seeds = np.array([[2.5, 3.5, 2.5], [8.5, 3.5, 2.5]])
    ph = host(B.elas_assign_grains(dims, seeds)).reshape(5, 7, 11)
    assert np.array_equal(ph.ravel(), oracle.assign_grains(dims, seeds))
    assert (ph[:, :, 5] == 0).all()
    ph2 = host(B.elas_assign_grains(dims, seeds[::-1].copy())).reshape(5, 7, 11)
    assert (ph2[:, :, 5] == 0).all() and (ph2[:, :, 2] == 1).all()


def _rot(rng):
    q = rng.normal(size=4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_pores_equal_the_oracle(oracle):
    rng = np.random.default_rng(7)
    dims = (40, 36, 44)
    seeds = rng.random((50, 3)) * np.array(dims)
    pores = []
    for p in range(30):
        c = rng.random(3) * np.array(dims)
        if p % 2:
            r = rng.uniform(1.0, 5.0)
            pores.append(np.concatenate([c, [r, r, r], np.eye(3).ravel()]))
        else:
            a = rng.uniform(1.0, 3.0)
            pores.append(np.concatenate([c, [a, a * rng.uniform(1, 2), a * rng.uniform(3, 6)], _rot(rng).ravel()]))
    pores = np.array(pores)
    ph = B.elas_assign_grains(dims, seeds)
    n_gpu = B.elas_stamp_pores(dims, pores, ph)
    ref = oracle.assign_grains(dims, seeds)
    n_ref = oracle.stamp_pores(dims, pores, ref)
    assert n_gpu == n_ref > 0
    assert np.array_equal(host(ph), ref)


def test_full_size_sampled_against_the_oracle(oracle):
    # the 500^3 cell with 20,000 grains of the large-solve workload: sampled voxels against the
    # brute-force oracle, and the whole grid against the host generator's k-d tree
    dims = (500, 500, 500)
    rng = np.random.Generator(np.random.PCG64(3))
    seeds = rng.random((20000, 3)) * np.array(dims)
    ph = B.elas_assign_grains(dims, seeds)
    vox = np.random.default_rng(8).choice(500 ** 3, size=3000, replace=False)
    got = host(ph[torch.from_numpy(vox).to("cuda")])
    assert np.array_equal(got, oracle.assign_voxels(dims, seeds, vox))
    assert (host(ph[:: 997]) >= 0).all()


def test_bad_arguments_are_refused():
    with pytest.raises(B.ElasError):
        B.elas_assign_grains((8, 8, 8), np.array([[8.0, 1.0, 1.0]]))  # seed outside [0, n)
    ph = B.elas_assign_grains((8, 8, 8), np.array([[1.0, 1.0, 1.0]]))
    with pytest.raises(B.ElasError):
        B.elas_stamp_pores((8, 8, 8), np.concatenate([[4, 4, 4], [4.5, 1, 1], np.eye(3).ravel()])[None], ph)
