"""The seeded input generators shared by the tests and the benchmark (no GPU): the serving stream's
arrivals follow the requested Poisson rate, and every request's own recipe (grid, tolerance, strain,
microstructure seed) depends only on its index, not on the rate."""
import numpy as np

from paper_2602_07354_gb300 import synth


def test_request_stream_arrivals_follow_the_rate():
    for rate in (20.0, 10.0):
        reqs = synth.request_stream(2000, rate=rate)
        t = np.array([r["arrival"] for r in reqs])
        assert np.all(np.diff(t) > 0)
        gaps = np.diff(np.concatenate([[0.0], t]))
        # exponential gaps: mean 1/rate, standard error of the mean (1/rate)/sqrt(2000) = 2.2%
        assert abs(gaps.mean() * rate - 1.0) < 0.1
        assert abs(gaps.std() * rate - 1.0) < 0.1


def test_request_recipes_do_not_depend_on_the_rate():
    a = synth.request_stream(50, rate=20.0)
    b = synth.request_stream(50, rate=10.0)
    for ra, rb in zip(a, b):
        assert ra["edge"] == rb["edge"] and ra["tol"] == rb["tol"] and ra["seed"] == rb["seed"]
        assert ra["n_grains"] == rb["n_grains"] and ra["pore_frac"] == rb["pore_frac"]
        np.testing.assert_array_equal(ra["strain"], rb["strain"])
        assert ra["edge"] in (48, 64, 96, 128, 160) and ra["tol"] in (1e-6, 1e-8)
        e = ra["strain"]  # tensor components E11, E22, E33, E23, E13, E12
        E = np.array([[e[0], e[5], e[4]], [e[5], e[1], e[3]], [e[4], e[3], e[2]]])
        assert abs(np.linalg.norm(E) - 1e-3) < 1e-15
