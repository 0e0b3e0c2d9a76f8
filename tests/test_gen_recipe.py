"""The seeded input recipe that stands in for the paper's meshes and
coefficients: the counter-based generator, its value distributions, and the
structure of the generated workloads (interior-only jitter, lognormal
coefficients of the stated parameters, the batched mix of element types and
sizes)."""
import math

import numpy as np
from scipy import stats

import gen


def _splitmix_sequential(seed: int, count: int) -> list[int]:
    """SplitMix64 from its published definition, one output at a time: the
    state advances by the golden-ratio gamma, then two xor-shift-multiply
    rounds and a final xor-shift."""
    mask = (1 << 64) - 1
    s = seed & mask
    out = []
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & mask
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def test_counter_form_equals_the_sequential_generator():
    for seed in (0, gen.SEED_JITTER, (1 << 63) + 5):
        got = gen.splitmix64(seed, np.arange(100, dtype=np.uint64))
        assert [int(v) for v in got] == _splitmix_sequential(seed, 100)
    # draws offset .. offset + n - 1 are the same wherever a call starts
    a = gen.uniform(gen.SEED_COEF, 50)
    assert np.array_equal(gen.uniform(gen.SEED_COEF, 20, offset=30), a[30:])


def test_uniform_and_normal_moments():
    n = 1_000_000
    u = gen.uniform(gen.SEED_JITTER, n)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) <= 5 * math.sqrt(1.0 / 12.0 / n)
    assert abs(u.var() - 1.0 / 12.0) <= 5 * math.sqrt((1.0 / 80.0 - 1.0 / 144.0) / n)
    z = gen.normal(gen.SEED_COEF, n)
    assert np.isfinite(z).all()
    assert abs(z.mean()) <= 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) <= 5 * math.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").statistic <= 2.0 / math.sqrt(n)


def test_lognormal_coefficients_of_the_workloads():
    """k_e = exp(0.5 z) in element order from the coefficient stream: the
    log has mean 0 and standard deviation 0.5."""
    prob = gen.elastic_problem(16)
    ne = prob["conn"].shape[0]
    assert np.array_equal(prob["coef"], np.exp(0.5 * gen.normal(gen.SEED_COEF, ne)))
    lk = np.log(prob["coef"])
    assert abs(lk.mean()) <= 5 * 0.5 / math.sqrt(ne)
    assert abs(lk.std() - 0.5) <= 5 * 0.5 / math.sqrt(2 * ne)
    assert np.array_equal(gen.thermal_q1_problem(8)["coef"], np.exp(0.5 * gen.normal(gen.SEED_COEF, 512)))


def test_jitter_moves_interior_nodes_only_within_the_bound():
    n, alpha = 12, 0.15
    h = 1.0 / n
    m = gen.hex_mesh(n, alpha)
    lat = gen.hex_mesh(n, 0.0)["coords"]
    d = m["coords"] - lat
    idx = np.round(lat / h).astype(int)
    interior = np.all((idx > 0) & (idx < n), axis=1)
    assert np.array_equal(d[~interior], np.zeros_like(d[~interior]))  # the domain stays the unit cube
    di = d[interior]
    assert np.abs(di).max() <= alpha * h
    assert np.abs(di).max() >= 0.99 * alpha * h  # draws fill the interval
    assert abs(di.mean()) <= 5 * alpha * h / math.sqrt(3 * di.size)
    # the displacement of node v, coordinate i, is draw 3 v + i of the jitter stream
    u = gen.uniform(gen.SEED_JITTER, 3 * lat.shape[0]).reshape(-1, 3)
    assert np.array_equal(m["coords"][interior], lat[interior] + (2.0 * u[interior] - 1.0) * (alpha * h))


def test_batched_workload_mix_and_sizes():
    """512 problems: P1, P2 and Q1 drawn with probabilities 0.5, 0.3, 0.2;
    element counts log-uniform in [1e3, 2e5] rounded to whole grids."""
    specs = gen.batch_specs(512)
    kinds = [s["type"] for s in specs]
    for t, p in (("P1", 0.5), ("P2", 0.3), ("Q1", 0.2)):
        share = kinds.count(t) / 512
        assert abs(share - p) <= 4 * math.sqrt(p * (1 - p) / 512), (t, share)
    counts = np.array([s["n"] ** 3 if s["type"] == "Q1" else 2 * s["n"] ** 2 for s in specs], dtype=float)
    assert counts.min() >= 900 and counts.max() <= 2.1e5
    # log-uniform: log counts spread evenly over [log 1e3, log 2e5]
    v = (np.log(counts) - math.log(1e3)) / (math.log(2e5) - math.log(1e3))
    assert stats.kstest(np.clip(v, 0, 1), "uniform").statistic <= 0.1
    assert int(counts.sum()) == 19_121_571  # the batched workload's element total
