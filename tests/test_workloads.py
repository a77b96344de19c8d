"""Seeded input generators (workloads.py): the counter-based SplitMix64
stream against its published definition written out with Python integers,
the ranges and structure of each recipe, and the receding-horizon step."""
import numpy as np

from paper_1903_10041_gb300 import workloads as W

MASK = (1 << 64) - 1


def _splitmix_finalizer(z: int) -> int:
    # SplitMix64 output function (Steele, Lea, Flood 2014): xor-shift 30, 27, 31
    # with the two published odd multipliers
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def test_uniform_is_the_splitmix64_stream():
    seed, tags, size = 1903, (11, 5), 7
    key = seed & MASK
    for t in tags:
        key = _splitmix_finalizer(key ^ t)
    gamma = 0x9E3779B97F4A7C15  # the golden-ratio increment
    want = [(_splitmix_finalizer((key + i * gamma) & MASK) >> 11) / 2.0**53 for i in range(1, size + 1)]
    assert np.array_equal(W.uniform(seed, tags, size), np.array(want))


def test_recipes_have_the_stated_ranges_and_shapes():
    P = W.config(2)
    assert (P.n, P.m, P.q) == (100_000, 4, 20) and P.f2.shape == (4, 20, 100_000)
    assert P.f2.min() >= 0.1 and P.f2.max() < 1.0 and P.g2.min() >= 0.01 and P.g2.max() < 0.1
    assert np.all(P.lo == -1.0) and np.all(P.hi == 2.0) and P.y.min() >= 0.5 and P.y.max() < 2.0
    # c = 0.6 min_j sum_k g(2): the split x = y/m stays within it
    g_split = (P.g2 * (P.y / P.m)[None] ** 2 + P.g1 * (P.y / P.m)[None]).sum(axis=2)
    assert np.all(g_split.max(axis=1) <= P.c)
    H = W.config(1)
    assert np.all(H.g2[0] == 0) and np.all(H.g1[0] == 0) and np.isinf(H.c[0]) and H.c[1] == 0.3 * H.n
    assert np.all(H.f2[1] == 0) and np.all(H.lo[0] == 0.0) and np.all(H.hi[0] == 3.0)


def test_batched_shapes_cover_the_stated_ranges():
    shapes = [W.batch_shape(t) for t in range(4096)]
    n = np.array([s[0] for s in shapes])
    assert n.min() >= 50 and n.max() <= 5000
    assert {s[1] for s in shapes} == {2, 3, 4} and {s[2] for s in shapes} == set(range(1, 21))
    assert abs(np.median(np.log(n)) - np.log(500.0)) < 0.1  # log-uniform on [50, 5000]


def test_shared_maps_expand_to_the_dense_problem():
    S = W.shared_problem(30, 3, 4, seed=9)
    D = S.dense()
    assert S.coef_shared and not D.coef_shared and D.f2.shape == (3, 4, 30)
    for j in range(4):
        assert np.array_equal(D.g2[:, j, :], S.g2)
    assert np.array_equal(D.y, S.y) and np.array_equal(D.c, S.c)


def test_receding_step_moves_every_per_step_array_one_step():
    P = W.random_problem(40, 2, 3, seed=4)
    Q = W.receding_step(P, step=1, seed=4)
    for k in ("f2", "f1", "g2", "g1"):
        assert np.array_equal(getattr(Q, k)[:, :, :-1], getattr(P, k)[:, :, 1:])
    assert np.array_equal(Q.y[:, :-1], P.y[:, 1:]) and np.array_equal(Q.c, P.c)
    d = W.step_data(2, 3, 1, seed=4)
    assert np.array_equal(Q.f2[:, :, -1], d["f2"]) and np.array_equal(Q.y[:, -1], d["y"])
