"""Seeded DC-SBM input generator: shapes, determinism and planted structure."""
import numpy as np

from paper_2508_19737_gb300 import synth


def test_equal_blocks_of_the_small_config():
    g = synth.dcsbm(1000, 11, 20, 2.5, 10, seed=0)
    sizes = np.bincount(g.blocks)
    assert sorted(sizes.tolist()) == [90] + [91] * 10
    assert g.M == 10000 and g.src.dtype == np.int32
    assert g.src.min() >= 0 and g.src.max() < 1000


def test_deterministic_by_seed():
    a = synth.dcsbm(5000, 7, 12, 2.5, 4, seed=3, dirichlet_alpha=2)
    b = synth.dcsbm(5000, 7, 12, 2.5, 4, seed=3, dirichlet_alpha=2)
    c = synth.dcsbm(5000, 7, 12, 2.5, 4, seed=4, dirichlet_alpha=2)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    assert not np.array_equal(a.src, c.src)


def test_per_pair_ratio_gives_expected_intra_fraction():
    # equal blocks and equal propensity mass: intra fraction = r / (r + B - 1)
    N, B, r = 20000, 8, 6.0
    g = synth.dcsbm(N, B, 20, 2.5, r, seed=1)
    th = g.theta
    Tb = np.bincount(g.blocks, weights=th)
    # exact expectation for P(u,v) ~ th_u th_v w
    intra_mass = r * np.sum(Tb ** 2)
    total = intra_mass + (Tb.sum() ** 2 - np.sum(Tb ** 2))
    expect = intra_mass / total
    got = np.mean(g.blocks[g.src] == g.blocks[g.dst])
    assert abs(got - expect) < 0.01


def test_dirichlet_sizes_nonempty_and_sum():
    rng = np.random.default_rng(0)
    s = synth.block_sizes(rng, 1000, 128, dirichlet_alpha=0.3)
    assert s.sum() == 1000 and s.min() >= 1


def test_block_degree_order_is_block_major():
    g = synth.dcsbm(3000, 5, 10, 2.2, 6, seed=2, dirichlet_alpha=5, order="block_degree")
    assert np.all(np.diff(g.blocks) >= 0)


def test_snowball_increments_are_induced_and_growing():
    g = synth.dcsbm(2000, 6, 10, 2.5, 5, seed=5)
    incs = synth.split_increments(g, T=10, mode="snowball", seed=1)
    assert len(incs) == 10
    sizes = [n for _, _, n in incs]
    assert sizes == sorted(sizes) and sizes[-1] == 2000
    assert sum(s.size for s, _, _ in incs) == g.M
    for s, d, n in incs:
        if s.size:
            assert max(s.max(), d.max()) < n


def test_random_increments_partition_edges():
    g = synth.dcsbm(500, 3, 8, 2.5, 5, seed=6)
    incs = synth.split_increments(g, T=10, mode="random", seed=1)
    allk = np.sort(np.concatenate([s.astype(np.int64) * 500 + d for s, d, _ in incs]))
    assert np.array_equal(allk, np.sort(g.src.astype(np.int64) * 500 + g.dst))


def test_batch_sizes_in_range():
    gs = synth.batch_dcsbm(6, 1000, 50000, 10, 40, 2.5, 5, seed=0)
    assert len(gs) == 6
    for g in gs:
        assert 1000 <= g.N <= 50000
