"""The seeded input generators (no GPU): SplitMix64 against its published outputs, and the
designs and outcomes against the properties their docstrings state."""
import numpy as np

import synth
from synth.designs import SplitMix64, draw_outcomes, kset_design, tapestry_like_design


def test_splitmix64_known_answers():
    """First outputs of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; the reference C code that
    seeds the xoshiro generators) for seed 1234567."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [int(v) for v in SplitMix64(1234567).u64(5)] == want
    r = SplitMix64(1234567)                      # the stream continues across calls
    assert [int(v) for v in np.concatenate([r.u64(2), r.u64(3)])] == want


def test_kset_rows_are_distinct_sorted_pools():
    ptr, pools = kset_design(1298, 97, 6, 5007)
    rows = pools.reshape(1298, 6)
    assert ptr.tolist() == list(range(0, 1299 * 6, 6))
    assert (np.diff(rows, axis=1) > 0).all() and rows.min() >= 0 and rows.max() < 97
    assert np.array_equal(kset_design(1298, 97, 6, 5007)[1], pools)
    assert not np.array_equal(kset_design(1298, 97, 6, 5008)[1], pools)


def test_tapestry_shapes_are_regular():
    """Each sample in 3 pools and every pool the same size: 20 per pool at 320 x 48 and 31 per
    pool at 961 x 93, the Tapestry designs' shapes."""
    for n, m, size in ((320, 48, 20), (961, 93, 31)):
        ptr, pools = tapestry_like_design(n, m, 3, 90 + m)
        rows = pools.reshape(n, 3)
        assert (np.diff(rows, axis=1) > 0).all()
        assert (np.bincount(pools, minlength=m) == size).all()
    sizes = np.bincount(tapestry_like_design(100, 7, 3, 1)[1], minlength=7)
    assert sizes.max() - sizes.min() <= 1        # 300 slots over 7 pools: 42 or 43


def test_noiseless_outcomes_are_the_latent_pool_states():
    ptr, pools = kset_design(200, 30, 4, 3)
    positives, y = draw_outcomes(200, 30, ptr, pools, 5, 0.0, 0.0, 4)
    assert len(set(positives.tolist())) == 5
    latent = np.zeros(30, np.uint8)
    for i in positives:
        latent[pools[ptr[i]:ptr[i + 1]]] = 1
    assert np.array_equal(y, latent)


def test_bench_horizon():
    assert synth.budget_horizon(4e10, 524288) == 38146


def test_batched_instances_follow_their_recipe():
    """n in [200, 5000], m = round(n / 13), k in 4..8, 1..6 positives, fp in [.005, .1],
    fn in [.02, .25], q = positives / n; every instance valid for the library."""
    from paper_2608_30239_gb300 import mcpd
    for inst in synth.batched_configs(count=24, seed=11):
        k = int(np.diff(inst.clone_ptr)[0])
        assert 200 <= inst.n <= 5000 and inst.m == int(np.floor(inst.n / 13 + 0.5))
        assert 4 <= k <= 8 and (np.diff(inst.clone_ptr) == k).all()
        assert 1 <= len(inst.positives) <= 6 and np.isclose(inst.q, len(inst.positives) / inst.n)
        assert 0.005 <= inst.fp <= 0.1 and 0.02 <= inst.fn <= 0.25
        mcpd.mcpd_inspect(inst, slots=16, horizon=20 * inst.n)


def test_mixed_degree_rows():
    """Each clone's degree lies in [deg_lo, deg_hi], its pools distinct and sorted; every degree
    in the range occurs on a design of this size."""
    from synth.designs import mixed_degree_design
    ptr, pools = mixed_degree_design(260, 23, 2, 8, 31)
    degs = np.diff(ptr)
    assert degs.min() >= 2 and degs.max() <= 8 and set(degs.tolist()) == set(range(2, 9))
    for i in range(260):
        row = pools[ptr[i]:ptr[i + 1]]
        assert (np.diff(row) > 0).all() and row.min() >= 0 and row.max() < 23
