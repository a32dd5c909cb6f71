"""The autotuner's choice among timed plans (host logic): the fastest plan, except that a
staged-hit variant within 1 % of it is preferred (lower DRAM traffic at a tie)."""
from paper_1504_03687_gb300 import tune


def test_staged_variant_taken_only_at_a_tie():
    timed = [((1, 10, 0), 100.0), ((1, 12, 0), 98.0), ((1, 15, 0), 98.9), ((2, 0, 0), 150.0)]
    assert tune.choose_plan(timed) == ((1, 15, 0), 98.9)  # 98.9 <= 98 * 1.01
    timed = [((1, 10, 0), 100.0), ((1, 12, 0), 98.0), ((1, 15, 0), 99.1)]
    assert tune.choose_plan(timed) == ((1, 12, 0), 98.0)  # 99.1 > 98.98


def test_fastest_staged_variant_among_ties():
    timed = [((1, 12, 0), 50.0), ((1, 18, 0), 50.4), ((1, 19, 0), 50.2), ((1, 15, 0), 50.6)]
    assert tune.choose_plan(timed) == ((1, 19, 0), 50.2)


def test_only_mixed_tiled_staged_variants_count():
    # variant 15 of another kernel (the j-streamed one has variants 0-2 only) is no staged form
    timed = [((1, 12, 0), 10.0), ((2, 15, 0), 10.05)]
    assert tune.choose_plan(timed) == ((1, 12, 0), 10.0)
    assert set(tune.STAGED_VARIANTS) == {15, 16, 17, 18, 19}
    assert all((1, v, 0) in tune.MIXED_CANDIDATES for v in tune.STAGED_VARIANTS)


def test_merge_keeps_the_buckets_not_retuned():
    from paper_1504_03687_gb300 import tune
    old = [[1.0, 2, 0, 0, 0.05], [2.0, 2, 0, 0, 0.05], [64.0, 1, 9, 0, 0.15]]
    new = [(2, 2, 1, 0, 0.04), (4, 2, 1, 0, 0.045)]
    got = tune.merge_table(old, new)
    assert [e[0] for e in got] == [1.0, 2.0, 4.0, 64.0]
    assert got[1] == [2.0, 2, 1, 0, 0.04] and got[0] == old[0] and got[3] == old[2]
    assert tune.merge_table(None, new) == [[2.0, 2, 1, 0, 0.04], [4.0, 2, 1, 0, 0.045]]
