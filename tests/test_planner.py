"""Host planner pinned against the paper's iteration Tables (Sec. 4) and the
aggregation sizes; runs on CPU (planning needs no GPU)."""
import os

import pytest

from paper_1510_00903_gb300 import bbc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_iteration_tables.txt")


@pytest.fixture(scope="module")
def ctx52():
    c = bbc.bbc_create(16, 32, 0, 0.3, 0.4, bbc.BBC_FP64, list(range(52)))
    yield c
    bbc.bbc_destroy(c)


def golden_rows():
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        ch, pairs, its, tot = [x.strip() for x in line.split("|")]
        want = [int(x) for x in its.split()]
        for pr in pairs.split(";"):
            t3, t4 = map(int, pr.split(","))
            yield int(ch), t3, t4, want, int(tot)


def test_paper_iteration_tables(ctx52):
    """Every row: the same number of diagrams, the same multiset of
    (iterations x parity) and the same total as printed.  Relative signs
    within a row are compared; the overall sign of a row depends on the
    reference permutation, which the paper does not fix for rows whose
    source differs from the sink."""
    n = 0
    for ch, t3, t4, want, tot in golden_rows():
        got = bbc.bbc_plan_stats(ctx52, ch, t3, t4)
        assert sum(abs(x) for x in got) == tot, (ch, t3, t4)
        assert sorted(got) == sorted(want) or sorted(got) == sorted(-x for x in want), (ch, t3, t4, got, want)
        n += 1
    assert n == 145


def test_diagonal_rows_keep_the_printed_signs(ctx52):
    """For <B1 B2 | Bbar1 Bbar2> with identical source terms the identity
    contraction is the reference; signs then match exactly."""
    for ch, t3, t4, want, tot in golden_rows():
        if ch in (0, 5, 16, 23, 30, 46, 51) or (ch in (1, 42) and t4 == 0):
            assert sorted(bbc.bbc_plan_stats(ctx52, ch, t3, t4)) == sorted(want)


def test_aggregation_sizes(ctx52):
    """52 channels, upper spin components: 655 diagram instances with
    43,507 open-index iterations per spin (sum of the Tables' totals), stored
    as 24 shared blocks of 7,368 complex entries per site (Appendix A
    aggregation, including the sub-block identity n^(2) in n^(3)), and 153
    block-pair tasks: 255 distinct ones, 175 once tasks equal up to the order
    of their two open indices are merged, 153 once tasks whose products all
    vanish (every step meets a row whose weights cancelled) are dropped --
    174,208 complex multiply-adds per site per q."""
    s = bbc.bbc_plan_sizes(ctx52)
    assert s["blocks"] == 24
    assert s["block_outputs"] == 7368
    assert s["pair_items"] == 16 * 153
    assert s["pair_macs_per_site"] == 174208
    total, n_diag = 0, 0
    for pos in range(52):
        for t3 in range(3):
            for t4 in range(3):
                d = bbc.bbc_plan_stats(ctx52, pos, t3, t4)
                total += sum(abs(x) for x in d)
                n_diag += len(d)
    assert (n_diag, total) == (655, 43507)


def test_single_channel_plan():
    c = bbc.bbc_create(4, 4, 0, 0.3, 0.4, bbc.BBC_FP64, [1])
    try:
        s = bbc.bbc_plan_sizes(c)
        assert s["blocks"] > 0 and s["block_outputs"] > 0
        assert [sum(abs(x) for x in bbc.bbc_plan_stats(c, 0, 0, t)) for t in range(3)] == [370, 397, 370]
    finally:
        bbc.bbc_destroy(c)
