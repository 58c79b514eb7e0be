"""The autotuner's host-side rules, without a GPU: checkpoint memory per spacing M and the choice
among timed candidates (fastest; within the tie margin, the fewest checkpoint bytes)."""

import pytest

from paper_2304_06200_gb300.hg import checkpoint_bytes, select_candidate


def test_checkpoint_bytes_follow_the_spacing_rule():
    # C3: d = 4000, n = 4, N = 2000; one stored state is 4000 * 4 complex128 = 256,000 bytes
    assert checkpoint_bytes(50, 2000, 4000, 4) == 39 * 256_000       # floor(1999 / 50) = 39
    assert checkpoint_bytes(0, 2000, 4000, 4) == 39 * 256_000        # 0 = automatic: M = min(50, N)
    assert checkpoint_bytes(200, 2000, 4000, 4) == 9 * 256_000
    assert checkpoint_bytes(1000, 2000, 4000, 4) == 1 * 256_000
    assert checkpoint_bytes(-1, 2000, 4000, 4) == 0                  # no checkpoints
    assert checkpoint_bytes(0, 30, 10, 2) == 0                       # automatic M = N: none stored
    assert checkpoint_bytes(1, 5, 3, 1) == 4 * 48                    # every step but the last
    assert checkpoint_bytes(7, 1, 3, 1) == 0                         # a single step stores nothing


def _cand(ms, mem, tag):
    return {"ms": ms, "checkpoint_bytes_full_N": mem, "tag": tag}


def test_fastest_wins_outside_the_tie_margin():
    c = [_cand(10.0, 100, "a"), _cand(12.0, 0, "b"), _cand(10.5, 0, "c")]
    assert select_candidate(c, tie=0.02)["tag"] == "a"               # 10.5 is 5% slower


def test_least_memory_wins_inside_the_tie_margin():
    c = [_cand(10.0, 100, "a"), _cand(10.15, 10, "b"), _cand(10.19, 0, "c"), _cand(10.3, 0, "d")]
    assert select_candidate(c, tie=0.02)["tag"] == "c"               # within 2%: fewest bytes
    assert select_candidate(c, tie=0.0)["tag"] == "a"


def test_equal_memory_prefers_the_faster():
    c = [_cand(10.1, 5, "a"), _cand(10.0, 5, "b")]
    assert select_candidate(c, tie=0.05)["tag"] == "b"


def test_no_candidate_is_an_error():
    with pytest.raises(RuntimeError):
        select_candidate([], tie=0.02)
