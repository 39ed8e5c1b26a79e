"""The autotuner's choice rule (host logic, no GPU): the fastest candidate
wins unless the library default is within the tie margin, so the chosen
kernels do not flip between runs on timing noise."""
import pytest

from paper_1708_02574_gb300.autotune import TIE, pick_fastest, pick_query


def test_pick_fastest():
    assert pick_fastest({0: 1.0, 1: 0.5, 2: 0.7}, default=0) == 1
    assert pick_fastest({0: 1.02, 1: 1.0}, default=0) == 0                 # within the margin: the default stays
    assert pick_fastest({0: 1.0 + 2 * TIE, 1: 1.0}, default=0) == 1
    assert pick_fastest({1: 2.0, 2: 1.0}, default=0) == 2                  # the default was not timed
    assert pick_fastest({3: 1.0}, default=3) == 3


def test_pick_query():
    defaults = {4: 10, 8: 20}
    res = [{"width": 4, "variant": 10, "seeds_per_s": 100.0}, {"width": 4, "variant": 11, "seeds_per_s": 150.0},
           {"width": 8, "variant": 20, "seeds_per_s": 148.0}, {"width": 8, "variant": 21, "seeds_per_s": 140.0}]
    # the best (width 4, variant 11) is not a default; its width's default is far behind,
    # the default width's default (8, 20) is within the margin
    assert pick_query(res, defaults, default_width=8) == res[2]
    res[2]["seeds_per_s"] = 120.0
    assert pick_query(res, defaults, default_width=8) == res[1]
    res[0]["seeds_per_s"] = 149.0                                          # the best width's default now ties
    assert pick_query(res, defaults, default_width=8) == res[0]
    with pytest.raises(ValueError):
        pick_query([], defaults, default_width=8)
