"""The autotuner's coordinate search (host logic, no GPU)."""
from paper_2008_13461_gb300.autotune import SPACE, coordinate_search


def test_coordinate_search_finds_the_separable_minimum_and_evaluates_each_tuning_once():
    best_v = {knob: values[-1] for knob, values in SPACE}      # a corner of the space
    calls = []

    def cost(t):
        calls.append(tuple(sorted(t.items())))
        return sum(0 if t[k] == v else 1 + abs(t[k] - v) / v for k, v in best_v.items())

    base = {knob: values[0] for knob, values in SPACE}
    base["connect_lanes"] = 8
    best, seen = coordinate_search(cost, base, SPACE)
    assert {k: best[k] for k in best_v} == best_v
    assert best["connect_lanes"] == 8                 # not a searched knob
    assert len(calls) == len(set(calls)) == len(seen)


def test_coordinate_search_keeps_the_base_when_nothing_is_faster():
    base = {"n_t_bins": 32, "n_phi_bins": 128, "doublet_lanes": 8, "blocks_per_sm": 8}
    best, seen = coordinate_search(lambda t: 0.0 if t == base else 1.0, base, SPACE)
    assert best == base
