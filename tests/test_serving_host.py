"""Host-side logic of ragged serving (no GPU): the split of a batch over the model family
(2D share, even split within a family, disjoint seeds per instance) and the inputs each group
carries."""
import numpy as np

from paper_2307_16894_gb300 import inputs, serving


def test_make_groups_split_and_seeds():
    B_total = 103
    groups = serving.make_groups(B_total, share_2d=0.75, steps=3)
    assert sum(g["B"] for g in groups) == B_total
    n2 = sum(g["B"] for g in groups if g["rom"]["d"] == 2)
    n3 = B_total - n2
    if any(g["rom"]["d"] == 3 for g in groups):
        assert n2 == round(0.75 * B_total)
    for fam in (2, 3):
        sizes = [g["B"] for g in groups if g["rom"]["d"] == fam]
        if sizes:
            assert max(sizes) - min(sizes) <= 1                      # even split within a family
    # instance b of the whole batch has seed 40000 + b: rebuild a few and compare
    b0 = 0
    for g in groups:
        d = g["rom"]["d"]
        assert g["paths"].shape == (g["B"], 3, d, d) and g["mu"].shape[0] == g["B"]
        lo, hi = (0.2, 0.35) if d == 2 else (0.15, 0.35)
        assert np.all(g["mu"] >= lo) and np.all(g["mu"] <= hi)
        for b in (0, g["B"] - 1):
            assert np.array_equal(g["paths"][b], inputs.stretch_path(d, 40_000 + b0 + b, 50)[:3])
            assert np.array_equal(g["mu"][b], inputs.batch_mu(d, 1, 40_000 + b0 + b, lo, hi)[0])
        assert np.array_equal(g["coef"], inputs.map_coefficients(d, g["mu"]))
        b0 += g["B"]
    assert n3 >= 0


def test_plan_waves_budget():
    """Admission by footprint: every instance lands in exactly one wave, in group order; each
    wave's states fit the budget; a group that does not fit is split at the budget boundary."""
    import pytest
    rng = np.random.default_rng(4)
    for _ in range(20):
        G = int(rng.integers(1, 7))
        sizes = [int(x) for x in rng.integers(1, 300, G)]
        per = [int(x) for x in rng.integers(10, 500, G)]
        budget = int(rng.integers(max(per), 40 * max(per)))
        waves = serving.plan_waves(sizes, per, budget)
        seen = [np.zeros(B, int) for B in sizes]
        order = []
        for wave in waves:
            assert wave and sum(cnt * per[g] for g, s0, cnt in wave) <= budget
            for g, s0, cnt in wave:
                assert cnt >= 1
                seen[g][s0:s0 + cnt] += 1
                order.append((g, s0))
        assert all((s == 1).all() for s in seen)
        assert order == sorted(order)
    assert serving.plan_waves([10, 5], [100, 200], 10 ** 6) == [[(0, 0, 10), (1, 0, 5)]]
    assert serving.plan_waves([10], [100], 350) == [[(0, 0, 3)], [(0, 3, 3)], [(0, 6, 3)], [(0, 9, 1)]]
    with pytest.raises(ValueError):
        serving.plan_waves([2], [500], 499)
