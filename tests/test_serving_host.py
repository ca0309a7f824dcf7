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
