"""Table 4 of the paper (Sec. 4.3, lid-driven porous cavity): the oracle's steady
mean Nu = Sh on the bottom wall against the printed values for several buoyancy
ratios N.  The paper's walls are node-based (non-equilibrium extrapolation); the
halfway walls here are held to 2 %.  Stored by tests/golden/make_table4.py, which
calls only oracle/."""
import json
import os

import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_matches_table4():
    path = os.path.join(HERE, "table4_oracle.json")
    if not os.path.exists(path):
        pytest.skip("table4_oracle.json not generated")
    gold = json.load(open(path))
    paper = json.load(open(os.path.join(HERE, "table4_paper.json")))
    assert len(gold["rows"]) >= 3
    for row in gold["rows"]:
        ref = paper["nu"][paper["N"].index(int(row["N"]))]
        assert abs(row["nu_bottom"] - ref) <= 0.02 * ref, row
        assert abs(row["sh_bottom"] - ref) <= 0.02 * ref, row
        assert abs(row["nu_bottom"] - row["sh_bottom"]) <= 1e-6 * ref   # Le = 1
