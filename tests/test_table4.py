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


def test_oracle_with_the_papers_walls_table4():
    """The same cavity with the paper's own walls (Sec. 3.3, 129 x 129 wall nodes): Nu = Sh
    on the bottom wall within 5 % of Table 4 (they come out 0.75-4.1 % low, the largest
    gaps at N > 0, where the flow is nearly stagnant and conduction dominates; the
    extrapolated walls pass 1-3 % more heat through the top wall than through the
    bottom one at steady state, so the wall-flux discretisation sets the gap)."""
    path = os.path.join(HERE, "table4_nee_oracle.json")
    gold = json.load(open(path))
    paper = json.load(open(os.path.join(HERE, "table4_paper.json")))
    assert len(gold["rows"]) >= 3
    for row in gold["rows"]:
        ref = paper["nu"][paper["N"].index(int(row["N"]))]
        assert abs(row["nu_bottom"] - ref) <= 0.05 * ref, row
        assert abs(row["nu_bottom"] - row["sh_bottom"]) <= 1e-6 * ref   # Le = 1


def test_table5_present_model_and_model_a():
    """Table 5 (eps = 0.6): the paper's model gives Nu = Sh on the bottom wall, model A
    (Eqs. 30-32) does not; both within 2 % of the printed values, and model A's split
    has the printed sign (Sh > Nu)."""
    gold = json.load(open(os.path.join(HERE, "table5_oracle.json")))
    paper = json.load(open(os.path.join(HERE, "table5_paper.json")))
    for prow in paper["rows"]:
        rows = {r["model_a"]: r for r in gold["rows"] if int(r["N"]) == prow["N"]}
        pres, ma = rows[False], rows[True]
        assert abs(pres["nu_bottom"] - pres["sh_bottom"]) <= 1e-6 * pres["nu_bottom"]
        assert abs(pres["nu_bottom"] - prow["present_nu"]) <= 0.02 * prow["present_nu"]
        assert abs(ma["nu_bottom"] - prow["model_a_nu"]) <= 0.02 * prow["model_a_nu"]
        assert abs(ma["sh_bottom"] - prow["model_a_sh"]) <= 0.02 * prow["model_a_sh"]
        assert ma["sh_bottom"] - ma["nu_bottom"] > 1e-5
