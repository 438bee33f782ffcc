"""Table 1 of the paper (Sec. 4.1, non-porous double-diffusive cavity, A = 2,
100 x 200): the oracle's steady mean Nu, Sh and peak velocities against the
printed values, and the GPU FP64 path against the oracle.

The paper's own walls are node-based non-equilibrium extrapolation; the
halfway walls used here give a slightly different discretisation, so the
oracle is held to 2 % of the paper (the paper's own values differ from the
FDM reference it quotes by 0.9 %).  The stored oracle values are written by
tests/golden/make_table1.py, which calls only oracle/."""
import json
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_oracle_matches_table1():
    paper, ora = load("table1_paper.json"), load("table1_oracle.json")
    for key, ref in (("nu_left", paper["nu"]), ("sh_left", paper["sh"]),
                     ("ux_max_alpha_over_L", paper["ux_max"]),
                     ("uy_max_alpha_over_L", paper["uy_max"])):
        assert abs(ora[key] - ref) <= 0.02 * ref, (key, ora[key], ref)
    # left and right walls carry the same flux at steady state
    assert abs(ora["nu_left"] - ora["nu_right"]) <= 1e-4 * ora["nu_left"]
    assert abs(ora["sh_left"] - ora["sh_right"]) <= 1e-4 * ora["sh_left"]


@pytest.mark.gpu
def test_gpu_fp64_matches_oracle_table1_case():
    from paper_1708_07525_gb300 import lbm
    ora = load("table1_oracle.json")
    c = lbm.Cavity(100, 200, 1e5, 1e8, 1.0, 1.0, 2.0, -0.8, precision="f64", seed=7, noise=1e-3)
    c.step(ora["steps"])
    ns = c.nusselt_sherwood()
    ref = np.array([ora["nu_left"], ora["sh_left"], ora["nu_right"], ora["sh_right"]])
    np.testing.assert_allclose(ns, ref, rtol=1e-9)
    fl = c.fields(("ux", "uy"))
    p = c.params
    alpha = p.nu / 1.0
    assert abs(np.abs(fl["ux"]).max() * 100 / alpha - ora["ux_max_alpha_over_L"]) < 1e-7
    assert abs(np.abs(fl["uy"]).max() * 100 / alpha - ora["uy_max_alpha_over_L"]) < 1e-7


def test_oracle_with_the_papers_walls_matches_table1():
    """The same cavity with the paper's own walls (Sec. 3.3: 101 x 201 nodes on the
    walls, L = 100): steady Nu, Sh and peak velocities within 0.5 % of Table 1 (the
    stored run gives 0.01 %, 0.07 %, 0.34 % and 0.02 %); the two walls carry the same
    flux to the extrapolation's accuracy."""
    paper, ora = load("table1_paper.json"), load("table1_nee_oracle.json")
    for key, ref in (("nu_left", paper["nu"]), ("sh_left", paper["sh"]),
                     ("ux_max_alpha_over_L", paper["ux_max"]),
                     ("uy_max_alpha_over_L", paper["uy_max"])):
        assert abs(ora[key] - ref) <= 0.005 * ref, (key, ora[key], ref)
    assert abs(ora["nu_left"] - ora["nu_right"]) <= 0.01 * ora["nu_left"]
    assert abs(ora["sh_left"] - ora["sh_right"]) <= 0.01 * ora["sh_left"]


@pytest.mark.gpu
def test_gpu_fp64_matches_oracle_table1_with_the_papers_walls():
    from paper_1708_07525_gb300 import lbm
    ora = load("table1_nee_oracle.json")
    p = lbm.lbm_derive_params_nee(101, 201, 1e5, 1e8, 1.0, 1.0, 2.0, -0.8)
    c = lbm.Cavity(params=p, precision="f64", seed=7, noise=1e-3)
    c.step(ora["steps"])
    ns = c.nusselt_sherwood()
    ref = np.array([ora["nu_left"], ora["sh_left"], ora["nu_right"], ora["sh_right"]])
    np.testing.assert_allclose(ns, ref, rtol=1e-9)
    fl = c.fields(("ux", "uy"))
    alpha = p.nu / 1.0
    assert abs(np.abs(fl["ux"]).max() * 100 / alpha - ora["ux_max_alpha_over_L"]) < 1e-7
    assert abs(np.abs(fl["uy"]).max() * 100 / alpha - ora["uy_max_alpha_over_L"]) < 1e-7
    c.close()
