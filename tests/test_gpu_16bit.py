"""16-bit storage (shifted FP16 / BF16 populations, FP32 arithmetic) against the FP64
oracle, element by element, on the cavities with the workloads' halfway walls.

The bar is stated in units of the storage format's unit roundoff u_s (2^-8 for BF16,
2^-11 for FP16): after 1000 steps the relative L2 error of u_x, u_y, T - T0, C - C0 is
at most 8 u_s, and that of each mean Nu / Sh (Eq. 38) at most 16 u_s.  Stochastic
rounding stores each population with an error below one ulp, zero on average; the
measured errors sit at 1-5 u_s on the fields and up to 8 u_s on Nu / Sh.  A storage
that rounds to nearest instead stagnates (per-step changes below half an ulp are lost)
and misses the Nu / Sh bar on every cavity here: the bar is checked to have that
margin.  Grids with even nx run the two-nodes-per-thread kernels (with the edge set
in a launch of its own); odd nx runs the in-place layout on the one-node kernels.
"""
import os

import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import SMALL_AIDING, CavitySpec

pytestmark = pytest.mark.gpu

UNIT = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}
FIELD_BAR, NUSH_BAR = 8, 16          # in units of UNIT[precision]
KEYS = ("ux", "uy", "T", "C")
SPECS = [
    CavitySpec(33, 17, Ra=1e5, Da=1e-1, eps=0.8, Le=3.0, N=2.0, sigma=1.7, seed=13, noise=0.02),
    CavitySpec(130, 67, Ra=3e4, Da=1e-2, eps=0.5, Le=0.7, N=-2.0, sigma=0.6, seed=14, noise=0.01),
    SMALL_AIDING,
]
STEPS = 1000
_oracle_cache = {}


@pytest.fixture(scope="module", autouse=True)
def _threads(oracle_mod):
    oracle_mod.set_threads(os.cpu_count() or 1)


def oracle_after(O, spec, steps):
    key = (spec, steps)
    if key not in _oracle_cache:
        o = O.Oracle(O.derive(*spec.args()), seed=spec.seed, noise=spec.noise)
        o.step(steps)
        _oracle_cache[key] = (o.fields(), o.nusselt_sherwood())
    return _oracle_cache[key]


def errors(O, spec, precision, layout, steps=STEPS, round_nearest=False):
    fo, no = oracle_after(O, spec, steps)
    g = lbm.Cavity(*spec.args(), precision=precision, layout=layout, seed=spec.seed,
                   noise=spec.noise, round_nearest=round_nearest)
    g.step(steps)
    fg, ng = g.fields(), g.nusselt_sherwood()
    g.close()
    e = {}
    for k in KEYS:
        a, b = fg[k], fo[k]
        if k in ("T", "C"):
            a, b = a - 0.5, b - 0.5
        e[k] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    e["nush"] = float(np.max(np.abs(ng - no) / np.abs(no)))
    return e


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("precision", ["bf16", "f16"])
@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"{s.nx}x{s.ny}")
def test_16bit_storage_within_the_bar(oracle_mod, spec, precision, layout):
    e = errors(oracle_mod, spec, precision, layout)
    u = UNIT[precision]
    for k in KEYS:
        assert e[k] <= FIELD_BAR * u, (k, e)
    assert e["nush"] <= NUSH_BAR * u, e


@pytest.mark.parametrize("precision", ["bf16", "f16"])
@pytest.mark.parametrize("spec", SPECS, ids=lambda s: f"{s.nx}x{s.ny}")
def test_round_to_nearest_storage_misses_the_bar(oracle_mod, spec, precision):
    """The negative control: the same storage rounded to nearest stagnates and misses
    the Nu / Sh bar, so the bar can tell unbiased rounding from a biased one."""
    e = errors(oracle_mod, spec, precision, "ab", round_nearest=True)
    assert e["nush"] > NUSH_BAR * UNIT[precision], e


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("nx,ny", [(8, 5), (10, 7), (9, 6)])
def test_16bit_smallest_grids(oracle_mod, nx, ny, layout):
    """The smallest grids of the two-nodes-per-thread path (nx = 8: two column pairs) and
    an odd nx beside them, over 300 steps."""
    spec = CavitySpec(nx, ny, Ra=1e5, Da=1e-2, eps=0.6, Le=2.0, N=1.0, seed=31, noise=0.05)
    e = errors(oracle_mod, spec, "bf16", layout, steps=300)
    for k in ("T", "C"):
        assert e[k] <= FIELD_BAR * UNIT["bf16"], (k, e)
