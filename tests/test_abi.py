"""CPU-side checks of the C ABI: liblbm.so builds for sm_103a, loads, exports
every entry point include/*.h declares, and rejects invalid input before any
device work (no GPU needed for these)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_1708_07525_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(lbm\w*)\s*\(", src):
            names.add(m.group(1))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_library_builds_and_exports_all_declared_symbols():
    path = build.build()
    L = C.CDLL(path)
    syms = declared_symbols()
    assert "lbm_step" in syms and "lbm_create" in syms and "lbm_nusselt_sherwood" in syms
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_derive_params_matches_paper_mapping():
    """Sec. 4.1: 1/s_nu = 1/2 + Ma J L sqrt(Pr) / (c_s sqrt(Ra)), L = nx; Eq. 29; Eq. 7."""
    p = lbm.lbm_derive_params(64, 64, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0)
    cs = 1 / np.sqrt(3)
    inv_snu = 0.5 + 0.1 * 1 * 64 * 1 / (cs * 100)
    assert abs(p.s[7] - 1 / inv_snu) < 1e-15
    nu = 0.1 * cs * 64 * np.sqrt(1 / 1e4)
    assert abs(p.nu - nu) < 1e-16
    assert abs(p.zeta[1] - 1 / (0.5 + nu / 0.2)) < 1e-14
    assert abs(p.eta[1] - 1 / (0.5 + nu / 2 / 0.2)) < 1e-14
    assert abs(p.Feps - 1.75 / np.sqrt(150 * 0.6 ** 3)) < 1e-15
    assert abs(p.K - 0.01 * 64 * 64) < 1e-12
    assert list(p.s)[:7] == [1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2]
    assert list(p.zeta)[3:] == [1.5, 1.5] and list(p.eta)[3:] == [1.5, 1.5]


@pytest.mark.parametrize("bad", [
    dict(nx=2), dict(eps=0.0), dict(eps=1.5), dict(Da=0.0), dict(Ra=-1.0), dict(Le=0.0),
])
def test_invalid_parameters_rejected(bad):
    kw = dict(nx=16, ny=16, Ra=1e4, Da=1e-2, eps=0.6, Pr=1.0, Le=2.0, N=1.0)
    kw.update(bad)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_derive_params(**kw)
    assert ei.value.status == lbm.ERR_INVALID
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Cavity(**kw, allocator=None)
    assert ei.value.status == lbm.ERR_INVALID


def test_rate_outside_stable_range_rejected():
    # Ra tiny at a large grid -> nu_e huge -> s_nu tiny but valid; Le huge -> eta_D near 2
    p = lbm.lbm_derive_params(16, 16, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0)
    p.s[7] = 2.0
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Cavity(params=p, allocator=None)
    assert ei.value.status == lbm.ERR_INVALID
    assert "relaxation rate" in str(ei.value)


def test_derive_nee_and_convective_match_the_oracle(oracle_mod):
    """The node-on-wall mapping (L = nx - 1) and the Sec. 4.2 convective cavity agree
    with the oracle's independent derivation, field by field."""
    O = oracle_mod
    pairs = [(lbm.lbm_derive_params_nee(21, 13, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0, sigma=0.8),
              O.derive(21, 13, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0, sigma=0.8, nee=True)),
             (lbm.lbm_derive_params_convective(40, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, 200.0),
              O.derive_convective(40, 1e4, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0, 200.0))]
    for g, o in pairs:
        assert (g.nx, g.ny, g.nee) == (o.nx, o.ny, 1)
        for k in ("eps", "sigma", "varpi", "nu", "K", "Feps", "gbT", "gbC", "T0", "C0"):
            assert abs(getattr(g, k) - getattr(o, k)) <= 1e-15 * max(1.0, abs(getattr(o, k))), k
        for k in ("s", "zeta", "eta", "Tw", "Cw", "BiT", "BiC"):
            np.testing.assert_allclose(list(getattr(g, k)), list(getattr(o, k)), rtol=1e-15, atol=0)
    g = pairs[1][0]
    assert (g.nx, g.ny) == (41, 41) and g.BiT[1] == 1.0 and g.BiC[1] == 200.0
    # L = 40 spacings: K = Da L^2
    assert abs(g.K - 1e-2 * 40 * 40) < 1e-12


def test_nee_misuse_rejected():
    p = lbm.lbm_derive_params(16, 16, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0)
    p.BiT[1] = 1.0                        # a convective wall needs wall nodes
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Cavity(params=p, allocator=None)
    assert "nee" in str(ei.value)
    q = lbm.lbm_derive_params_nee(16, 16, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0)
    with pytest.raises(lbm.LbmError) as ei:   # the rebuild reads the two-buffer pull layout
        lbm.Cavity(params=q, layout="aa", allocator=None)
    assert ei.value.status == lbm.ERR_INVALID
    with pytest.raises(lbm.LbmError):
        lbm.lbm_derive_params_nee(4, 16, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0)


def test_block_shape_rejected_beyond_the_kernels_bounds():
    """The step kernels take blocks of at most 256 threads; a larger or ragged launch tile
    is refused at creation (before any device work), also where a zero (default) block_x
    would make the tile too large."""
    p = lbm.lbm_derive_params(256, 16, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0)
    for block in ((512, 1), (128, 4), (48, 1), (0, 4), (256, 2)):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.Cavity(params=p, block=block, allocator=None)
        assert ei.value.status == lbm.ERR_INVALID, block


def test_derive_lid_nee_matches_the_oracle(oracle_mod):
    g = lbm.lbm_derive_params_lid_nee(129, 129, 100.0, 1e2, 0.1, 0.95, 1.0, 1.0, -500.0)
    o = oracle_mod.derive_lid(129, 129, 100.0, 1e2, 0.1, 0.95, 1.0, 1.0, -500.0, nee=True)
    assert g.nee == 1 and o.nee == 1
    for k in ("nu", "K", "gbT", "gbC", "T0", "C0"):
        assert abs(getattr(g, k) - getattr(o, k)) <= 1e-15 * max(1.0, abs(getattr(o, k))), k
    for k in ("s", "zeta", "eta", "Tw", "Cw"):
        np.testing.assert_allclose(list(getattr(g, k)), list(getattr(o, k)), rtol=1e-15, atol=0)
    assert g.uw[3][0] == o.uw[3][0] == 0.1
    # L = 128 spacings: Re = L U0 / nu, K = Da L^2
    assert abs(g.nu - 128 * 0.1 / 100.0) < 1e-15 and abs(g.K - 0.1 * 128 * 128) < 1e-9


def test_slab_misuse_rejected():
    """A slab of a cavity split along y: rows must lie in the cavity, and slabs take halfway
    walls, the two-buffer layout and a uniform medium (checked before any device work)."""
    p = lbm.lbm_derive_params(16, 20, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0)
    for y0, h in ((-1, 5), (15, 6), (3, 0)):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.Cavity(params=p, slab=(y0, h), allocator=None)
        assert ei.value.status == lbm.ERR_INVALID
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Cavity(params=p, slab=(0, 10), layout="aa", allocator=None)
    assert ei.value.status == lbm.ERR_INVALID
    q = lbm.lbm_derive_params_nee(16, 20, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Cavity(params=q, slab=(0, 10), allocator=None)
    assert ei.value.status == lbm.ERR_INVALID
