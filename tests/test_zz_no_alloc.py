"""lbm_residual_noalloc, the residual entry point that allocates nothing (for
callers whose device memory is already reserved by a host framework, or that
must not stall on cudaMalloc / cudaFree), checked through the C ABI against
lbm_residual on two calls in a row.  Collected last on purpose."""
import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import CavitySpec

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,layout", [("f32", "ab"), ("f64", "aa"), ("bf16", "ab")])
def test_noalloc_residual_matches_allocating_entry_point(precision, layout):
    import torch
    spec = CavitySpec(130, 67, Ra=3e4, Da=1e-2, eps=0.5, Le=0.7, N=-2.0, sigma=0.6, seed=14,
                      noise=0.01)
    cav = lbm.Cavity(*spec.args(), precision=precision, layout=layout, seed=spec.seed,
                     noise=spec.noise)
    snap = torch.zeros(4 * spec.nx * spec.ny, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    cav.step(500)
    assert cav.residual() == float("inf")
    assert cav.residual_noalloc(snap.data_ptr(), False) == float("inf")
    fl = cav.fields(("ux", "uy", "T", "C"))
    host = snap.view(4, spec.ny, spec.nx).cpu().numpy()
    # the snapshot holds u_x, u_y, T - T0, C - C0 (T0 = C0 = 1/2)
    for q, (k, ref) in enumerate((("ux", 0.0), ("uy", 0.0), ("T", 0.5), ("C", 0.5))):
        np.testing.assert_allclose(host[q], fl[k] - ref, rtol=0, atol=1e-15)
    for _ in range(2):                                      # two calls in a row
        cav.step(101)
        r_ref = cav.residual()
        r_new = cav.residual_noalloc(snap.data_ptr(), True)
        assert np.isfinite(r_ref) and r_ref > 0
        assert abs(r_new - r_ref) <= 1e-12 * r_ref, (r_new, r_ref)
    cav.close()


def test_noalloc_takes_grids_beyond_its_scratch_blocks():
    """More than LBM_NOALLOC_MAX_BLOCKS x 1024 nodes: the first pass still fits the
    fixed scratch (each block loops over tiles and rows) and gives lbm_residual's r."""
    import torch
    n = 2049                                    # 4.2 M nodes
    cav = lbm.Cavity(n, n, 1e5, 1e-3, 0.4, 1.0, 5.0, -1.0, precision="bf16", layout="aa")
    snap = torch.zeros(4 * n * n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    cav.step(20)
    cav.residual()
    cav.residual_noalloc(snap.data_ptr(), False)
    cav.step(10)
    r_ref = cav.residual()
    r_new = cav.residual_noalloc(snap.data_ptr(), True)
    assert np.isfinite(r_ref) and r_ref > 0
    assert abs(r_new - r_ref) <= 1e-12 * r_ref, (r_new, r_ref)
    cav.close()


def test_noalloc_reports_non_finite_fields_and_clears_its_flag():
    """A NaN in the initial T (made on the host) gives ERR_DIVERGED from the shared scratch's
    flag slot; the next call, on a healthy cavity, clears the slots and returns a finite r
    equal to lbm_residual's."""
    import torch
    n = 16
    T = np.full((n, n), 0.5)
    T[8, 8] = np.nan
    bad = lbm.Cavity(n, n, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0, precision="f32", T_init=T,
                     C_init=np.full((n, n), 0.5))
    snap_bad = torch.zeros(4 * n * n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    bad.step(50)
    with pytest.raises(lbm.LbmError) as ei:
        bad.residual_noalloc(snap_bad.data_ptr(), False)
    assert ei.value.status == lbm.ERR_DIVERGED
    bad.close()
    good = lbm.Cavity(n, n, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0, precision="f32", seed=3, noise=0.02)
    snap = torch.zeros(4 * n * n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    good.step(40)
    good.residual()
    good.residual_noalloc(snap.data_ptr(), False)
    good.step(30)
    r_ref = good.residual()
    r_new = good.residual_noalloc(snap.data_ptr(), True)
    assert np.isfinite(r_new) and r_new > 0
    assert abs(r_new - r_ref) <= 1e-12 * r_ref, (r_new, r_ref)
    good.close()
