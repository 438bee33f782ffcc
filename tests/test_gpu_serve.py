"""Serving loop: results alone equal results in the mix (bitwise), admission by
the memory budget, step cap and divergence statuses."""
import numpy as np
import pytest

from paper_1708_07525_gb300 import lbm
from paper_1708_07525_gb300.workloads import draw_batch

pytestmark = pytest.mark.gpu


def requests(n, seed):
    return [lbm.make_instance(s) for s in draw_batch(n, seed=seed, sizes=(32, 48, 64))]


@pytest.mark.parametrize("precision", ["bf16", "f32"])
def test_result_alone_equals_result_in_mix(precision):
    reqs = requests(10, seed=21)
    budget = sum(lbm.batch_instance_bytes(r.params.nx, r.params.ny, precision) for r in reqs) * 2
    mix = lbm.Server(budget, max_slots=16, check_every=50, precision=precision)
    for k, r in enumerate(reqs):
        mix.submit(r, tol=1e-4, max_steps=3000, rid=k)
    got = {r["id"]: r for r in mix.drain()}
    assert sorted(got) == list(range(10))
    for k in (0, 3, 7):
        solo = lbm.Server(budget, max_slots=2, check_every=50, precision=precision)
        solo.submit(reqs[k], tol=1e-4, max_steps=3000, rid=k)
        (res,) = solo.drain()
        assert res["status"] == got[k]["status"]
        assert res["steps"] == got[k]["steps"]
        assert res["nush"] == got[k]["nush"]
        assert res["residual"] == got[k]["residual"]


def test_budget_admission_queues_and_completes():
    reqs = [lbm.make_instance(s) for s in draw_batch(12, seed=22, sizes=(48,))]
    one = lbm.batch_instance_bytes(48, 48, "bf16")
    budget = 2 * one + 4096          # room for exactly two of these cavities
    srv = lbm.Server(budget, max_slots=8, check_every=20, precision="bf16")
    for k, r in enumerate(reqs):
        srv.submit(r, tol=1e-3, max_steps=400, rid=k)
    seen_active = 0
    results = []
    for _ in range(10000):
        a = srv.tick()
        seen_active = max(seen_active, a)
        assert srv.info()["arena_used"] <= budget
        results += srv.poll()
        if a == 0 and srv.info()["queued"] == 0:
            break
    assert seen_active == 2
    assert sorted(r["id"] for r in results) == list(range(12))
    for r in results:
        assert r["status"] in (lbm.OK, lbm.ERR_UNCONVERGED)
        assert r["steps"] <= 400 + 20 and r["t_done"] >= r["t_admit"] >= r["t_submit"]


def test_step_cap_and_divergence_statuses():
    srv = lbm.Server(1 << 26, max_slots=4, check_every=20, precision="f32")
    ok = requests(1, seed=23)[0]
    srv.submit(ok, tol=1e-30, max_steps=60, rid=1)              # cannot converge in 60 steps
    bad = lbm.make_instance(params=lbm.lbm_derive_params(16, 16, 1e4, 1e-2, 0.6, 1.0, 2.0, 1.0),
                            seed=3, noise=0.1)
    bad.params.K = 1e30          # no drag ...
    bad.params.Feps = 0.0
    bad.params.gbT = 5.0         # ... and an absurd buoyancy: the flow blows up
    srv.submit(bad, tol=1e-7, max_steps=100000, rid=2)
    res = {r["id"]: r for r in srv.drain()}
    assert res[1]["status"] == lbm.ERR_UNCONVERGED and res[1]["steps"] == 60
    assert res[2]["status"] == lbm.ERR_DIVERGED


def test_wall_node_requests_alone_equal_in_mix():
    """Requests with the paper's own walls and convective walls (Sec. 3.3, Eq. 39) are
    served beside halfway-wall requests; each result equals the request served alone."""
    mixed = requests(6, seed=31)
    walls = [lbm.make_instance(params=lbm.lbm_derive_params_convective(n, 1e4, 1e-2, 0.6, 1.0,
                                                                         1.0, 1.0, 1.0, bic),
                               seed=7 + n, noise=1e-3)
             for n, bic in ((32, 1.0), (40, 200.0))]
    reqs = mixed[:3] + walls + mixed[3:]
    budget = sum(lbm.batch_instance_bytes(r.params.nx, r.params.ny, "f32") for r in reqs) * 2
    mix = lbm.Server(budget, max_slots=16, check_every=50, precision="f32")
    for k, r in enumerate(reqs):
        mix.submit(r, tol=1e-4, max_steps=3000, rid=k)
    got = {r["id"]: r for r in mix.drain()}
    for k in (3, 4, 0):
        solo = lbm.Server(budget, max_slots=2, check_every=50, precision="f32")
        solo.submit(reqs[k], tol=1e-4, max_steps=3000, rid=k)
        (res,) = solo.drain()
        assert res["status"] == got[k]["status"]
        assert res["steps"] == got[k]["steps"]
        assert res["nush"] == got[k]["nush"]
