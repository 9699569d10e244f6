"""GPU test of the serving loop: requests of mixed lattice, size, parameters
and length, admitted under a memory budget that forces queueing, all finish,
and every result equals the same request run alone (bitwise: the batch
kernels perform the same arithmetic as the single-domain kernels)."""
import numpy as np
import pytest

from paper_2101_06769_gb300 import Domain, serve

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone_runs():
    reqs = serve.request_stream(10, seed=11, sides2=(32, 64), sides3=(16, 24), steps_range=(40, 160), rate=50.0)
    budget = 3 * max(r.state_bytes() for r in reqs)
    live = {"bytes": 0}
    srv = serve.Server(hbm_reserve=0, round_steps=24,
                       free_hbm=lambda: budget - sum(r.state_bytes() for r, _ in srv.running.values()))
    out = srv.run(reqs)
    srv.close()
    assert out["done"] + out["failed"] == len(reqs) and out["unserved"] == 0
    assert out["done"] >= len(reqs) - 2
    assert out["mlups"] > 0 and out["p99_s"] >= out["p50_s"] > 0
    checked = 0
    for r in reqs:
        if r.status != "done" or checked == 4:
            continue
        d = Domain(r.D, r.dims, r.periodic, **r.phys)
        d.init(r.kind, r.args, seed=r.seed)
        d.step(r.steps)
        ob = d.observables().as_dict()
        for k in ("mass", "kinetic_energy", "max_u", "p_in", "p_out", "tip_spike", "tip_bubble", "step"):
            assert ob[k] == r.obs[k], (r.rid, k, ob[k], r.obs[k])
        d.close()
        checked += 1
    assert checked >= 3
