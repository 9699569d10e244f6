"""Degenerate cases of the method on the GPU: single-phase rest states and
uniform flows (nothing may move), and the smallest grids the ABI accepts
(every cell a wall or periodic neighbour of itself), against the FP64
oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2101_06769_gb300 import Domain
from paper_2101_06769_gb300.lbmp import FP16_SHIFTED, FP32

from test_gpu_parity import TOL, rel_err

pytestmark = pytest.mark.gpu

PHYS = dict(rho_ratio=20.0, nu_ratio=2.0, nu_h=0.05, mobility=0.02, width=4.0, sigma=1e-3, g_accel=1e-5)


@pytest.mark.parametrize("storage", [FP32, FP16_SHIFTED])
@pytest.mark.parametrize("phi0", [0.0, 1.0])
@pytest.mark.parametrize("D", [2, 3])
def test_single_phase_rest_state_stays(D, phi0, storage):
    """A single phase at rest with a uniform pressure and no gravity (a
    uniform pressure does not balance a body force): no gradient of phi, no
    force, so the state is a fixed point up to the FP32 rounding of the
    collision."""
    dims = (16, 12, 10) if D == 3 else (16, 12, 1)
    per = (1, 1, 0) if D == 3 else (1, 0, 1)
    phys = dict(PHYS, g_accel=0.0)
    d = Domain(D, dims, per, storage=storage, **phys)
    d.init("uniform", [phi0, 1e-3, 0.0, 0.0, 0.0])
    f0, g0, p0 = d.get_state()
    d.step(100)
    f1, g1, p1 = d.get_state()
    ob = d.observables()
    assert ob.health == 0 and ob.max_u < 1e-9
    assert rel_err(f1, f0) < 1e-6 and rel_err(g1, g0) < 1e-6
    assert np.abs(p1 - phi0).max() < 1e-6


@pytest.mark.parametrize("D", [2, 3])
def test_uniform_flow_stays_uniform(D):
    """phi = 1 moving at a uniform velocity on a periodic grid: the state
    stays uniform and every cell keeps u0.  (f' itself relaxes from the
    second-order equilibrium it starts in to the cumulant model's product
    equilibrium, an O(u^2) relative change, as in the oracle.)"""
    dims = (16, 12, 10) if D == 3 else (16, 12, 1)
    u0 = [0.03, -0.02, 0.01 if D == 3 else 0.0]
    d = Domain(D, dims, (1, 1, 1), **dict(PHYS, g_accel=0.0))
    d.init("uniform", [1.0, 0.0] + u0)
    o = O.Oracle(D, dims, (1, 1, 1), **dict(PHYS, g_accel=0.0))
    o.init("uniform", [1.0, 0.0] + u0)
    d.step(100)
    o.step(100)
    f1, g1, p1 = d.get_state()
    fo, go, po = o.get_state()
    Q = f1.shape[0]
    spread = (f1.reshape(Q, -1).max(1) - f1.reshape(Q, -1).min(1)).max()
    assert spread <= 1e-7 * np.abs(f1).max()
    assert rel_err(f1, fo) <= TOL and rel_err(g1, go) <= TOL
    assert abs(d.observables().max_u - np.linalg.norm(u0)) < 1e-6


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("D,dims,per", [(3, (2, 2, 2), (1, 1, 0)), (3, (2, 2, 3), (1, 1, 1)), (2, (2, 2, 1), (1, 0, 1))])
def test_smallest_grids_match_oracle(D, dims, per, kernel):
    """The smallest grids the ABI accepts: every neighbour of a cell is
    itself or its one periodic partner, or a wall; the step and the phi
    ghosts still follow the oracle."""
    phys = dict(PHYS)
    o = O.Oracle(D, dims, per, **phys)
    d = Domain(D, dims, per, **phys)
    o.init("uniform", [0.6, 1e-3, 0.01, -0.005, 0.0])
    f0, g0, _ = o.get_state()
    o.set_state(f0, g0)
    d.set_state(f0, g0)
    d.set_kernel(kernel)
    o.step(50)
    d.step(50)
    fo, go, po = o.get_state()
    fg, gg, pg = d.get_state()
    assert rel_err(fg, fo) <= TOL and rel_err(gg, go) <= TOL and rel_err(pg, po) <= TOL
    assert abs(d.observables().mass_drift_rel) < 1e-6
