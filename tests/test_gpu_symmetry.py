"""The symmetry x axis of the 2-D splash (Sec. 3.4; reading A28: half-way
specular reflection, the phi ghost equal to the boundary cell) on the GPU.

A periodic domain of width 2L whose drop is centred on a cell face stays
mirror-symmetric, so its right half evolves like a half domain of width L
with symmetry faces at both ends.  In FP32 the mirrored cells of the full
domain sum in another order, so the two agree to rounding, far below what a
wrong reflection would leave (the order of the populations themselves).  The
parity of the symmetric domains with the FP64 oracle is checked with the
other parity cases (`sym2d`, `sym2d_red` in test_gpu_parity.py)."""
import numpy as np
import pytest

from paper_2101_06769_gb300 import Domain
from test_gpu_parity import rel_err

pytestmark = pytest.mark.gpu

L, NY = 150, 60
PHYS = dict(rho_ratio=100.0, nu_ratio=5.0, We=200.0, Re=200.0, U0=0.05, L_ref=20.0, mobility=0.05, width=4.0)


@pytest.mark.parametrize("flags", [0, 8])
@pytest.mark.parametrize("kernel", [0, 1])
def test_half_domain_equals_half_of_the_symmetric_full_domain(flags, kernel):
    phys = dict(PHYS, flags=flags)
    full = Domain(2, (2 * L, NY, 1), (1, 0, 1), **phys)
    half = Domain(2, (L, NY, 1), (2, 0, 1), **phys)
    try:
        full.init("drop_sheet", [20.0, 6.0, 0.05, 0.0, L - 0.5], seed=1)
        half.init("drop_sheet", [20.0, 6.0, 0.05, 0.0, -0.5], seed=1)
        half.set_kernel(kernel)
        full.step(300)
        half.step(300)
        sf, sh = full.get_state(), half.get_state()
        for a_full, a_half in zip(sf, sh):
            assert rel_err(a_half, a_full[..., L:]) <= 1e-5
        ob = half.observables()
        assert ob.health == 0 and abs(ob.mass_drift_rel) < 1e-6
    finally:
        full.close()
        half.close()
