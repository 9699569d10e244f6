"""lbmp_mass_noalloc: the mass reduction for callers that cannot allocate
device memory (for instance a host framework that owns all device memory and
only lends views into its pool).  Its result must equal the mass that the
allocating path, lbmp_observables, reports for the same state, on two calls
in a row (the second call reuses the fixed device array the first one left
behind).  This file sorts last so that a run stopping at the first failure
has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2101_06769_gb300 import Domain, lbmp

pytestmark = pytest.mark.gpu


def test_mass_noalloc_matches_observables_on_two_calls():
    torch = pytest.importorskip("torch")
    L = lbmp.load()
    d = Domain(3, (64, 48, 40), (1, 1, 0), atwood=0.5, nu_ratio=1.0, Re=512.0, g_accel=5e-5,
               L_ref=64.0, mobility=0.02, width=5.0, sigma=1e-3)
    d.init("rt", [20.0, 3.0, 1e-3, 1.0], seed=17)
    for call in range(2):
        if call == 1:
            d.step(9)  # a different state for the second call
        ob = d.observables()
        nbytes = d.state_bytes()
        host = np.empty(nbytes, dtype=np.uint8)
        d.download(host.ctypes.data, nbytes)
        d.sync()
        g = host[nbytes // 2:].view(np.float32)  # the g population set (any layout)
        g_dev = torch.from_numpy(g.copy()).to("cuda")  # the caller owns this memory
        torch.cuda.synchronize()
        mass = C.c_double(-1.0)
        rc = L.lbmp_mass_noalloc(C.c_void_p(g_dev.data_ptr()), C.c_longlong(g.size), C.byref(mass), None)
        assert rc == 0, L.lbmp_last_error()
        # the same FP32 values summed in FP64 by both paths, in different orders
        assert abs(mass.value / ob.mass - 1.0) < 1e-12, (call, mass.value, ob.mass)
    # sizes beyond the fixed array are rejected before any device work
    rc = L.lbmp_mass_noalloc(C.c_void_p(g_dev.data_ptr()), C.c_longlong((1 << 33) + 1), C.byref(mass), None)
    assert rc == -1 and b"2^33" in L.lbmp_last_error()
    d.close()
