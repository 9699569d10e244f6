"""Failure detection of the step kernels without a GPU fault: a staging
barrier armed for more bytes than its copies deliver (test option) makes the
bounded waits of the bulk-copy kernel run out; the kernel records the time-out
in the handle's status word and returns, the host reports LBMP_ERR_TIMEOUT,
and the context stays usable."""
import numpy as np
import pytest

from paper_2101_06769_gb300 import Domain, LbmpError
from paper_2101_06769_gb300.lbmp import OPT_TEST_STALL, OPT_WAIT_LIMIT_NS

from test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


def make(name="splash3d"):
    c = CASES[name]
    d = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
    d.init(c["case"], c["args"], seed=c["seed"])
    return c, d


def test_wait_timeout_is_reported_and_recoverable():
    c, d = make()
    assert c["dims"][0] % 4 == 0
    d.set_kernel(2)  # the bulk-copy staging kernel, whose waits are on mbarriers
    d.set_option(OPT_WAIT_LIMIT_NS, 2_000_000)  # 2 ms
    d.set_option(OPT_TEST_STALL, 1)
    d.step(1)
    with pytest.raises(LbmpError) as ei:
        d.sync()
    assert ei.value.code == -4
    with pytest.raises(LbmpError) as ei:
        d.observables()
    assert ei.value.code == -4
    # recovery: clear the stall, re-initialise, and the domain steps exactly
    # like a fresh one
    d.set_option(OPT_TEST_STALL, 0)
    d.init(c["case"], c["args"], seed=c["seed"])
    d.step(5)
    d.sync()
    _, ref = make()
    ref.set_kernel(2)
    ref.step(5)
    assert all(np.array_equal(x, y) for x, y in zip(d.get_state(), ref.get_state()))
    assert d.observables().health == 0


def test_bad_wait_limit_rejected():
    _, d = make("thin3d")
    for v in (0, 999, 60_000_000_001):
        with pytest.raises(LbmpError):
            d.set_option(OPT_WAIT_LIMIT_NS, v)
    with pytest.raises(LbmpError):
        d.set_option(OPT_TEST_STALL, 2)
