"""GPU parity of the LBMP_FLAG_DIVU variant (the w cs2 rho div(u) term of Xi
kept, div(u) the isotropic difference of the previous step's stored
velocity) against the FP64 oracle with the same flag.

The term cancels the pressure's response to the divergence, so several
cases amplify perturbations with it: in the FP64 oracle itself a relative
perturbation of 1e-7 in g grows to a phi difference of 1.4e-5 (rt2d) and
2e-5 (rt3d) within 100 steps, and splash3d turns non-finite.  The FP32 bar
(1e-5) is therefore checked after 100 steps on the cases that stay
well-conditioned (drop2d: x0.3, thin3d: x0.07) and after 10 steps on the
others.
"""
import numpy as np
import pytest

import oracle as O
from paper_2101_06769_gb300 import Batch, Domain, LbmpError
from paper_2101_06769_gb300.lbmp import FLAG_DIVU, FLAG_PHASE_REDUCED, FP16_SHIFTED

from test_gpu_parity import CASES, TOL, rel_err

pytestmark = pytest.mark.gpu

STEPS = {"drop2d": 100, "thin3d": 100, "rt2d": 10, "rt3d": 10, "ragged3d": 10, "ragged2d": 10, "wide3d": 10}


def with_divu(name):
    c = dict(CASES[name])
    phys = dict(c["phys"])
    phys["flags"] = int(phys.get("flags", 0)) | FLAG_DIVU
    c["phys"] = phys
    return c


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("name", sorted(STEPS))
def test_step_parity_divu(name, kernel):
    c = with_divu(name)
    o = O.Oracle(c["D"], c["dims"], c["periodic"], **c["phys"])
    d = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
    o.init(c["case"], c["args"], seed=c["seed"])
    f0, g0, _ = o.get_state()
    o.set_state(f0, g0)
    d.set_state(f0, g0)
    d.set_kernel(kernel)
    o.step(STEPS[name])
    d.step(STEPS[name])
    fo, go, po = o.get_state()
    fg, gg, pg = d.get_state()
    ef, eg, ep = rel_err(fg, fo), rel_err(gg, go), rel_err(pg, po)
    assert ef <= TOL and eg <= TOL and ep <= TOL, (name, kernel, ef, eg, ep)


def test_divu_observables_match_oracle():
    """p_h of the observables includes the term's cs2 rho div(u)/2."""
    c = with_divu("drop2d")
    o = O.Oracle(c["D"], c["dims"], c["periodic"], **c["phys"])
    d = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
    o.init(c["case"], c["args"], seed=c["seed"])
    d.init(c["case"], c["args"], seed=c["seed"])
    o.step(100)
    d.step(100)
    ob, og = o.observables(), d.observables()
    scale = max(abs(ob.p_in), abs(ob.p_out))
    assert abs(og.p_in - ob.p_in) < 1e-4 * scale and abs(og.p_out - ob.p_out) < 1e-4 * scale
    assert abs(og.max_u / ob.max_u - 1) < 1e-3


def test_divu_changes_the_step():
    c = CASES["drop2d"]
    states = []
    for flags in (0, FLAG_DIVU):
        phys = dict(c["phys"])
        phys["flags"] = flags
        d = Domain(c["D"], c["dims"], c["periodic"], **phys)
        d.init(c["case"], c["args"], seed=c["seed"])
        d.step(20)
        states.append(d.get_state()[0])
    assert rel_err(states[1], states[0]) > 1e-4


def test_checkpoint_resume_is_bitwise_divu():
    c = with_divu("ragged3d")
    a = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
    a.init(c["case"], c["args"], seed=c["seed"])
    a.step(7)
    nb = a.state_bytes()
    assert nb == 4 * int(np.prod(c["dims"])) * (2 * a.Q + c["D"])
    buf = np.empty(nb, np.uint8)
    a.download(buf.ctypes.data, nb)
    a.sync()
    a.step(5)
    want = a.get_state()
    b = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
    b.upload(buf.ctypes.data, nb)
    b.sync()
    b.step(5)
    assert all(np.array_equal(x, y) for x, y in zip(b.get_state(), want))


def test_divu_rejections():
    c = with_divu("thin3d")
    with pytest.raises(LbmpError):
        Domain(c["D"], c["dims"], c["periodic"], storage=FP16_SHIFTED, **c["phys"])
    phys = dict(c["phys"])
    phys["flags"] |= FLAG_PHASE_REDUCED
    with pytest.raises(LbmpError):
        Domain(c["D"], c["dims"], c["periodic"], **phys)
    d = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
    d.init(c["case"], c["args"], seed=c["seed"])
    b = Batch()
    with pytest.raises(LbmpError):
        b.add(d, 10)
    b.close()
