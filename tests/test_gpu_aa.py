"""In-place AA storage (LBMP_FLAG_AA): one population set each for f' and
g, even steps reading and writing each cell's own slots, odd steps pulling
from and pushing to the neighbours' slots, phi from a phase-aware pass.
Checked against the FP64 oracle at the FP32 bar after odd and even step
counts, against the two-set kernel (separately compiled, so to within
rounding), for mass conservation, checkpoints and the halved state."""
import numpy as np
import pytest

import oracle as O
from paper_2101_06769_gb300 import Batch, Domain, LbmpError
from paper_2101_06769_gb300.lbmp import FLAG_AA, FLAG_PHASE_REDUCED, FP16_SHIFTED

from test_gpu_parity import CASES, TOL, rel_err

pytestmark = pytest.mark.gpu

NAMES = ["rt3d", "splash3d", "ragged3d", "wide3d", "thin3d"]


def aa_dom(name, **kw):
    c = CASES[name]
    phys = dict(c["phys"])
    phys["flags"] = int(phys.get("flags", 0)) | FLAG_AA
    d = Domain(c["D"], c["dims"], c["periodic"], **phys, **kw)
    return c, d


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("steps", [100, 37])
def test_aa_parity_with_oracle(name, steps):
    c, d = aa_dom(name)
    o = O.Oracle(c["D"], c["dims"], c["periodic"], **c["phys"])
    o.init(c["case"], c["args"], seed=c["seed"])
    f0, g0, _ = o.get_state()
    d.set_state(f0, g0)
    d.step(steps)
    o.step(steps)
    fg, gg, pg = d.get_state()
    fo, go, po = o.get_state()
    ef, eg, ep = rel_err(fg, fo), rel_err(gg, go), rel_err(pg, po)
    assert ef <= TOL and eg <= TOL and ep <= TOL, (name, steps, ef, eg, ep)
    ob, oo = d.observables(), o.observables()
    assert ob.health == 0 and abs(ob.mass / oo.mass - 1) < 1e-6


@pytest.mark.parametrize("name", ["rt3d", "splash3d", "wide3d"])
def test_aa_equals_two_sets_to_rounding(name):
    c, a = aa_dom(name)
    b = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
    for d in (a, b):
        d.init(c["case"], c["args"], seed=c["seed"])
        d.step(25)
    for x, y in zip(a.get_state(), b.get_state()):
        assert rel_err(x, y) <= 5e-6
    oa, ob = a.observables(), b.observables()
    assert abs(oa.mass / ob.mass - 1) < 1e-7


def test_aa_mass_and_graph_replays():
    """Runs of 16 steps replay captured graphs (on a caller's stream): the
    result equals plain single-step launches bitwise, and mass is kept."""
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    c, a = aa_dom("rt3d", stream=s.cuda_stream)
    _, b = aa_dom("rt3d")
    for d in (a, b):
        d.init(c["case"], c["args"], seed=c["seed"])
    a.step(48)
    for _ in range(48):
        b.step(1)
    assert all(np.array_equal(x, y) for x, y in zip(a.get_state(), b.get_state()))
    ob = a.observables()
    assert ob.health == 0 and abs(ob.mass_drift_rel) < 1e-6


def test_aa_checkpoint_resume_is_bitwise():
    c, a = aa_dom("splash3d")
    a.init(c["case"], c["args"], seed=c["seed"])
    a.step(10)
    nbytes = a.state_bytes()
    host = np.empty(nbytes, dtype=np.uint8)
    a.download(host.ctypes.data, nbytes)
    a.sync()
    a.step(10)
    _, b = aa_dom("splash3d")
    b.init(c["case"], c["args"], seed=c["seed"])
    b.step(10)  # same step parity (phase) as the image
    b.upload(host.ctypes.data, nbytes)
    b.step(10)
    assert all(np.array_equal(x, y) for x, y in zip(a.get_state(), b.get_state()))


def test_aa_halves_the_state():
    torch = pytest.importorskip("torch")
    c = CASES["rt3d"]
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    _, a = aa_dom("rt3d", allocator="torch")
    m1 = torch.cuda.memory_allocated()
    b = Domain(c["D"], c["dims"], c["periodic"], allocator="torch", **c["phys"])
    m2 = torch.cuda.memory_allocated()
    N = a.N
    # AA: one f' and one g set (2 x 108 B/cell) and phi (8 B/cell); two sets: 4 x 108 B/cell
    assert (m1 - m0) < 0.55 * (m2 - m1)
    assert (m1 - m0) >= 216 * N and (m2 - m1) >= 432 * N
    a.close()
    b.close()


def test_aa_limits():
    c = CASES["rt3d"]
    for extra in (dict(storage=FP16_SHIFTED), dict(flags=FLAG_AA | FLAG_PHASE_REDUCED)):
        phys = dict(c["phys"], flags=FLAG_AA)
        phys.update(extra)
        with pytest.raises(LbmpError):
            Domain(c["D"], c["dims"], c["periodic"], **phys)
    with pytest.raises(LbmpError):  # D2Q9
        c2 = CASES["rt2d"]
        Domain(c2["D"], c2["dims"], c2["periodic"], **dict(c2["phys"], flags=FLAG_AA))
    _, d = aa_dom("rt3d")
    with pytest.raises(LbmpError):
        d.set_kernel(1)
    b = Batch()
    with pytest.raises(LbmpError):
        b.add(d, 5)
    b.close()
    d.close()
