"""z-slabs of the CUDA library in one process on one GPU: two or three
slabs of a domain, stepped by the fused kernel with the ghost exchange of
paper_2101_06769_gb300.slab between steps (device copies; no kernel waits on
another), reproduce the undivided domain bitwise, walled or periodic in z;
their summed mass and kinetic energy equal the domain's to rounding."""
import numpy as np
import pytest

from paper_2101_06769_gb300 import Domain, LbmpError
from paper_2101_06769_gb300 import slab as S

from test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,world", [("rt3d", 2), ("rt3d", 3), ("ragged3d", 3), ("splash3d", 2)])
def test_slabs_equal_the_undivided_domain(name, world):
    pytest.importorskip("torch")
    c = CASES[name]
    steps = 24
    ref = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
    ref.init(c["case"], c["args"], seed=c["seed"])
    ref.step(steps)
    f, g, _ = ref.get_state()
    ob = ref.observables()
    slabs = [S.SlabDomain(c["dims"], c["periodic"], r, world, **c["phys"]) for r in range(world)]
    for s in slabs:
        s.init(c["case"], c["args"], seed=c["seed"])
    S.local_step(slabs, steps)
    for s in slabs:
        fs, gs = s.own_state()
        assert np.array_equal(fs, f[:, s.z0:s.z1]) and np.array_equal(gs, g[:, s.z0:s.z1]), (s.rank, s.z0, s.z1)
    obs = [s.backend.observables() for s in slabs]
    assert abs(sum(o.mass for o in obs) / ob.mass - 1.0) < 1e-12
    assert abs(sum(o.kinetic_energy for o in obs) / ob.kinetic_energy - 1.0) < 1e-9
    assert max(o.max_u for o in obs) == pytest.approx(ob.max_u, rel=1e-12)
    assert all(np.isnan(o.tip_spike) for o in obs)
    for s in slabs:
        s.close()


def test_slab_limits():
    c = CASES["rt3d"]
    from paper_2101_06769_gb300.lbmp import FP16_SHIFTED
    with pytest.raises(LbmpError):  # one plane is too few
        S.LibBackend(c["dims"], c["periodic"], 10, 11, **c["phys"])
    with pytest.raises(LbmpError):  # the whole walled axis is not a slab
        S.LibBackend(c["dims"], c["periodic"], 0, c["dims"][2], **c["phys"])
    with pytest.raises(LbmpError):  # FP32 only
        S.LibBackend(c["dims"], c["periodic"], 0, 32, storage=FP16_SHIFTED, **c["phys"])
    b = S.LibBackend(c["dims"], c["periodic"], 0, 32, **c["phys"])
    assert b.layout == (0, 32, 0, 2, 34)  # wall below, two ghost planes above
    from paper_2101_06769_gb300.lbmp import load
    with pytest.raises(LbmpError):  # one step at a time
        from paper_2101_06769_gb300.lbmp import _check
        _check(load().lbmp_step(b.h, 2))
    b.close()
