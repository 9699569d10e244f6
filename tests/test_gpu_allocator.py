"""Caller-supplied device memory (lbmp_create_ex): with torch's caching
allocator the handle's arrays are torch's (counted by
torch.cuda.memory_allocated and given back at lbmp_destroy), the results
equal those of a domain on cudaMalloc bitwise, and an allocator that runs
dry fails the call with NOMEM after giving back what it had handed out."""
import numpy as np
import pytest

from paper_2101_06769_gb300 import Domain, LbmpError
from paper_2101_06769_gb300.lbmp import make_allocator

from test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


def dom(name, **kw):
    c = CASES[name]
    d = Domain(c["D"], c["dims"], c["periodic"], **c["phys"], **kw)
    d.init(c["case"], c["args"], seed=c["seed"])
    return d


@pytest.mark.parametrize("name", ["splash3d", "rt2d"])
def test_torch_allocator_results_and_accounting(name):
    torch = pytest.importorskip("torch")
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    a = dom(name, allocator="torch")
    held = torch.cuda.memory_allocated() - before
    assert held >= 2 * a.state_bytes()  # both population sets of f' and g come from torch
    b = dom(name)
    for d in (a, b):
        d.step(21)
    assert all(np.array_equal(x, y) for x, y in zip(a.get_state(), b.get_state()))
    oa, ob = a.observables(), b.observables()
    assert oa.mass == ob.mass and oa.kinetic_energy == ob.kinetic_energy
    a.close()
    b.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before


def test_reference_pair_phi_comes_from_the_allocator():
    torch = pytest.importorskip("torch")
    torch.cuda.synchronize()
    a = dom("thin3d", allocator="torch")
    held = torch.cuda.memory_allocated()
    a.set_kernel(1)  # the reference pair keeps phi (8 bytes per cell) in an array of its own
    assert torch.cuda.memory_allocated() - held >= 8 * a.N
    b = dom("thin3d")
    b.set_kernel(1)
    a.step(7)
    b.step(7)
    assert all(np.array_equal(x, y) for x, y in zip(a.get_state(), b.get_state()))
    a.close()
    b.close()


def test_allocator_running_dry_gives_everything_back():
    torch = pytest.importorskip("torch")
    live = {}
    calls = {"alloc": 0}

    def alloc(n, stream):
        calls["alloc"] += 1
        if calls["alloc"] > 3:
            return 0  # the fourth request fails
        p = torch.cuda.caching_allocator_alloc(n, torch.cuda.current_device(), stream)
        live[p] = n
        return p

    def free(p, n, stream):
        assert live.pop(p) == n
        torch.cuda.caching_allocator_delete(p)

    al = make_allocator(alloc, free)
    c = CASES["rt3d"]
    with pytest.raises(LbmpError) as ei:
        Domain(c["D"], c["dims"], c["periodic"], allocator=al, **c["phys"])
    assert ei.value.code == -2  # NOMEM
    assert calls["alloc"] == 4 and live == {}
