"""GPU tests of the batch form: members of uneven sizes advanced together by
one persistent kernel per step (CUDA-graph replays) give bitwise the states
of stepping each alone, respect their own step counts, and the HBM budget."""
import numpy as np
import pytest

import oracle as O
from paper_2101_06769_gb300 import Batch, Domain, LbmpError

pytestmark = pytest.mark.gpu

MEMBERS = [
    dict(dims=(32, 32, 64), periodic=(1, 1, 0),
         phys=dict(atwood=0.5, nu_ratio=1.0, Re=1024.0, g_accel=5e-5, L_ref=32.0, mobility=0.02, width=5.0),
         case="rt", args=[32.0, 3.2, 1e-4, 1.0], seed=2),
    dict(dims=(37, 29, 23), periodic=(1, 1, 1),
         phys=dict(rho_ratio=20.0, nu_ratio=2.0, nu_h=0.05, sigma=1e-2, mobility=0.02, width=4.0),
         case="drop_static", args=[7.0, 1.0, 1e-2], seed=5),
    dict(dims=(64, 64, 32), periodic=(1, 1, 0),
         phys=dict(rho_ratio=1000.0, nu_ratio=15.0, We=8000.0, Re=1000.0, U0=0.05, L_ref=16.0,
                   mobility=0.02, width=4.0),
         case="drop_sheet", args=[16.0, 3.2, 0.05, 1e-4], seed=3),
    dict(dims=(8, 6, 5), periodic=(1, 1, 0),
         phys=dict(rho_ratio=3.0, nu_ratio=1.0, nu_h=0.05, sigma=1e-2, g_accel=1e-4, mobility=0.02, width=3.0),
         case="rt", args=[2.0, 0.5, 1e-2, 1.0], seed=7),
]


def make(m):
    d = Domain(3, m["dims"], m["periodic"], **m["phys"])
    d.init(m["case"], m["args"], seed=m["seed"])
    return d


def test_batch_is_bitwise_stepping_alone():
    steps = [37, 12, 50, 21]  # uneven step counts, not multiples of the graph length
    alone = []
    for m, n in zip(MEMBERS, steps):
        d = make(m)
        d.step(n)
        alone.append(d.get_state())
    b = Batch()
    doms = [make(m) for m in MEMBERS]
    for d, n in zip(doms, steps):
        b.add(d, n)
    finished = 0
    for _ in range(3):
        finished += b.step(25)
    assert finished == len(MEMBERS)
    assert all(left == 0 for _, left in b.members())
    for d, ref, n in zip(doms, alone, steps):
        got = d.get_state()
        for a, r in zip(got, ref):
            assert np.array_equal(a, r)
        assert d.observables().step == n


def test_batch_member_leaves_and_continues_alone():
    m = MEMBERS[0]
    ref = make(m)
    ref.step(30)
    d = make(m)
    b = Batch()
    b.add(d, 17)
    b.step(100)
    b.remove(d)
    d.step(13)  # continue through its own handle
    for a, r in zip(d.get_state(), ref.get_state()):
        assert np.array_equal(a, r)


def test_batch_matches_oracle():
    m = MEMBERS[1]
    o = O.Oracle(3, m["dims"], m["periodic"], **m["phys"])
    o.init(m["case"], m["args"], seed=m["seed"])
    o.step(40)
    d = make(m)
    b = Batch()
    b.add(d, 40)
    b.step(40)
    fo, go, po = o.get_state()
    fg, gg, pg = d.get_state()
    for x, y in ((fg, fo), (gg, go), (pg, po)):
        assert np.abs(x - y).max() / np.abs(y).max() <= 1e-5


def test_batch_budget_and_errors():
    doms = [make(MEMBERS[0]), make(MEMBERS[2])]
    one = doms[0].state_bytes() * 2  # two population sets per family
    b = Batch(hbm_budget=one + 1)
    b.add(doms[0], 5)
    assert b.try_add(doms[1], 5) is False  # does not fit
    with pytest.raises(LbmpError):
        b.add(doms[0], 5)  # already a member
    with pytest.raises(LbmpError):
        b.add(doms[1], 0)


MEMBERS_2D = [
    dict(dims=(64, 256, 1), periodic=(1, 0, 1),
         phys=dict(atwood=0.5, nu_ratio=1.0, Re=256.0, g_accel=2.5e-5, L_ref=64.0, mobility=0.02, width=5.0),
         case="rt", args=[128.0, 6.4, 1e-4, 1.0], seed=1),
    dict(dims=(48, 48, 1), periodic=(1, 1, 1),
         phys=dict(rho_ratio=1000.0, nu_ratio=1.0, nu_h=0.1, sigma=1e-3, mobility=0.02, width=5.0),
         case="drop_static", args=[12.0, 0.0, 1e-3], seed=4),
    dict(dims=(200, 33, 1), periodic=(1, 0, 1),
         phys=dict(rho_ratio=10.0, nu_ratio=5.0, nu_h=0.02, sigma=5e-3, g_accel=1e-5, mobility=0.03, width=4.0,
                   flags=2),
         case="rt", args=[16.0, 3.0, 1e-2, 1.0], seed=6),
]


def make2(m):
    d = Domain(2, m["dims"], m["periodic"], **m["phys"])
    d.init(m["case"], m["args"], seed=m["seed"])
    return d


def test_mixed_2d_3d_batch_is_bitwise_stepping_alone():
    specs = [(3, MEMBERS[0], 19), (2, MEMBERS_2D[0], 33), (2, MEMBERS_2D[1], 8), (3, MEMBERS[3], 27),
             (2, MEMBERS_2D[2], 40)]
    alone, doms = [], []
    b = Batch()
    for D, m, n in specs:
        a = make(m) if D == 3 else make2(m)
        a.step(n)
        alone.append(a.get_state())
        d = make(m) if D == 3 else make2(m)
        b.add(d, n)
        doms.append(d)
    b.step(16)
    b.step(100)
    for d, ref in zip(doms, alone):
        for x, r in zip(d.get_state(), ref):
            assert np.array_equal(x, r)


@pytest.mark.parametrize("kernel", [0, 1])
def test_fused_2d_matches_oracle(kernel):
    for m in MEMBERS_2D:
        o = O.Oracle(2, m["dims"], m["periodic"], **m["phys"])
        o.init(m["case"], m["args"], seed=m["seed"])
        f0, g0, _ = o.get_state()
        d = Domain(2, m["dims"], m["periodic"], **m["phys"])
        d.set_state(f0, g0)
        d.set_kernel(kernel)
        o.step(100)
        d.step(100)
        fo, go, po = o.get_state()
        fg, gg, pg = d.get_state()
        for x, y in ((fg, fo), (gg, go), (pg, po)):
            assert np.abs(x - y).max() / np.abs(y).max() <= 1e-5


def test_batch_autotune_keeps_results():
    """The batch autotuner's trials advance no member, and after tuning the
    batch steps each member like stepping it alone with the chosen tile shape
    (the tile builds agree to within rounding; same bar as the tile tests)."""
    from paper_2101_06769_gb300.lbmp import OPT_TILE
    b = Batch()
    doms = [make(m) for m in MEMBERS]
    for d in doms:
        b.add(d, 12)
    before = [d.get_state() for d in doms]
    best, trials = b.autotune(reps=1)
    assert best is not None and len(trials) == 12
    for d, st in zip(doms, before):
        assert all(np.array_equal(x, y) for x, y in zip(d.get_state(), st))
    b.step(12)
    for m, d in zip(MEMBERS, doms):
        r = make(m)
        r.set_option(OPT_TILE, best[2])
        r.step(12)
        for x, y in zip(d.get_state(), r.get_state()):
            scale = np.abs(y).max()
            assert np.abs(x - y).max() <= 5e-6 * (scale if scale > 0 else 1.0)
    b.close()


def test_batch_autotune_keeps_reduced_members():
    """Members on the reduced phase lattice keep their stored previous phi u
    across the batch autotuner's trials: after tuning, a few steps of the
    batch equal the same steps of untuned twins stepped alone (same tile
    build, so bitwise)."""
    from paper_2101_06769_gb300.lbmp import FLAG_PHASE_REDUCED
    red = []
    for m in MEMBERS[:3]:
        r = dict(m)
        r["phys"] = dict(m["phys"], flags=FLAG_PHASE_REDUCED)
        red.append(r)
    b = Batch()
    doms = [make(m) for m in red]
    twins = [make(m) for m in red]
    for d in doms:
        b.add(d, 7)
    b.step(3)  # a stored phi u from real steps
    for t in twins:
        t.step(3)
    b.autotune(reps=1)
    b.step(4)
    for t in twins:
        t.step(4)
    for d, t in zip(doms, twins):
        assert all(np.array_equal(x, y) for x, y in zip(d.get_state(), t.get_state()))
    b.close()


def test_batch_phases_are_bitwise_stepping_alone():
    """An odd number of single steps leaves the batch in its other phase; the
    graphs of that phase (16-step and single-step) must then step every
    member on the population sets of its current parity.  Runs of 3, 20, 1,
    33 and 5 steps use both phases of both graphs; FP32 members on both
    phase lattices (the member-grid kernels) equal twins stepped alone
    bitwise after every run."""
    from paper_2101_06769_gb300.lbmp import FLAG_PHASE_REDUCED
    ms = list(MEMBERS)
    for m in MEMBERS[:2]:
        r = dict(m)
        r["phys"] = dict(m["phys"], flags=FLAG_PHASE_REDUCED)
        ms.append(r)
    b = Batch()
    doms = [make(m) for m in ms]
    twins = [make(m) for m in ms]
    for d in doms:
        b.add(d, 1000)
    for n in (3, 20, 1, 33, 5):
        b.step(n)
        for t in twins:
            t.step(n)
        for d, t in zip(doms, twins):
            assert all(np.array_equal(x, y) for x, y in zip(d.get_state(), t.get_state())), n
    b.close()


def test_batch_of_more_members_than_one_launch_holds():
    """35 FP32 D3Q27 members (more than the kernel parameters of one launch
    hold, so each step takes two launches of the batch kernel) with uneven
    sizes and step counts equal their runs alone bitwise."""
    base = MEMBERS[3]  # Rayleigh-Taylor, walled z
    ms, steps = [], []
    for k in range(35):
        m = dict(base)
        m["dims"] = (6 + 2 * (k % 5), 4 + (k % 3), 5 + (k % 4))
        m["seed"] = 50 + k
        ms.append(m)
        steps.append(5 + (k % 7))
    alone = []
    for m, n in zip(ms, steps):
        d = make(m)
        d.step(n)
        alone.append(d.get_state())
    b = Batch()
    doms = [make(m) for m in ms]
    for d, n in zip(doms, steps):
        b.add(d, n)
    b.step(3)
    b.step(20)
    for d, ref in zip(doms, alone):
        assert all(np.array_equal(x, y) for x, y in zip(d.get_state(), ref))
    b.close()


def test_batch_writes_every_slot():
    """Every member's target set is poisoned with NaN before each batch step;
    no NaN survives."""
    from paper_2101_06769_gb300.lbmp import OPT_TEST_POISON
    b = Batch()
    doms = [make(m) for m in MEMBERS]
    for d in doms:
        b.add(d, 3)
    for _ in range(3):
        for d in doms:
            d.set_option(OPT_TEST_POISON, 1)
            d.sync()  # the poison runs on the member's stream, the batch on its own
        b.step(1)
    for d in doms:
        f, g, phi = d.get_state()
        assert np.isfinite(f).all() and np.isfinite(g).all() and np.isfinite(phi).all()
    b.close()


def test_batch_with_symmetry_axis_members_is_bitwise_stepping_alone():
    """D2Q9 members with a symmetry x axis (reading A28), on both phase
    lattices, next to periodic ones: the batch kernel takes each member's
    boundary from its parameters, and every member equals its run alone
    bitwise."""
    from test_gpu_parity import CASES as P
    names = ["sym2d", "sym2d_red", "rt2d", "ragged2d"]
    steps = [23, 17, 30, 9]

    def mk(name):
        c = P[name]
        d = Domain(c["D"], c["dims"], c["periodic"], **c["phys"])
        d.init(c["case"], c["args"], seed=c["seed"])
        return d

    alone = []
    for name, n in zip(names, steps):
        d = mk(name)
        d.step(n)
        alone.append(d.get_state())
        d.close()
    b = Batch()
    doms = [mk(name) for name in names]
    for d, n in zip(doms, steps):
        b.add(d, n)
    b.step(5)
    b.step(30)
    for d, ref in zip(doms, alone):
        assert all(np.array_equal(x, y) for x, y in zip(d.get_state(), ref))
    b.close()
