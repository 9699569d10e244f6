"""Launch-shape options and the autotuner on the GPU: speed only, never
results."""
import numpy as np
import pytest

from paper_2101_06769_gb300 import Domain, LbmpError
from paper_2101_06769_gb300.lbmp import FLAG_PHASE_REDUCED, OPT_CHUNK, OPT_CTAS_PER_SM, OPT_TILE, FP16_SHIFTED

from test_gpu_parity import CASES

pytestmark = pytest.mark.gpu


def dom(name, **kw):
    c = CASES[name]
    d = Domain(c["D"], c["dims"], c["periodic"], **c["phys"], **kw)
    d.init(c["case"], c["args"], seed=c["seed"])
    return d


@pytest.mark.parametrize("name,storage", [("splash3d", 0), ("rt2d", 0), ("rt3d", FP16_SHIFTED)])
def test_launch_shapes_give_identical_results(name, storage):
    ref = dom(name, storage=storage)
    ref.step(9)
    want = ref.get_state()
    for chunk, ctas in ((1, 1), (3, 2), (7, 0), (1000, 5)):
        d = dom(name, storage=storage)
        d.set_option(OPT_CHUNK, chunk)
        d.set_option(OPT_CTAS_PER_SM, ctas)
        d.step(9)
        got = d.get_state()
        assert all(np.array_equal(a, b) for a, b in zip(got, want)), (chunk, ctas)


@pytest.mark.parametrize("name", ["splash3d", "wide3d", "ragged3d", "thin3d"])
def test_tile_shapes_agree(name):
    """The 16 x 8 and 8 x 16 tile builds of the FP32 D3Q27 kernel perform the
    same per-cell operations; compiled as separate units they may fuse a
    multiply-add differently, so they agree to within rounding (the FP32
    parity bar against the oracle is 1e-5)."""
    ref = dom(name)
    ref.step(25)
    want = ref.get_state()
    for tile in (1, 2):
        d = dom(name)
        d.set_option(OPT_TILE, tile)
        d.step(25)
        for a, b in zip(d.get_state(), want):
            scale = np.abs(b).max()
            assert np.abs(a - b).max() <= 5e-6 * (scale if scale > 0 else 1.0), tile


def test_bad_options_rejected():
    d = dom("thin3d")
    for opt, v in ((OPT_CHUNK, -1), (OPT_CTAS_PER_SM, -2), (OPT_CTAS_PER_SM, 65), (OPT_TILE, 3), (7, 0)):
        with pytest.raises(LbmpError):
            d.set_option(opt, v)


@pytest.mark.parametrize("name,storage,flags", [("splash3d", 0, 0), ("rt2d", 0, 0), ("rt3d", FP16_SHIFTED, 0),
                                                ("rt3d", 0, FLAG_PHASE_REDUCED), ("rt2d", 0, FLAG_PHASE_REDUCED)])
def test_autotune_does_not_advance_or_change_state(name, storage, flags, tmp_path, monkeypatch):
    """Trial launches change nothing a later step sees: the populations, the
    step count and, on the reduced phase lattice, the stored previous phi u
    (a step after tuning equals the same step of an untuned twin bitwise)."""
    monkeypatch.setenv("LBMP_TUNE_CACHE", str(tmp_path / "tune.json"))
    kw = dict(storage=storage)
    if flags:
        kw["flags"] = flags
    a, b = dom(name, **kw), dom(name, **kw)
    a.step(4)
    b.step(4)
    before = a.get_state()
    chunk, ctas, trials = a.autotune(reps=2)
    assert len(trials) >= 3 and all(t[2] > 0 for t in trials)
    assert (chunk, ctas) in [(t[0], t[1]) for t in trials]
    after = a.get_state()
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    assert a.observables().step == 4
    a.step(5)
    b.step(5)
    assert all(np.array_equal(x, y) for x, y in zip(a.get_state(), b.get_state()))
    # second call: served from the cache, same choice, no trials
    c = dom(name, **kw)
    chunk2, ctas2, trials2 = c.autotune(reps=2)
    assert (chunk2, ctas2) == (chunk, ctas) and trials2 == []
