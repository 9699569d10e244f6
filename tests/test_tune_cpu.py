"""Host logic of the launch-shape tuning cache (no GPU)."""
import json
import types

from paper_2101_06769_gb300 import tune


def fake_dom(D=3, dims=(128, 128, 512), storage=0, periodic=(1, 1, 0), reduced=False):
    Q = 27 if D == 3 else 9
    return types.SimpleNamespace(D=D, dims=dims, storage=storage, periodic=periodic, Q=Q,
                                 Qg=2 * D + 1 if reduced else Q)


def test_key_separates_every_field():
    base = tune.key_of(fake_dom(), "GB300")
    others = [tune.key_of(fake_dom(D=2, dims=(128, 128, 1)), "GB300"),
              tune.key_of(fake_dom(storage=1), "GB300"),
              tune.key_of(fake_dom(dims=(128, 128, 256)), "GB300"),
              tune.key_of(fake_dom(periodic=(1, 1, 1)), "GB300"),
              tune.key_of(fake_dom(), "other GPU"),
              tune.key_of(fake_dom(reduced=True), "GB300")]
    assert len({base, *others}) == 7


def test_cache_round_trip_and_corrupt_file(tmp_path):
    p = str(tmp_path / "sub" / "tune.json")
    assert tune.read_cache(p) == {}
    tune.write_cache(p, {"k": {"chunk": 16, "ctas_per_sm": 2, "ms": 1.0}})
    assert tune.read_cache(p)["k"]["chunk"] == 16
    with open(p, "w") as fh:
        fh.write("{not json")
    assert tune.read_cache(p) == {}
    with open(p, "w") as fh:
        json.dump([1, 2], fh)
    assert tune.read_cache(p) == {}


def test_cache_path_env(monkeypatch, tmp_path):
    monkeypatch.setenv("LBMP_TUNE_CACHE", str(tmp_path / "x.json"))
    assert tune.cache_path() == str(tmp_path / "x.json")
