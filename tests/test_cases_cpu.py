"""JSON case files (host logic, no GPU)."""
import json

import pytest

from paper_2101_06769_gb300 import cases


def test_shipped_cases_load_and_map():
    names = cases.shipped()
    assert {"rt2d", "rt3d", "splash3d", "splash3d_large"} <= set(names)
    for n in names:
        c = cases.load(n)
        wl = cases.as_workload(c)
        assert wl["D"] in (2, 3) and len(wl["dims"]) == 3
        assert (wl["D"] == 2) == (wl["dims"][2] == 1)


def test_invalid_cases_rejected(tmp_path):
    good = cases.load("rt3d")
    for mutate in (lambda c: c.pop("grid"), lambda c: c.update(lattice="D3Q19"),
                   lambda c: c["params"].update(bogus=1.0), lambda c: c["init"].update(case="nope"),
                   lambda c: c.update(periodic=[1, 1])):
        c = json.loads(json.dumps(good))
        mutate(c)
        p = tmp_path / "bad.json"
        p.write_text(json.dumps(c))
        with pytest.raises(ValueError):
            cases.load(str(p))
