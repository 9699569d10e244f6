"""The oracle and the CUDA path share no code, and the product never reaches
the oracle: no file of the package (binding, CUDA sources, public header)
names the oracle, no oracle file names the package, its sources or its
header, and the binding raises instead of falling back when the CUDA
library is missing."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PRODUCT = (glob.glob(os.path.join(ROOT, "paper_2101_06769_gb300", "*.py")) +
           glob.glob(os.path.join(ROOT, "paper_2101_06769_gb300", "csrc", "*")) +
           glob.glob(os.path.join(ROOT, "include", "*")))
ORACLE = [p for p in glob.glob(os.path.join(ROOT, "oracle", "*")) if os.path.isfile(p)]


def _text(p):
    with open(p, errors="replace") as fh:
        return fh.read()


def test_product_never_names_the_oracle():
    assert PRODUCT
    for p in PRODUCT:
        if os.path.isfile(p):
            assert not re.search(r"\boracle\b|lbmo", _text(p)), p


def test_oracle_never_names_the_product():
    assert ORACLE
    for p in ORACLE:
        assert not re.search(r"paper_2101_06769_gb300|csrc|lbmp|lbmp\.h", _text(p)), p


def test_binding_fails_loudly_without_the_library(monkeypatch):
    from paper_2101_06769_gb300 import lbmp
    monkeypatch.setattr(lbmp, "_lib", None)
    monkeypatch.setattr(lbmp, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "liblbmp.so"))
    monkeypatch.delenv("LBMP_LIBRARY", raising=False)
    with pytest.raises(RuntimeError, match="not built"):
        lbmp.load()
