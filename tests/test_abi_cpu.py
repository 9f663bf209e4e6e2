"""CPU-side checks of the C-ABI library: it builds, loads without a GPU and
exports every entry point the headers declare. No compute call is made."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in ("bse.h", "bse_stages.h"):
        with open(os.path.join(ROOT, "include", h)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:[a-z_]+\s+)*[a-z_]+\s*\*?\s*(bse_[A-Za-z0-9_]+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1501_03830_gb300 import build as b

    b.build()
    from paper_1501_03830_gb300 import bse

    L = bse.lib()
    declared = _declared()
    assert len(declared) >= 25
    missing = sorted(s for s in declared if not hasattr(L, s))
    assert not missing, missing
    assert set(bse.EXPORTS) == declared
    assert "sm_103a" in bse.version()


def test_status_codes_match_header():
    from paper_1501_03830_gb300 import bse

    with open(os.path.join(ROOT, "include", "bse.h")) as f:
        src = f.read()
    codes = dict(re.findall(r"#define (BSE_[A-Z0-9_]+) \(?(-?\d+)\)?", src))
    for k, v in codes.items():
        assert getattr(bse, k) == int(v), k


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    """No silent CPU path: a missing library is an error, not a fallback."""
    from paper_1501_03830_gb300 import bse

    monkeypatch.setattr(bse, "_lib", None)
    monkeypatch.setattr(bse, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        bse.lib()


def test_oracle_not_imported_by_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1501_03830_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith(".py"):
                with open(os.path.join(dirpath, fn)) as f:
                    assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", f.read(), flags=re.M)
