"""The C-ABI library loads and exports every entry point include/hc.h
declares (no GPU needed: nothing is called that touches a device), and the
product binding refuses to run without it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hc.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"HC_API\s+[\w\s\*]+?\b(hc_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libhc():
    from paper_1209_0410_gb300 import _build
    path = _build.build_hc()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = declared_symbols()
    for name in ("hc_build", "hc_query", "hc_free", "hc_strerror", "hc_query_host",
                 "hc_build_host", "hc_hilbert_keys", "hc_sort_keys", "hc_query_positions",
                 "hc_bruteforce", "hc_query_ordered", "hc_query_ordered_workspace"):
        assert name in syms


def test_library_exports_every_declared_symbol(libhc):
    missing = [s for s in declared_symbols() if not hasattr(libhc, s)]
    assert not missing, "declared in hc.h but not exported: %s" % missing


def test_no_undeclared_exports(libhc):
    """Every exported hc_* symbol is declared in the header."""
    import subprocess
    from paper_1209_0410_gb300 import _build
    out = subprocess.run(["nm", "-D", "--defined-only", _build.HC_LIB], stdout=subprocess.PIPE,
                         text=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if " T hc_" in ln})
    assert set(exported) <= set(declared_symbols())


def test_strerror_without_gpu(libhc):
    libhc.hc_strerror.restype = ctypes.c_char_p
    assert libhc.hc_strerror(0) == b"ok"
    assert libhc.hc_strerror(-2) == b"out of memory"
    assert libhc.hc_strerror(12345) == b"unknown status"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1209_0410_gb300 import hc
    monkeypatch.setattr(hc, "_LIB", None)
    monkeypatch.setattr(hc, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        hc.lib()


def test_product_path_does_not_import_oracle():
    """The binding and the library sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_1209_0410_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert "from oracle" not in text and "import oracle" not in text, f
                assert "hc_oracle" not in text and "liboracle" not in text, f


def test_checked_build_exports_the_same_entry_points():
    import subprocess
    from paper_1209_0410_gb300 import _build
    _build.build_hc_check()

    def exported(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], stdout=subprocess.PIPE,
                             text=True).stdout
        return {ln.split()[-1] for ln in out.splitlines() if " T hc_" in ln}

    assert exported(_build.HC_CHECK_LIB) == exported(_build.HC_LIB)


def test_normal_build_reports_checks_disabled(libhc):
    from paper_1209_0410_gb300 import hc
    assert hc.hc_check_status() == dict(enabled=0, site=0, violations=0, index=0, bound=0)
