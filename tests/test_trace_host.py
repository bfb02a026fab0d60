"""NVTX ranges (domain "hc") around the entry points, recorded by an
injection library: the host-only paths of hc_load and hc_save open and close
their range even when they fail before any device work (no GPU needed)."""
import pytest

from trace_tools import balanced, record


def test_failed_calls_close_their_ranges(tmp_path):
    code = ("import ctypes\n"
            "from paper_1209_0410_gb300 import hc\n"
            "L = hc.lib()\n"
            "h = ctypes.c_void_p()\n"
            "assert L.hc_load(b'/nonexistent/idx.hcx', None, None, ctypes.byref(h)) == hc.HC_ERR_IO\n"
            "assert L.hc_save(None, b'x', None) == hc.HC_ERR_ARG\n")
    lines = record(code, tmp_path, timeout=300)
    assert lines == ["push hc hc_load", "pop hc", "push hc hc_save", "pop hc"]
    assert balanced(lines)
