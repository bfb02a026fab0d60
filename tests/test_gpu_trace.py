"""NVTX ranges of the device paths, recorded by the injection library in a
child process: hc_build opens "hc_build" with its "keys" and "sort" phases,
hc_query_ordered its "order", "search" and "walk" phases, and every range
closes."""
import pytest

from trace_tools import balanced, record

pytestmark = pytest.mark.gpu

CODE = """
import torch
from paper_1209_0410_gb300 import datagen, hc
db = torch.from_numpy(datagen.make_db(5000, 128, seed=1)).cuda()
q = torch.from_numpy(datagen.make_queries(db.cpu().numpy(), 64, seed=2)).cuda()
idx = hc.hc_build(db)
hc.hc_query(idx, q, 10, 16)
hc.hc_query_ordered(idx, q, 10, 16)
torch.cuda.synchronize()
idx.free()
"""


def test_device_paths_record_their_ranges(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lines = record(CODE, tmp_path)
    assert balanced(lines)

    def seq(*names):
        out = []
        for n in names:
            out += n if isinstance(n, list) else ["push hc " + n, "pop hc"]
        return out

    text = "\n".join(lines)
    build = ["push hc hc_build"] + seq("keys", "sort") + ["pop hc"]
    ordered = ["push hc hc_query_ordered"] + seq("order", "search", "walk") + ["pop hc"]
    assert "\n".join(build) in text
    assert "\n".join(["push hc hc_query", "pop hc"]) in text
    assert "\n".join(ordered) in text
