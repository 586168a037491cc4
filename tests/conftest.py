import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    if os.environ.get("DBMP_LIBRARY") == "checked":
        strict_index_checks()


def strict_index_checks():
    """With DBMP_LIBRARY=checked the whole suite runs on the index-checked library,
    whose kernels record the first out-of-range tile range, list entry or bitmap row in
    the status block and skip the access: a status poll that finds one recorded fails
    the test that made it (the skipped access alone might go unnoticed)."""
    from paper_2602_22625_gb300 import dbmp as D
    poll = D.dbmp_status_poll

    def strict_poll(ws, stream=None, raise_on_error=True):
        st = poll(ws, stream, raise_on_error)
        assert not st.bad_kind, f"index check fired: kind {st.bad_kind}, index {st.bad_index}"
        return st
    D.dbmp_status_poll = strict_poll


def pytest_collection_modifyitems(config, items):
    import pytest
    try:
        import torch
        has_cuda = torch.cuda.is_available()
    except Exception:
        has_cuda = False
    if has_cuda:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
