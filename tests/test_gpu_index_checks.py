"""Device-side index checks (the checked build, libdbmp_checked.so), in place of a
device-assert build: a failing assert would trap the GPU.  Three bad indices are
planted in a binned workspace with dbmp_workspace_debug_set, each inside the
allocations, so that a missing check could only produce a wrong value:
  - a tile-list entry naming a stale record past N (a valid primitive of an earlier
    binning), in the middle of the longest list;
  - the last tile's list range ending past sum_t d_t, over entries naming primitive 0;
  - a record's bitmap row set to a row inside the texel plane that starts no bitmap.
The checked build must name the first bad index in the status block, skip the access,
and render every other pixel like the FP64 oracle (the tile that lost an entry like the
oracle without that primitive)."""
import json
import os
import subprocess
import sys

import pytest

from paper_2602_22625_gb300 import dbmp as D
from _helpers import cuda

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(os.environ.get("DBMP_LIBRARY") == "checked",
                    reason="the suite itself runs on the checked library")
def test_the_default_build_has_no_checks():
    cuda()
    assert D.dbmp_index_checks() is False


def test_checked_build_names_the_first_bad_index_and_skips_it():
    cuda()
    env = dict(os.environ, DBMP_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_checked_worker.py")], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checks"] is True
    assert out["clean"] == {"bad_kind": 0, "err": out["clean"]["err"]} and out["clean"]["err"] <= 1e-5
    e = out["list_entry"]
    assert (e["bad_kind"], e["bad_index"]) == (D.BAD_LIST_ENTRY, e["want_index"])
    assert e["err_other"] <= 1e-5 and e["err_tile"] <= 1e-5, e
    e = out["tile_range"]
    assert (e["bad_kind"], e["bad_index"]) == (D.BAD_TILE_RANGE, e["want_index"]) and e["err"] <= 1e-5, e
    e = out["bitmap_row"]
    assert (e["bad_kind"], e["bad_index"]) == (D.BAD_BITMAP_ROW, e["want_index"]) and e["err"] <= 1e-5, e
