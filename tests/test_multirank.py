"""The N > 1 paths on CPU: two gloo ranks (spawned processes, 127.0.0.1).
Replicas (bench.py's default): each rank renders its own canvas of the same workload,
the line reports the slowest rank, rank 0 alone prints.  Shared parameters
(sharded.py): one canvas split into bands of tile rows, the bands' gradients summed
by one all-reduce, checked with the FP64 oracle standing in for each rank's kernels."""
import json
import os
import socket

import torch.multiprocessing as mp

import _dist_worker


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_take_the_slowest_time_and_render_their_own_canvas(tmp_path):
    mp.start_processes(_dist_worker.run, args=(2, free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    r = [json.loads((tmp_path / f"rank{i}.json").read_text()) for i in range(2)]
    for i in range(2):
        assert r[i]["world"] == 2 and r[i]["rank"] == i and r[i]["local"] == i
        assert r[i]["max"] == [2.0, 10.0]                 # max over ranks of (1 + r, 10 - r)
    assert r[0]["seed"] != r[1]["seed"] and r[0]["tgt_seed"] != r[1]["tgt_seed"]
    assert r[0]["shape"] == r[1]["shape"]                 # weak scaling: same work per rank
    assert r[0]["param_sum"] != r[1]["param_sum"]         # ... on different canvases


def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    mp.start_processes(_dist_worker.reference_arm, args=(2, str(tmp_path)), nprocs=2, start_method="spawn")
    out0 = (tmp_path / "ref0.txt").read_text().strip().splitlines()
    out1 = (tmp_path / "ref1.txt").read_text().strip()
    assert out1 == "" and float((tmp_path / "ref1.time").read_text()) < 5.0   # no work on rank 1
    line = json.loads(out0[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"


def test_band_partition_covers_the_tile_rows_once():
    from paper_2602_22625_gb300 import sharded as S
    for H, tile in ((1024, 32), (70, 16), (77, 8), (32, 32)):
        nty = -(-H // tile)
        for world in (1, 2, 3, 4, 8, 40):
            bands = [S.band_rows(H, world, r, tile) for r in range(world)]
            assert bands[0][0] == 0 and bands[-1][1] == nty * tile
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
            sizes = [(b - a) // tile for a, b in bands]
            assert max(sizes) - min(sizes) <= 1 and all(a % tile == 0 for a, _ in bands)


def test_two_ranks_sum_their_bands_to_the_whole_canvas_gradient(tmp_path):
    mp.start_processes(_dist_worker.sharded, args=(2, free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    r = [json.loads((tmp_path / f"shard{i}.json").read_text()) for i in range(2)]
    assert r[0]["rows"] == [0, 48] and r[1]["rows"] == [48, 80]
    for x in r:
        assert x["err"] <= 1e-12, x          # the all-reduced sum is the whole gradient
        assert 0.05 < x["own"], x            # and each band carries a real part of it
