"""Host logic of bench.py on CPU: the multi-rank path (two gloo ranks with different step
times agree on the slowest rank's time, and the whole-job throughput counts both ranks'
units: replicas, weak scaling) and the reference arm's sampling of the image."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (t, bench.job_throughput(world, 10, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    times = [123.0, 456.5]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == max(times)
        assert v == pytest.approx(world * 10 / (max(times) / 1e3))


def test_one_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_throughput(1, 4, 2000.0) == pytest.approx(2.0)


def test_reference_slices_cover_every_row_once_per_cycle():
    for H, h, cores in ((680, 16, 15), (680, 1, 16), (680, 8, 4), (17, 16, 3)):
        slices = bench.image_slices(H, h, cores)
        rows = [r for sl in slices for r0, nr in sl for r in range(r0, r0 + nr)]
        assert rows == list(range(H))
        assert all(1 <= len(sl) <= cores for sl in slices) and all(len(sl) == cores for sl in slices[:-1])
        assert all(nr == h for sl in slices for r0, nr in sl[:-1])


def test_reference_band_height_fits_the_budget():
    # 1-row steps 0.5 s, 16-row steps 2 s, so 8, 4 and 2 rows take 1.2, 0.8 and 0.6 s: the
    # tallest band whose step fits budget / (steps + warm-up) is chosen
    assert bench.reference_band_rows(0.5, 2.0, 10, 2, 240.0) == 16      # 20 s per step
    assert bench.reference_band_rows(0.5, 2.0, 200, 10, 240.0) == 4     # 1.14 s per step
    assert bench.reference_band_rows(0.5, 2.0, 300, 10, 240.0) == 2     # 0.77 s per step
    assert bench.reference_band_rows(0.5, 2.0, 1000, 10, 240.0) == 1    # 0.24 s per step


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops_sustained"] == 1700.0


def test_tile_walk_counts_each_tile_at_its_longest_pixel():
    import torch
    nc = torch.tensor([[1, 5, 0, 2, 7],
                       [3, 0, 4, 4, 1],
                       [9, 2, 0, 0, 6]], dtype=torch.int32).view(-1)
    # 2x2 tiles: maxima 5, 4, 7 (top row), 9, 0, 6 (bottom row, padded); 4 pixels each
    assert bench.tile_evals(nc, 5, 3, 2, 2) == 4 * (5 + 4 + 7 + 9 + 0 + 6)
    assert bench.tile_evals(nc, 5, 3, 5, 3) == 15 * 9          # one tile
    assert bench.tile_evals(nc, 5, 3, 1, 1) == int(nc.sum())   # a tile per pixel: E itself
