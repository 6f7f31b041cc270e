"""Host-side logic of bench.py: byte models, whole-job throughput and the
multi-rank timing reduction (world_size 2, gloo, on CPU)."""
import os
import socket

import pytest

import bench


def test_level_pixels_and_lk_bytes():
    assert bench.level_pixels(4000, 1500, 3) == [6_000_000, 1_500_000, 375_000]
    b = bench.lk_alg_bytes(4000, 1500, 2)
    # level 0: 2 directions x (T + J 8 B, coarse flow 8 B per coarse pixel, flow out 8 B)
    assert b[0] == 2 * (8 * 6_000_000 + 8 * 1_500_000 + 8 * 6_000_000)
    assert b[1] == 2 * (8 * 1_500_000 + 8 * 1_500_000)


def test_issue_roofline_against_the_schedulers_peak():
    # 1.2587e11 warp instructions per second = 152 SMs x 4 schedulers x 2070 MHz / 10
    counters = {"kernel": "lk_stream_kernel", "workload": "pair_4000x1500_rgb_u8_lv6",
                "warp_inst_per_launch": 125.5e6}
    launch_ms = 125.5e6 / (0.1 * 152 * 4 * 2070e6) * 1e3
    r = bench.issue_roofline(counters, launch_ms, 2070.0, 152)
    assert r["peak"] == pytest.approx(152 * 4 * 2.07)
    assert r["frac"] == pytest.approx(0.1)
    # no counters, no clock sample: no figure
    assert bench.issue_roofline(None, 1.0, 2070.0, 152) is None
    assert bench.issue_roofline(counters, 1.0, None, 152) is None


def test_path_bytes_follow_the_per_pixel_model():
    # 4000x1500 RGB u8, 6 levels: strips 6 B, luma levels 8 S, flow 36 S (minus the
    # coarsest level's missing coarse read), blend 25 B: about 90 B per pixel
    n = 4000 * 1500
    b = bench.path_alg_bytes(4000, 1500, 3, 6)
    assert 89.0 < b / n < 90.0
    # the REDUCE re-read model adds 8 B per pixel of levels 0-4
    rr = bench.path_alg_bytes(4000, 1500, 3, 6, reduce_reread=True)
    assert rr - b == 8 * sum(bench.level_pixels(4000, 1500, 6)[:-1])
    # a one-channel float strip is its own level 0: no level-0 write
    g = bench.path_alg_bytes(256, 512, 1, 4, in_bytes=4)
    npx = bench.level_pixels(256, 512, 4)
    assert g == 2 * 4 * 256 * 512 + 8 * sum(npx[1:]) + sum(bench.lk_alg_bytes(256, 512, 4)) + 28 * 256 * 512


def test_ncu_counters_round_trip_and_go_stale_with_the_source(tmp_path, monkeypatch):
    csv = tmp_path / "raw.csv"
    csv.write_text(
        '"ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum","smsp__inst_executed.sum",'
        '"gpu__time_duration.sum"\n'
        '"","","Mbyte","Kbyte","inst","nsecond"\n'
        '"0","void lk_stream_kernel<2, 5, 96, 12, float>(LkArgs, int)","110.5","2,000","368200597","623600"\n'
        '"1","void lk_stream_batch_kernel<2, 5, 96, 12, float>(LkBatch)","1","1","1","1"\n'
        '"2","lk_stream_kernel<2, 5, 96, 12, float>","18.5","0","90773349","172300"\n')
    rows = bench.parse_ncu_raw_csv(str(csv), "lk_stream_kernel")
    assert len(rows) == 2
    assert rows[0]["dram_bytes"] == pytest.approx(110.5e6 + 2e6)
    assert rows[1]["warp_inst"] == 90773349
    out = bench.ingest_ncu(str(csv), "lk_stream_kernel", "pair_4000x1500_rgb_u8_lv6", "cmd",
                           profiles_dir=str(tmp_path))
    assert os.path.exists(out)
    c = bench.read_counters("lk_stream_kernel", "pair_4000x1500_rgb_u8_lv6", profiles_dir=str(tmp_path))
    assert c["dram_bytes_per_launch"] == pytest.approx((112.5e6 + 18.5e6) / 2)
    assert c["warp_inst_per_launch"] == pytest.approx((368200597 + 90773349) / 2)
    # the kernel's sources change: the counters no longer apply
    monkeypatch.setattr(bench, "source_digest", lambda files: "0" * 64)
    assert bench.read_counters("lk_stream_kernel", "pair_4000x1500_rgb_u8_lv6", profiles_dir=str(tmp_path)) is None


def test_throughput_counts_every_rank():
    # 6 MP per step, 10 steps, 2 ranks, slowest rank 20 ms in total
    assert bench.throughput(6_000_000, 10, 2, 20.0) == pytest.approx(6000.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        total_ms = 10.0 + 5.0 * rank          # rank 1 is slower
        m = bench.reduce_max(total_ms, world)
        value = bench.throughput(1_000_000, 4, world, m)
        q.put((rank, m, value, bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_reduce_max_and_barrier_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, value, env in res:
        assert m == 15.0                       # max over ranks
        assert value == pytest.approx(1_000_000 * 4 * 2 / 15e-3 / 1e6)
        assert env[0] == rank and env[1] == 2


def test_reference_arm_on_nonzero_rank_exits_quietly(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"]) == 0
    assert capsys.readouterr().out == ""


def test_warmup_below_three_is_rejected():
    with pytest.raises(SystemExit):
        bench.main(["--warmup", "2"])


def test_rig_level_kernels_follow_the_size_rule_and_forced_kinds():
    widths = bench.RIG_WORKLOAD["widths"]
    plan = bench.rig_level_kernels(4000, widths, 6, [bench.PANO_LK_AUTO] * 6)
    # level 3 is 500 rows: every width (>= 100) gives >= 50000 pixels; level 4
    # (250 rows) is tiled, with 16 x 8 tiles for the pairs below 16000 pixels
    # (widths 50 and 60); level 5 is small for every pair
    assert plan[3] == [("lk_stream_batch_kernel", list(range(8)))]
    assert plan[4] == [("lk_level_batch_kernel", [0, 1]), ("lk_level_batch_kernel", [2, 3, 4, 5, 6, 7])]
    assert plan[0] == [("lk_stream_batch_kernel", list(range(8)))]
    assert plan[5] == [("lk_level_batch_kernel", list(range(8)))]
    tuned = bench.rig_level_kernels(4000, widths, 6, [bench.PANO_LK_TILE] * 6, [(32, 8)] * 6)
    assert all(p == [("lk_level_batch_kernel", list(range(8)))] for p in tuned)
    forced = bench.rig_level_kernels(4000, widths, 6, [bench.PANO_LK_TILE] + [bench.PANO_LK_STREAM] * 5)
    assert forced[0] == [("lk_level_batch_kernel", list(range(8)))]
    assert all(p == [("lk_stream_batch_kernel", list(range(8)))] for p in forced[1:])
