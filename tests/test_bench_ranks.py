"""bench.py's multi-rank path (replicas, one per GPU): the slowest rank's time and the sum
of all ranks' iterations, checked with two gloo ranks on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, its = bench.reduce_over_ranks(100.0 + 50.0 * rank, 57 + rank, dist, "cpu")
    out.put((rank, ms, its))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_iterations():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert res == [(0, 150.0, 115.0), (1, 150.0, 115.0)]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(12.5, 7, None, "cpu") == (12.5, 7.0)


def test_clock_summary_reads_nvidia_smi_lines():
    """The clocks object of a bench line: median SM clock under load, the maximum, and the
    throttle reasons seen Active in any sample (the ones that void a measurement)."""
    sys.path.insert(0, ROOT)
    import bench

    c = bench.ClockSampler(0)
    c.lines = [
        "0, 1590, 2070, 1380.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2025, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1300.0, 0x0, Not Active, Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                                               "samples": 0}


def test_measured_traffic_is_keyed_on_source_size_and_setting(tmp_path, monkeypatch):
    """A traffic figure from profiles/roofline_traffic.txt is used only for the kernel
    source it was captured on (sha256), the captured sizes and, for the Gram, the
    captured launch setting; anything else gives None (the line's traffic is null)."""
    import hashlib

    sys.path.insert(0, ROOT)
    import bench

    csrc = tmp_path / "paper_1710_10769_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "adjoint.cu").write_text("// kernel v1\n")
    (csrc / "gram_tc.cu").write_text("// gram v1\n")
    sha = lambda name: hashlib.sha256((csrc / name).read_bytes()).hexdigest()
    (tmp_path / "profiles" / "roofline_traffic.txt").write_text(
        "# comment = ignored\n"
        f"dense_grad.src_sha256={sha('adjoint.cu')}\ndense_grad.p=16384\ndense_grad.n=4096\n"
        "dense_grad.dram_bytes=1755441824\n"
        f"gram.src_sha256={sha('gram_tc.cu')}\ngram.p=65536\ngram.n=32768\n"
        "gram.band16.maxima1.sched1.dram_bytes=163673027072\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("dense_grad", 16384, 4096) == 1755441824.0
    assert bench.measured_traffic("dense_grad", 8192, 4096) is None
    assert bench.measured_traffic("gram", 65536, 32768, "band16.maxima1.sched1.") == 163673027072.0
    assert bench.measured_traffic("gram", 65536, 32768, "band32.maxima1.sched1.") is None
    assert bench.measured_traffic("screen_pass", 65536, 32768) is None       # no entry, no source
    (csrc / "adjoint.cu").write_text("// kernel v2\n")                      # the kernel changed
    assert bench.measured_traffic("dense_grad", 16384, 4096) is None


def test_lemma31_flop_counts():
    """The bench's statement of Lemma 3.1: F_Cov = 2np^2 + 2dp^2(st+1) and
    F_Obs = 2np^2 s + 2dnp(st+1), hand-evaluated; and its Cov-is-cheaper condition
    d/p < n/((p-n)t) agrees with comparing the two counts once s is large."""
    sys.path.insert(0, ROOT)
    import bench

    m = bench.lemma31_flops(n=100, p=400, s=10, t=3, d=5)
    assert m["flops_cov"] == 2 * 100 * 400 ** 2 + 2 * 5 * 400 ** 2 * 31
    assert m["flops_obs"] == 2 * 100 * 400 ** 2 * 10 + 2 * 5 * 100 * 400 * 31
    for n, p, t, d in [(100, 400, 3, 5), (100, 40000, 2.9, 8), (8192, 16384, 3, 1.2), (500, 520, 4, 40),
                       (12800, 40000, 3, 200), (100, 40000, 3, 0.5)]:
        big = bench.lemma31_flops(n, p, 1e9, t, d)
        assert big["cov_cheaper"] == (big["flops_cov"] < big["flops_obs"]), (n, p, t, d)
    assert bench.lemma31_flops(n=500, p=400, s=3, t=2, d=9)["cov_cheaper"] is True     # p <= n
