"""bench.py's multi-GPU mode runs independent replicas (one analysis per rank,
no collective on the data path); its whole-job numbers are the slowest rank's
time and the sum of all ranks' evaluations. Checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ms, ev = bench.reduce_ranks(dist, total_ms=100.0 + 50.0 * rank, evals=1000 + rank)
    out.put((rank, ms, ev))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ms, ev in res:
        assert ms == 150.0 and ev == 2001.0


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_ranks(None, 12.5, 7) == (12.5, 7.0)


def test_mixed_roofline_takes_the_binding_pipe():
    """The mixed form's roofline is that of the pipe its instruction counts bind:
    the FP32 pipe for the rotation form (tiles of 32+ bins), the MUFU pipe for
    the direct tiled form (6 sin/cos per point-bin at 3 detectors)."""
    import bench
    assert bench.mixed_fp32_per_point_bin(3, 128) == 37.5
    assert bench.mixed_mufu_per_point_bin(3, 128) == 2.0
    assert bench.mixed_fp32_per_point_bin(3, 16) == 45.0
    assert bench.mixed_mufu_per_point_bin(3, 16) == 6.0
    assert bench.mixed_fp32_per_point_bin(3, 0) == 156.0
    pb, secs = 1e12, 1.0
    frac, pipe = bench.mixed_roofline(pb, secs, 3, 128)
    assert pipe == "FP32" and abs(frac - pb * 37.5 / bench.FP32_LANE_OPS) < 1e-12
    frac, pipe = bench.mixed_roofline(pb, secs, 3, 16)
    assert pipe == "SFU" and abs(frac - pb * 6.0 / bench.SFU_LANE_OPS) < 1e-12
    # one detector in the direct form: 23 FP32 against 2 MUFU -> FP32 binds (23/128 > 2/16)
    frac, pipe = bench.mixed_roofline(pb, secs, 1, 16)
    assert pipe == "FP32"


def test_recorded_traffic_is_dropped_when_the_kernel_changes(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu summary only while
    the hash of the kernel's sources it records matches the current sources."""
    import bench
    f = tmp_path / "traffic.md"
    sha = bench.kernel_source_sha16()
    f.write_text(f"source_sha16: {sha}\ndram_bytes_per_launch: 123456\npoint_bins_per_launch: 1000\n")
    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(f))
    assert bench.recorded_traffic() == (123456, 1000)
    f.write_text("source_sha16: 0123456789abcdef\ndram_bytes_per_launch: 123456\n")
    assert bench.recorded_traffic() == (None, None)
    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.recorded_traffic() == (None, None)


def test_both_arms_describe_the_same_configuration():
    import bench
    assert bench.config_dict(1) == bench.config_dict(1)
    assert bench.config_dict(2)["parallelism"] == "replicas2"


def test_executed_count_drops_the_low_degree_horner_steps():
    """The executed FP32 count per point-bin is the frozen one (rotation form,
    degree-7 tiles) on bins of degree-7 groups and 4 fewer on bins of the
    degree-3 groups, weighted by their share."""
    import bench
    frozen = bench.mixed_fp32_per_point_bin(3, 128)
    assert frozen == 37.5
    assert bench.executed_count(1000, 0, 3, 128) == frozen
    assert bench.executed_count(1000, 1000, 3, 128) == frozen - 4.0
    assert abs(bench.executed_count(1000, 250, 3, 128) - (frozen - 1.0)) < 1e-12
    r = bench.executed_roofline(1e10, 5e9, 0.01, 3, 128, "FP32")
    assert abs(r["frac"] - 1e10 * (frozen - 2.0) / 0.01 / bench.FP32_LANE_OPS) < 1e-12
    assert bench.executed_roofline(1e10, 5e9, 0.01, 3, 16, "SFU") is None
