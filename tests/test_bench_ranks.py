"""bench.py's host-side arithmetic: the replica reduction across ranks (slowest time, summed
codewords, with two gloo ranks on the CPU), the roofline lines and the workload strings the
two arms share."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    secs, cw = bench.reduce_over_ranks(1.0 + rank, 10 ** 12 * (rank + 1), "cpu")
    out[rank] = (secs, cw)
    dist.destroy_process_group()


def test_reduce_over_two_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 3 * 10 ** 12)


def test_reduce_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 7, "cpu") == (3.5, 7)


def test_roofline_line_arithmetic():
    """The tensor roofline: 2 x 32 F flops per codeword (F = the product's packed words) over
    the per-launch time, against the sustained bf16 rate x 2 (fp8), with the method's own work
    (2 (n - k) flops per codeword) beside it; the popcount roofline: one POPC per codeword
    against 16 x 152 x 2070 MHz."""
    import types
    import bench
    peaks = bench.measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    args = types.SimpleNamespace(tensor=1)
    r = bench.roofline_line(args, 200, 100, 10, 4, 1.7e13, 1.5, 3)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(1.7e13 * 192 / 1.5 / 1e12)
    assert r["peak"] == pytest.approx(2 * bf16)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["method"]["achieved"] == pytest.approx(1.7e13 * 200 / 1.5 / 1e12)
    assert r["method"]["frac"] == pytest.approx(r["method"]["achieved"] / r["peak"])
    assert r["peak_codewords_per_s"] == pytest.approx(2 * bf16 * 1e12 / 192)
    assert r["traffic"] == bench.TC_KERNEL_TRAFFIC_BYTES
    # no word count reported: the full packed width (W = 4 for n - k = 100)
    r = bench.roofline_line(args, 200, 100, 10, 4, 1.7e13, 1.5, 0)
    assert r["achieved"] == pytest.approx(1.7e13 * 256 / 1.5 / 1e12)
    args.tensor = 0
    r = bench.roofline_line(args, 200, 100, 10, 4, 1.7e13, 5.0, 0)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(16 * 152 * 2070e6 / 1e9)
    assert r["achieved"] == pytest.approx(1.7e13 / 5.0 / 1e9)


def test_clock_matched_denominator():
    """The clock-matched tensor roofline: md_mma_rate's flops per SM per clock x SMs x MHz;
    16384 flops/clk/SM (one M = 128, N = 256, K = 32 MMA per 128 cycles) x 152 x 2070 MHz is
    5155 TFLOP/s, and both fractions divide the line's own achieved figures by it."""
    import types
    import bench
    r = bench.roofline_line(types.SimpleNamespace(tensor=1), 200, 100, 10, 4, 1.7e13, 1.5, 3)
    c = bench.clock_matched(r, 16384.0, 152, 2070.0)
    assert c["peak"] == pytest.approx(16384 * 152 * 2070e6 / 1e12)
    assert c["peak"] == pytest.approx(5155.0, rel=1e-3)
    assert c["frac"] == pytest.approx(r["achieved"] / c["peak"])
    assert c["frac_method"] == pytest.approx(r["method"]["achieved"] / c["peak"])


@pytest.mark.parametrize("workload", ["rand64x32", "rand128x64", "rand200x100"])
def test_workload_strings_name_the_drawn_code(workload):
    """Both arms print the same `data` and `config` for a workload, and they name that code's
    own size and seed (the reference arm and ours call the same two functions)."""
    import types
    import bench
    from paper_1911_08963_gb300 import inputs
    c = inputs.SINGLE[workload]
    args = types.SimpleNamespace(workload=workload, max_stage=10, filter=1)
    cfg = bench.workload_config(args, c["n"], c["k"])
    assert cfg["workload"].startswith("random [%d,%d] seed %d," % (c["n"], c["k"], c["seed"]))
    data = bench.data_string(workload)
    assert "I_%d|R" % c["k"] in data and "seed %d" % c["seed"] in data
    if workload == "rand200x100":
        assert data == bench.DATA
