"""Host-side pieces of bench.py: clock parsing, the algorithmic work model,
the max-over-ranks reduction on two gloo ranks, and the reference arm (the
FP64 oracle timed on the host), alone and under torchrun with two ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_parse_clocks():
    lines = ["0, 1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Active\n",
             "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active\n",
             "0, 1800, 2070, 1100.0, 0x0, Active, Not Active, Not Active, Not Active\n",
             "garbage\n"]
    c = bench.parse_clocks(lines)
    assert c["sm_mhz"] == 1965 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_stage_work_model():
    w = bench.stage_work(256, 512, 6, 512, 92160, 23639040)
    f = w["forward"]
    assert f["x_pass"]["bytes"] == 4 * 256 ** 3 + 8 * 256 * 256 * 512
    assert f["z_pass"]["bytes"] == 8 * 256 * 512 * 512 + 8 * 512 ** 3
    assert f["gather"]["flops"] == 8 * (216 + 36 + 6) * 23639040
    assert w["adjoint"]["spread"]["smem_bytes"] == 2 * f["gather"]["smem_bytes"]
    # the fixed-point spread moves two 4-byte reductions per tap, as many bytes as the gather's reads
    wf = bench.stage_work(256, 512, 6, 512, 92160, 23639040, spread_tap_bytes=8)
    assert wf["adjoint"]["spread"]["smem_bytes"] == f["gather"]["smem_bytes"] == 216 * 8 * 23639040


def test_resample_source_hash_is_separate():
    # the traffic entries of the interpolation kernels and of the polar resampler
    # are keyed by the hashes of their own sources
    assert bench.source_hash() != bench.source_hash(bench.RESAMPLE_SOURCES)
    assert len(bench.source_hash(bench.RESAMPLE_SOURCES)) == 16


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _max_worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    q.put((rank, bench.max_over_ranks(world, 1.5 + rank)))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]


def test_reference_arm_prints_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "tiny32", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "pts/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port),
                        os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny32",
                        "--steps", "1", "--warmup", "1", "--gpus", "2"],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["n_gpus"] == 2
