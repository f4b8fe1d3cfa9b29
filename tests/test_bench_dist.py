"""Host logic of the benchmark under several ranks, on CPU with gloo.

The benchmark runs one replica of the workload per rank (the components are
independent, so nothing crosses ranks on the data path); its only collective
is the max over ranks of the measured times. These tests run that reduction
and the whole-job rate with world size 2, and check that the reference arm
leaves all work to rank 0.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_env()
    ms = bench.max_over_ranks(times[rank], w, "cpu")
    rate = bench.whole_job_rate(1000, w, ms / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, w, loc, ms, rate))


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [3.5, 7.25]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, loc, ms, rate) in enumerate(res):
        assert (r, w, loc) == (rank, 2, rank)
        assert ms == 7.25                         # every rank reports the slowest rank's time
        assert rate == pytest.approx(2 * 1000 / 7.25e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(4.0, 1, "cpu") == 4.0
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    def boom(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "run_oracle_sample", boom)
    args = type("Args", (), {"warmup": 3, "steps": 2, "gpus": 2})()
    assert bench.run_reference(args) == 0


def test_clock_sampler_reads_nvml_state_and_falls_back(monkeypatch):
    """The NVML sampler reports the median SM clock and the union of the
    throttle reasons seen while it ran (a fake driver library here); without
    NVML the sampler is the nvidia-smi one."""
    import ctypes
    import types
    import bench

    class FakeLib:
        def __init__(self):
            self.clocks = iter([1900, 2070, 2070, 2070, 1950] + [2070] * 1000)

        def nvmlInit_v2(self):
            return 0

        def nvmlDeviceGetHandleByPciBusId_v2(self, bus, h):
            return 0

        def nvmlDeviceGetHandleByIndex_v2(self, i, h):
            return 0

        def nvmlDeviceGetClockInfo(self, h, kind, out):
            out._obj.value = next(self.clocks)
            return 0

        def nvmlDeviceGetMaxClockInfo(self, h, kind, out):
            out._obj.value = 2070
            return 0

        def nvmlDeviceGetCurrentClocksEventReasons(self, h, out):
            out._obj.value = 0x1 | 0x4          # idle + sw_power_cap
            return 0

    fake = FakeLib()
    monkeypatch.setattr(ctypes, "CDLL", lambda name: fake)
    props = types.SimpleNamespace(pci_domain_id=0, pci_bus_id=0x1b, pci_device_id=0)
    torch_stub = types.SimpleNamespace(cuda=types.SimpleNamespace(get_device_properties=lambda i: props))
    ck = bench.NvmlClocks(torch_stub, 0, period=0.001)
    ck.start()
    import time
    time.sleep(0.05)
    out = ck.stop()
    assert out["samples"] >= 5 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["sm_mhz"] == 2070.0

    monkeypatch.setattr(ctypes, "CDLL", lambda name: (_ for _ in ()).throw(OSError("no NVML")))
    assert isinstance(bench.clock_sampler(torch_stub, 0), bench.Clocks)


def test_parallel_oracle_baseline_runs_the_sample_on_every_core():
    """cpu_baseline_parallel: the oracle over a spawned pool of one-thread
    workers, per_core tasks per core, in LPT order; it reports the cores used
    and DoFs that match the serial sample's components."""
    import bench
    r = bench.run_oracle_sample(1, parallel=True)
    ncores = os.cpu_count() or 1
    assert r["cores"] == ncores and r["components"] == ncores and r["seconds"] > 0
    # p = 3 C^2: 2^l + 1 interior functions per direction
    per = [int(np.prod([2 ** l + 1 for l in lv])) for lv in bench.ORACLE_SAMPLE]
    assert r["dofs"] == sum(per[i % len(per)] for i in range(ncores))
