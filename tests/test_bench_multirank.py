"""The benchmark's multi-process path on CPU: two gloo ranks, each timing its
own replica; the job time is the slowest rank's and the throughput counts
the cells of every rank (weak scaling, replicas only)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.max_over_ranks(10.0 + 3.0 * rank)
    out[rank] = (m, bench.job_mlups(1000, world, 5, m / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == pytest.approx(13.0) and res[1][0] == pytest.approx(13.0)
    assert res[0][1] == pytest.approx(1000 * 2 * 5 / 0.013 / 1e6)


def test_reference_arm_other_ranks_do_nothing():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    class A:
        workload = "perf512_spinodal_f32"
        steps = 1
        warmup = 0
        gpus = 2
        storage = None
    assert bench.run_reference(A(), rank=1, world=2) is None


def test_reference_arm_line_on_cpu():
    """The reference arm runs without a GPU: the oracle on every host core,
    one JSON line with the contract's keys, its value the aggregate over the
    processes."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_kernel_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The committed DRAM-traffic figure stays valid across comment edits of
    the kernel's sources and is dropped after any code edit."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    csrc = tmp_path / "paper_1601_01237_gb300" / "csrc"
    csrc.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SOURCES, "k_probe", ("a.cu",))
    (csrc / "a.cu").write_text("// one\nint f() { return 1; }  /* x */\n")
    h0 = bench.kernel_source_hash("k_probe")
    (csrc / "a.cu").write_text("// two, longer\n\nint f() { return 1; }  /* y\n z */\n")
    assert bench.kernel_source_hash("k_probe") == h0
    (csrc / "a.cu").write_text("// one\nint f() { return 2; }\n")
    assert bench.kernel_source_hash("k_probe") != h0
