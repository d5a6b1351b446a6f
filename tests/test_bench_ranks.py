"""Host-side logic of the multi-process benchmark on CPU: two `gloo` ranks.

Each GPU runs an independent replica (a batch of its own images), so the only
exchanges are the barrier around the timed region and the max over ranks of the
measured times; the reported throughput is all ranks' restorations over the
slowest rank's time.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "measured" 100 + 7 r ms for the timed region and 2.5 - r s end to end
    got = bench.reduce_max([100.0 + 7 * rank, 2.5 - rank])
    bench.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [107.0, 2.5]


def test_single_process_reduce_is_identity_and_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3.0, 1.5]) == [3.0, 1.5]
    # 2 ranks x 8 images x 3 steps in 1.5 s (the slowest rank) = 32 restorations/s
    assert bench.job_rate(2, 8 * 3, 1.5) == pytest.approx(32.0)


def test_reference_arm_nonzero_rank_does_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_profiles_traffic_record_parses(tmp_path, monkeypatch):
    """The recorded DRAM traffic is used only while the kernel source it was
    captured from is unchanged."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel")
    rec = tmp_path / "t.md"
    h = hashlib.sha256(b"kernel").hexdigest()
    rec.write_text(f"per_launch_bytes: 12345\nkernel_source_sha256: `{h}`\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    assert bench.recorded_traffic() == 12345.0
    src.write_text("kernel changed")
    assert bench.recorded_traffic() is None
