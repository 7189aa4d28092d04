"""The replica path of bench.py (one process per GPU, no data-path
collective): whole-job rows/s = all ranks' rows / the slowest rank's time.
Run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, rows = bench.reduce_over_ranks(10.0 * (rank + 1), 1000 + rank, torch.device("cpu"))
    q.put((rank, ms, rows))
    dist.destroy_process_group()


def test_two_ranks_max_time_sum_rows():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 20.0, 2001), (1, 20.0, 2001)]


def test_one_process_unchanged():
    import bench
    assert bench.reduce_over_ranks(3.5, 42, torch.device("cpu")) == (3.5, 42)


def test_traffic_key_ignores_comments_only():
    """The DRAM counters are keyed to the kernel code: comments and layout do
    not change the key, a code change does."""
    import bench
    code = "int f(int a) {\n  return a + 1;  // one more\n}\n/* block\n   comment */\n"
    assert bench._code_only(code) == bench._code_only("int f(int a) {\n\n    return a + 1;\n}\n")
    assert bench._code_only(code) != bench._code_only("int f(int a) {\n  return a + 2;\n}\n")
    assert len(bench.src_sha()) == 16


def test_traffic_keyed_to_the_class_headers(tmp_path, monkeypatch):
    """A class's DRAM counters stay valid while the headers its kernels are
    compiled from keep their code; any other header may change."""
    import bench
    csrc = tmp_path / "paper_2010_00152_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    for f, body in (("sg_common.cuh", "int a;"), ("sg_sortfold.cuh", "int b;"), ("sg_merge.cuh", "int c;"),
                    ("sg_part.cuh", "int d;")):
        (csrc / f).write_text(body)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.src_sha(bench.CLASS_HEADERS["merge"])
    (tmp_path / "profiles" / "traffic.json").write_text(
        '{"merge": {"dram_bytes_per_launch": 123, "src_sha": "%s"}}' % sha)
    assert bench.traffic_for("merge") == 123
    assert bench.traffic_for("rungen") is None                    # no counters for that class
    (csrc / "sg_part.cuh").write_text("int d;  // comment\nint e;")  # a partition kernel changes
    assert bench.traffic_for("merge") == 123
    (csrc / "sg_merge.cuh").write_text("int c2;")                  # the merge kernel changes
    assert bench.traffic_for("merge") is None
