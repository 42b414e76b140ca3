"""The bench's host logic on CPU: multi-rank timing on gloo ranks (world
size 2) -- the job's time is the slowest rank's, its value counts every
rank's cells, the reference arm runs on rank 0 only -- and the code hash
that ties a DRAM traffic record to its kernel.  Every rank of the GPU path runs an
independent replica (no data-path collective), so this is the whole N > 1
logic."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.slowest_rank_ms(10.0 + 5.0 * rank)   # rank 1 is the slow one
        q.put((rank, ms, bench.job_gcups(2e9, world, ms), bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_cells():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [g[0] for g in got] == [0, 1]
    for rank, ms, val, env in got:
        assert ms == 15.0
        assert val == pytest.approx(2 * 2e9 / 15e-3 / 1e9)
        assert env == (rank, 2, rank)
    assert all(p.exitcode == 0 for p in procs)


def test_single_process_time_is_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(12.5) == 12.5
    assert bench.job_gcups(1e9, 1, 1000.0) == pytest.approx(1.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(workload="band", gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""


def test_traffic_records_ignore_comment_edits_only(tmp_path):
    """The DRAM traffic the bench reports stays tied to the kernel's code: a
    comment edit keeps the record's hash, a code edit changes it."""
    sys.path.insert(0, ROOT)
    import bench
    f = tmp_path / "k.cu"
    f.write_text('__global__ void k(int *p) { p[0] = 1; }  // one\n/* two */\nconst char *s = "//x";\n')
    h0 = bench.sources_sha([str(f)])
    f.write_text('// a new header comment\n__global__ void k(int *p) { p[0] = 1; }  // edited\n'
                 'const char *s = "//x";\n')
    assert bench.sources_sha([str(f)]) == h0
    f.write_text('__global__ void k(int *p) { p[0] = 2; }\nconst char *s = "//x";\n')
    assert bench.sources_sha([str(f)]) != h0


def test_traffic_record_of_a_region_ignores_the_rest_of_its_file(tmp_path):
    """A record that covers one kernel's region of a file (`path#from..to`)
    keeps its hash when code outside the region changes and loses it when
    the region's code changes or its markers are gone."""
    sys.path.insert(0, ROOT)
    import bench
    f = tmp_path / "k.cu"
    src = lambda fill, walk: (f"struct Args {{ int x; }};\n__global__ void fill(int *p) {{ p[0] = {fill}; }}\n"
                              f"struct WalkTask {{ int y; }};\n__global__ void walk(int *p) {{ p[1] = {walk}; }}\n")
    spec = [str(f) + "#struct Args {..struct WalkTask {"]
    f.write_text(src(1, 1))
    h0 = bench.sources_sha(spec)
    f.write_text(src(1, 2))  # the walk changed: not in the region
    assert bench.sources_sha(spec) == h0
    f.write_text(src(2, 2))  # the fill changed
    assert bench.sources_sha(spec) != h0
    f.write_text(src(1, 1).replace("struct WalkTask", "struct Other"))
    assert bench.sources_sha(spec) != h0
    assert bench.source_region("a\nb\nc\n", "a..c") == "a\nb"


def test_clock_summary_keeps_the_timed_window_and_reasons():
    """The bench's clock record: only samples inside the timed window count,
    the median SM clock and the active throttle reasons are reported."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = [(0.5, "1200, 2070, 900.1, Not Active, Not Active, Not Active, Active"),     # before the window
               (1.1, "2070, 2070, 1300.0, Not Active, Not Active, Not Active, Not Active"),
               (1.2, "2055, 2070, 1350.5, Not Active, Not Active, Not Active, Active"),
               (1.3, "2070, 2070, 1390.2, Not Active, Not Active, Not Active, Not Active"),
               (1.35, "garbage line"),
               (9.0, "300, 2070, 100.0, Active, Not Active, Not Active, Not Active")]      # after it
    c.window(1.0, 1.3)
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
