"""CPU checks of bench.py's multi-process host logic: under torchrun each
rank is an independent replica, joined only by a gloo barrier and a
max-over-ranks of the timings (world size 2, 127.0.0.1)."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    bench = _bench()
    r, w, local = bench.dist_info()
    d = bench.Dist(w)
    d.barrier()
    t_max = d.max(10.0 + 5.0 * r)      # the slower rank sets the time
    same = d.max(3.0)
    d.barrier()
    d.close()
    out.put((r, w, local, t_max, same))


def test_dist_info_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench = _bench()
    assert bench.dist_info() == (0, 1, 0)
    d = bench.Dist(1)  # one rank: no process group, max is the identity
    d.barrier()
    assert d.max(2.5) == 2.5
    d.close()


def test_two_ranks_barrier_and_max_over_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 and r[2] == r[0] for r in res)
    assert all(r[3] == 15.0 for r in res)  # max over ranks, seen by both
    assert all(r[4] == 3.0 for r in res)


def test_reference_arm_runs_on_rank_zero_only():
    bench = _bench()

    class Args:
        pass

    # a rank other than 0 returns at once, without touching the oracle or a GPU
    assert bench.run_reference(Args(), 1, 2) is None


def test_recorded_traffic_keyed_on_the_kernels_own_sources(tmp_path, monkeypatch):
    """profiles/traffic.json holds a kernel's DRAM bytes with a hash of the
    sources that kernel is compiled from: an edit to another CUDA file keeps
    the record, an edit to one of its own sources voids it (the bench then
    reports traffic null)."""
    import json
    import shutil
    bench = _bench()
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_2105_00115_gb300", "csrc"), root / "paper_2105_00115_gb300" / "csrc")
    shutil.copytree(os.path.join(ROOT, "include"), root / "include")
    (root / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.kernel_source_hash("k_onepass_items")
    rec = {"k_onepass_items": {"dram_bytes": 1000.0, "n": 10, "source_hash": h0}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("k_onepass_items", 40) == 4000.0  # scaled by n
    assert bench.recorded_traffic("k_bstream", 40) is None  # no record
    other = root / "paper_2105_00115_gb300" / "csrc" / "qdot_batched.cu"
    other.write_text(other.read_text() + "\n// edit\n")
    assert bench.kernel_source_hash("k_onepass_items") == h0
    assert bench.recorded_traffic("k_onepass_items", 40) == 4000.0
    own = root / "paper_2105_00115_gb300" / "csrc" / "qdot_chunk.cuh"
    own.write_text(own.read_text() + "\n// edit\n")
    assert bench.kernel_source_hash("k_onepass_items") != h0
    assert bench.recorded_traffic("k_onepass_items", 40) is None
