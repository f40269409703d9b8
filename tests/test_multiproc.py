"""Multi-process path of bench.py on the host (gloo, world size 2): instance sharding, the
max over ranks of the step time, and the reference arm under torchrun (rank 0 alone prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_range_partitions_every_unit_once():
    for n in [0, 1, 7, 8192, 8193]:
        for world in [1, 2, 3, 8]:
            got = [bench.shard_range(n, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            for (a, b), (c, d) in zip(got, got[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench as b
    w, r, _, pg = b.dist_setup(None)
    lo, hi = b.shard_range(8192, r, w)
    m = b.max_over_ranks(float(r) + 0.5, pg)
    b.barrier(pg)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "lo": lo, "hi": hi, "max": m}, f)
    pg.destroy_process_group()


def test_gloo_world2_sharding_and_max(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if torch.cuda.is_available():
        pytest.skip("the host-only (gloo) path is exercised where no GPU is visible")
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [x["world"] for x in res] == [2, 2]
    assert res[0]["lo"] == 0 and res[0]["hi"] == res[1]["lo"] and res[1]["hi"] == 8192
    assert all(x["max"] == 1.5 for x in res)


def test_reference_arm_under_torchrun_prints_once():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("the host-only (gloo) path is exercised where no GPU is visible")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--ref-sample", "6"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
