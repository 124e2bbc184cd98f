"""The multi-GPU path's host logic, as two gloo ranks on the CPU.

On several GPUs the bench and a user run one process per GPU, each with its
own model replica on its own rows; the only collectives are the barrier
around the timed region and the max / sum of the ranks' times and rows.
Here two CPU processes (gloo, 127.0.0.1) run the same `replicas.Group` code:
the reductions must give every rank the same max and sum, and row shards
computed separately (with the FP64 oracle standing in for each rank's
forward pass) and gathered must equal the whole batch computed at once.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from paper_2510_19689_b300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))


def _reduce_worker(rank, world, port, out_dir):
    _env(rank, world, port)
    g = replicas.Group("gloo")
    assert (g.world, g.rank) == (world, rank)
    g.barrier()
    ms = 10.0 + 5.0 * rank          # the slower rank decides the job's time
    rows = 1000 * (rank + 1)
    res = dict(max=g.max(ms), sum=g.sum(rows))
    res["value"] = replicas.throughput(res["sum"], res["max"])
    g.barrier()
    g.close()
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([res["max"], res["sum"], res["value"]]))


def _shard_worker(rank, world, port, out_dir):
    _env(rank, world, port)
    import torch.distributed as dist
    from oracle import tabnet_oracle as O
    from paper_2510_19689_b300 import synth
    g = replicas.Group("gloo")
    params = synth.make_params(synth.SPECS["c1"], synth.weight_seed("c1"), bn_affine="random")
    xn, xc = synth.make_rows("c1", 37)
    start, count = replicas.shard(xn.shape[0], g.world, g.rank)
    part = O.forward(params, xn[start:start + count], xc[start:start + count])
    parts = [None] * g.world
    dist.all_gather_object(parts, (start, count, part))
    g.close()
    if rank == 0:
        parts.sort(key=lambda p: p[0])
        lg = np.concatenate([p[2][0] for p in parts])
        mk = np.concatenate([p[2][1] for p in parts])
        ag = np.concatenate([p[2][2] for p in parts])
        np.save(os.path.join(out_dir, "lg.npy"), lg)
        np.save(os.path.join(out_dir, "mk.npy"), mk)
        np.save(os.path.join(out_dir, "ag.npy"), ag)
        np.save(os.path.join(out_dir, "ranges.npy"), np.array([[p[0], p[1]] for p in parts]))


def _run(fn, world, tmp_path):
    mp.start_processes(fn, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")


@pytest.mark.parametrize("total,world", [(0, 1), (1, 2), (7, 2), (65536, 2), (1000003, 8), (3, 4)])
def test_shard_covers_every_row_once(total, world):
    seen = np.zeros(total, dtype=np.int64)
    sizes = []
    for r in range(world):
        start, count = replicas.shard(total, world, r)
        seen[start:start + count] += 1
        sizes.append(count)
    assert (seen == 1).all()
    assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)
    with pytest.raises(ValueError):
        replicas.shard(-1, 2, 0)


def test_single_process_group_needs_no_backend(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    g = replicas.Group()
    assert (g.world, g.rank, g.dist) == (1, 0, None)
    assert g.max(3.5) == 3.5 and g.sum(7) == 7.0
    g.barrier()
    g.close()


def test_two_ranks_reduce_time_and_rows(tmp_path):
    _run(_reduce_worker, 2, tmp_path)
    got = [np.load(tmp_path / f"r{r}.npy") for r in range(2)]
    for g in got:
        assert g[0] == 15.0          # max of 10 and 15 ms
        assert g[1] == 3000.0        # 1000 + 2000 rows
        assert g[2] == pytest.approx(3000.0 / 0.015)
    np.testing.assert_array_equal(got[0], got[1])


def test_two_ranks_sharded_rows_equal_whole_batch(tmp_path):
    from oracle import tabnet_oracle as O
    from paper_2510_19689_b300 import synth
    _run(_shard_worker, 2, tmp_path)
    params = synth.make_params(synth.SPECS["c1"], synth.weight_seed("c1"), bn_affine="random")
    xn, xc = synth.make_rows("c1", 37)
    lg, mk, ag = O.forward(params, xn, xc)
    ranges = np.load(tmp_path / "ranges.npy")
    assert ranges.tolist() == [[0, 19], [19, 18]]
    np.testing.assert_array_equal(np.load(tmp_path / "lg.npy"), lg)
    np.testing.assert_array_equal(np.load(tmp_path / "mk.npy"), mk)
    np.testing.assert_array_equal(np.load(tmp_path / "ag.npy"), ag)
