"""Row-band sharding of one join: host logic on CPU (gloo, world_size 2) and
the band option of the CUDA path on one GPU."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1711_07295_b300 import inputs as I
from paper_1711_07295_b300 import shard


def _band_of_pairs(offsets, a, b, r0, r1):
    """Pairs whose later set in size order lies in rows [r0, r1)."""
    sizes = np.diff(offsets)
    order = np.argsort(sizes, kind="stable")
    pos = np.empty(len(order), np.int64)
    pos[order] = np.arange(len(order))
    later = np.maximum(pos[a], pos[b])
    sel = (later >= r0) & (later < r1)
    return a[sel], b[sel]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_band_split_covers_and_balances(world):
    off, tok = I.random_collection(20_000, 4_000, 1, 60, seed=world)
    bands = shard.band_split(off, 1, 2, world)
    assert bands[0][0] == 0 and bands[-1][1] == len(off) - 1
    assert all(bands[k][1] == bands[k + 1][0] for k in range(world - 1))
    w = shard.row_window_counts(shard.sorted_sizes(off), 1, 2)
    loads = [w[r0:r1].sum() for r0, r1 in bands]
    assert sum(loads) == O.filter_counts(off, tok, 1, 2, 64, O.XOR)[0]
    if world > 1:
        assert max(loads) <= 1.05 * (sum(loads) / world) + w.max()


def test_bands_partition_the_oracle_join():
    off, tok = I.random_collection(800, 200, 1, 20, seed=4, planted_frac=0.2)
    a, b = O.self_join(off, tok, 1, 2)
    parts = [_band_of_pairs(off, a, b, r0, r1) for r0, r1 in shard.band_split(off, 1, 2, 3)]
    assert sum(len(x[0]) for x in parts) == len(a)
    ma, mb = shard.merge_pairs(parts)
    assert np.array_equal(ma, a) and np.array_equal(mb, b)


def test_size_buckets_are_row_bands_of_the_larger_set():
    # the precision-by-size study joins one row band per size bucket: the bands
    # tile the rows, and a pair lies in a bucket's band exactly when its larger
    # set's size is in the bucket
    from paper_1711_07295_b300.study_filter_ratio import size_band_rows
    off, tok = I.random_collection(1_500, 300, 1, 40, seed=6, planted_frac=0.3)
    sizes = np.diff(off)
    bands = size_band_rows(sizes, (1, 4, 9, 10, 25, 60))
    assert bands[0][2] == 0 and bands[-1][3] == len(sizes)
    assert all(bands[k][3] == bands[k + 1][2] for k in range(len(bands) - 1))
    a, b = O.self_join(off, tok, 1, 2)
    larger = np.maximum(sizes[a], sizes[b])
    total = 0
    for lo, hi, r0, r1 in bands:
        ba, bb = _band_of_pairs(off, a, b, r0, r1)
        lb = np.maximum(sizes[ba], sizes[bb])
        assert np.all(lb >= lo) and (hi is None or np.all(lb < hi))
        want = np.count_nonzero((larger >= lo) & ((larger < hi) if hi is not None else True))
        assert len(ba) == want
        total += len(ba)
    assert total == len(a) > 0


@pytest.mark.parametrize("world", [1, 2, 5])
def test_rs_split_partitions_the_oracle_rs_join(world):
    # the ranks' ranges of R cover R, carry about equal window pairs, and their
    # RS-joins with all of S (R ids offset back) merge into the full RS-join
    off, tok = I.random_collection(1500, 300, 1, 25, seed=20 + world, planted_frac=0.2)
    ro, rt = off[:601].copy(), tok[:off[600]].copy()
    so, st = off[600:] - off[600], tok[off[600]:].copy()
    parts_r = shard.rs_split(ro, so, 3, 5, world)
    assert parts_r[0][0] == 0 and parts_r[-1][1] == 600
    assert all(parts_r[k][1] == parts_r[k + 1][0] for k in range(world - 1))
    w = shard.rs_row_windows(ro, so, 3, 5)
    assert w.sum() == O.rs_filter_counts(ro, rt, so, st, 3, 5, 64, O.XOR)[0]
    if world > 1:
        loads = [w[a:b].sum() for a, b in parts_r]
        assert max(loads) <= 1.05 * (w.sum() / world) + w.max()
    parts = []
    for r0, r1 in parts_r:
        po, pt = shard.rs_part(ro, rt, r0, r1)
        a, b = O.rs_join(po, pt, so, st, 3, 5)
        parts.append((a + np.uint32(r0), b))
    ma, mb = shard.merge_pairs(parts)
    fa, fb = O.rs_join(ro, rt, so, st, 3, 5)
    assert np.array_equal(ma, fa) and np.array_equal(mb, fb) and len(fa) > 0


def _gloo_worker(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off, tok = I.random_collection(1200, 300, 1, 25, seed=9, planted_frac=0.2)
    r0, r1 = shard.band_split(off, 3, 5, world)[rank]
    full_a, full_b = O.self_join(off, tok, 3, 5)
    a, b = _band_of_pairs(off, full_a, full_b, r0, r1)   # this rank's share, computed on the CPU
    ma, mb = shard.gather_pairs(a, b)
    if rank == 0:
        ok = np.array_equal(ma, full_a) and np.array_equal(mb, full_b)
        with open(result_path, "w") as f:
            f.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def _gloo_big_worker(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # 1,700 copies of one set (C(1700, 2) = 1,444,150 similar pairs) among random sets
    off, tok = I.random_collection(1200, 300, 1, 25, seed=19, planted_frac=0.2)
    sets = [tok[off[i]:off[i + 1]] for i in range(len(off) - 1)]
    sets += [np.array([4, 9, 17], np.int32)] * 1700
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in sets])
    tok = np.concatenate(sets).astype(np.int32)
    full_a, full_b = O.self_join(off, tok, 3, 5)
    r0, r1 = shard.band_split(off, 3, 5, world)[rank]
    a, b = _band_of_pairs(off, full_a, full_b, r0, r1)
    ma, mb = shard.gather_pairs(a, b)                 # every rank gets the merged list
    ok = len(full_a) > 1_000_000 and np.array_equal(ma, full_a) and np.array_equal(mb, full_b)
    got = shard.gather_pairs(a, b, dst=0)             # rank 0 only
    if rank == 0:
        ok = ok and np.array_equal(got[0], full_a) and np.array_equal(got[1], full_b)
    else:
        ok = ok and got is None
    oks = [None] * world
    dist.all_gather_object(oks, ok)
    if rank == 0:
        with open(result_path, "w") as f:
            f.write("ok" if all(oks) else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_gather_a_million_pairs(tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    path = str(tmp_path / "result.txt")
    mp.spawn(_gloo_big_worker, args=(2, port, path), nprocs=2, join=True)
    assert open(path).read() == "ok"


def test_gloo_two_ranks_gather(tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    path = str(tmp_path / "result.txt")
    mp.spawn(_gloo_worker, args=(2, port, path), nprocs=2, join=True)
    assert open(path).read() == "ok"


@pytest.mark.gpu
def test_gpu_bands_merge_to_full_join():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1711_07295_b300 import _bmj
    off, tok = I.random_collection(9000, 2000, 1, 50, seed=12, planted_frac=0.1)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    fa, fb, fst = _bmj.bmj_self_join(d_off, d_tok, 1, 2)
    for world in (2, 3, 5):
        parts, win, surv = [], 0, 0
        for r in range(world):
            a, b, st = shard.sharded_self_join(d_off, d_tok, 1, 2, r, world)
            parts.append((a, b))
            win += st["window_pairs"]
            surv += st["survivors"]
        ma, mb = shard.merge_pairs(parts)
        assert np.array_equal(ma, fa) and np.array_equal(mb, fb)
        assert (win, surv) == (fst["window_pairs"], fst["survivors"])
    with pytest.raises(_bmj.BmjError):
        _bmj.bmj_self_join(d_off, d_tok, 1, 2, row_begin=5, row_end=4)


@pytest.mark.gpu
def test_gpu_rs_parts_merge_to_full_rs_join():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1711_07295_b300 import _bmj
    off, tok = I.random_collection(9000, 2000, 1, 50, seed=13, planted_frac=0.15)
    ro, rt = off[:4001].copy(), tok[:off[4000]].copy()
    so, st_ = off[4000:] - off[4000], tok[off[4000]:].copy()
    fa, fb, fst = _bmj.bmj_rs_join(ro, rt, so, st_, 3, 5)
    for world in (2, 3):
        parts, win = [], 0
        for r in range(world):
            a, b, st = shard.sharded_rs_join(ro, rt, so, st_, 3, 5, r, world)
            parts.append((a, b))
            win += st["window_pairs"]
        ma, mb = shard.merge_pairs(parts)
        assert np.array_equal(ma, fa) and np.array_equal(mb, fb) and len(fa) > 0
        assert win == fst["window_pairs"]
