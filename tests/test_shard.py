"""Sets sharded across ranks: the range planner, and two gloo ranks on CPU whose gathered
likelihoods equal a single process's (the oracle evaluates the sets; Philox counters carry the
set id, so the sharded values are identical, not merely close)."""
import dataclasses
import os
import socket
import tempfile
from datetime import timedelta

import numpy as np
import pytest

import oracle as O
from paper_1904_00011_gb300 import shard
from paper_1904_00011_gb300 import workloads as W


def test_plan_contiguous_cover_and_balance():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        for n in (0, 1, 5, 37, 512):
            c = rng.uniform(0.1, 5.0, size=n)
            rs = shard.plan(c, world)
            assert len(rs) == world
            b = 0
            for lo, hi in rs:
                assert lo == b and hi >= lo
                b = hi
            assert b == n
            if n:
                share = c.sum() / world
                for lo, hi in rs:
                    assert c[lo:hi].sum() <= share + c.max() + 1e-9


def test_plan_edge_cases():
    rs = shard.plan([1.0] * 3, 5)          # more ranks than sets: some ranges are empty
    assert sum(hi - lo for lo, hi in rs) == 3 and max(hi - lo for lo, hi in rs) == 1
    assert shard.plan([0.0, 0.0], 2) == [(0, 1), (1, 2)]
    assert shard.plan([5.0, 0.0, 0.0, 0.0], 2)[0][0] == 0
    with pytest.raises(ValueError):
        shard.plan([1.0, -1.0], 2)
    with pytest.raises(ValueError):
        shard.plan([1.0, float("nan")], 2)
    with pytest.raises(ValueError):
        shard.plan([1.0], 0)


def test_single_rank_without_process_group_calls_once():
    calls = []

    def ev(p, n, fid):
        calls.append((len(p), fid))
        return np.arange(len(p), dtype=np.float64) + fid

    out = shard.evaluate_sharded(ev, [None] * 4, [16, 32, 16, 48], first_set_id=10)
    assert calls == [(4, 10)]
    assert np.array_equal(out, [10.0, 11.0, 12.0, 13.0])


def _workload():
    return W.batch(seed=9, n_sets=5, n_min=16, n_max=48, step=16)


def _mock(w):
    wm = dataclasses.replace(w, params=[W.batch_mock_params()], n_ims=[32], n_im=32)
    return O.model(wm, 0, set_id=999_999)


def _oracle_eval(w, mock, params, n_ims, first_id):
    out = []
    for k, (p, n) in enumerate(zip(params, n_ims)):
        wk = dataclasses.replace(w, params=[p], n_ims=[n], n_im=n)
        m = O.model(wk, 0, set_id=first_id + k)
        out.append(O.loglike(m["hist"], m["moments"], n * n, mock["hist"], mock["moments"],
                             mock["n_pix"], mode=W.LL_POISSON))
    return np.array(out)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=120))
    try:
        w = _workload()
        mock = _mock(w)
        seen = []

        def ev(p, n, fid):
            seen.append((fid, len(p)))
            return _oracle_eval(w, mock, p, n, fid)

        ll = shard.evaluate_sharded(ev, w.params, w.n_ims, first_set_id=7)
        np.save(os.path.join(out_dir, "ll%d.npy" % rank), ll)
        np.save(os.path.join(out_dir, "seen%d.npy" % rank), np.array(seen, np.int64).reshape(-1, 2))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_equal_single_process():
    import torch.multiprocessing as mp
    O.build()
    w = _workload()
    whole = _oracle_eval(w, _mock(w), w.params, w.n_ims, 7)
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True,
                           start_method="spawn")
        ll0 = np.load(os.path.join(d, "ll0.npy"))
        ll1 = np.load(os.path.join(d, "ll1.npy"))
        seen = [np.load(os.path.join(d, "seen%d.npy" % r)) for r in range(2)]
    assert np.array_equal(ll0, whole) and np.array_equal(ll1, whole)
    # each rank evaluated its own contiguous range once, with the global set ids
    ranges = shard.plan(shard.set_costs(w.n_ims), 2)
    for r in range(2):
        b, e = ranges[r]
        exp = [(7 + b, e - b)] if e > b else []
        assert [tuple(x) for x in seen[r]] == exp
    assert sum(len(s) for s in seen) == 2
